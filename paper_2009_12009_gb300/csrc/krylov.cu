// krylov.cu -- vector kernels of the top-level Krylov solvers (Sec. "Linear Solvers": native
// CG and BiCG solvers next to multigrid): the operator applied to a vector in one pass, and
// the fused vector updates of BiCGStab.  FP64; flat kernels run over every element of a
// level-0 field (ghosts and padding included, which carry no meaning), so they need no
// work list.
#include <algorithm>

#include "kernels.h"

namespace gmg {
namespace {

constexpr int KT = 256;

// out = A in on the valid cells: D in - sum over the six faces of w_f in_nbr (the ghosts of
// `in` filled first); one thread per cell
__global__ void __launch_bounds__(KT)
    k_apply(const DevBox* __restrict__ boxes, const Chunk* __restrict__ chunks, const double* __restrict__ in,
            const double* __restrict__ wx, const double* __restrict__ wy, const double* __restrict__ wz,
            const double* __restrict__ D, double* __restrict__ out) {
  const Chunk ch = chunks[blockIdx.x];
  const DevBox B = boxes[ch.item];
  const int t = ch.start + threadIdx.x;
  if (t >= B.nx * B.ny * B.nz) return;
  const int i = t % B.nx, j = (t / B.nx) % B.ny, k = t / (B.nx * B.ny);
  const int64_t q = elem_index(B, i, j, k);
  const int64_t sx = B.sx, sy = B.sy;
  double v = __ldg(D + q) * in[q];
  v = fma(-__ldg(wx + q), in[q - 1], v);
  v = fma(-__ldg(wx + q + 1), in[q + 1], v);
  v = fma(-__ldg(wy + q), in[q - sx], v);
  v = fma(-__ldg(wy + q + sx), in[q + sx], v);
  v = fma(-__ldg(wz + q), in[q - sy], v);
  v = fma(-__ldg(wz + q + sy), in[q + sy], v);
  out[q] = v;
}

// p = r + beta (p - omega v)
__global__ void k_bicg_direction(int64_t n, const double* __restrict__ r, double* __restrict__ p,
                                 const double* __restrict__ v, double beta, double omega) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = r[i] + beta * (p[i] - omega * v[i]);
}

// x += a y + b z
__global__ void k_add2(int64_t n, double* __restrict__ x, double a, const double* __restrict__ y, double b,
                       const double* __restrict__ z) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    x[i] += a * y[i] + b * z[i];
}

unsigned flat_grid(int64_t n) { return (unsigned)std::min<int64_t>((n + KT - 1) / KT, 152 * 16); }

// ---- one launch over every level of a composite vector: block ranges [b0[l], b0[l + 1])
// take level l, each with the grid-stride loop of the one-level kernel over its elements,
// and the same expression per element, so every value is bitwise that of one launch per level.

struct MlFlat {
  int nl;
  int64_t n[ML_MAX_SEG];
  int b0[ML_MAX_SEG + 1];
};
struct MlPtrs {
  const double* p[ML_MAX_SEG];
};
struct MlOut {
  double* p[ML_MAX_SEG];
};
struct MlScal {
  double a[ML_MAX_SEG], b[ML_MAX_SEG];
};

MlFlat ml_flat(int nl, const int64_t* n) {
  MlFlat F{};
  F.nl = nl;
  F.b0[0] = 0;
  for (int l = 0; l < nl; ++l) {
    F.n[l] = n[l];
    F.b0[l + 1] = F.b0[l] + (int)std::max<unsigned>(1, flat_grid(n[l]));  // each level: the one-level grid
  }
  return F;
}

// the level of this block, its first element and the stride of its range (the launch
// structs are __grid_constant__: indexed in parameter space, never copied per thread)
__device__ __forceinline__ int ml_level(const MlFlat& F, int64_t& i0, int64_t& stride) {
  int l = 0;
  while (l + 1 < F.nl && (int)blockIdx.x >= F.b0[l + 1]) ++l;
  i0 = (int64_t)(blockIdx.x - F.b0[l]) * KT + threadIdx.x;
  stride = (int64_t)(F.b0[l + 1] - F.b0[l]) * KT;
  return l;
}

// out_l = a_l x_l + b_l y_l (k_axpby's expression)
__global__ void k_axpby_ml(const __grid_constant__ MlFlat F, const __grid_constant__ MlPtrs x, const __grid_constant__ MlPtrs y, const __grid_constant__ MlOut out, const __grid_constant__ MlScal ab) {
  int64_t i0, st;
  const int l = ml_level(F, i0, st);
  const double a = ab.a[l], b = ab.b[l];
  const double* __restrict__ xl = x.p[l];
  const double* __restrict__ yl = y.p[l];
  double* __restrict__ ol = out.p[l];
  for (int64_t i = i0; i < F.n[l]; i += st) ol[i] = a * xl[i] + b * yl[i];
}

// o1_l = a_l x_l + 0 x_l, then o2_l = 1 o1_l + 0 o1_l: the values of two k_axpby passes (the
// second copying the first's output), in one
__global__ void k_scale2_ml(const __grid_constant__ MlFlat F, const __grid_constant__ MlPtrs x, const __grid_constant__ MlOut o1, const __grid_constant__ MlOut o2, const __grid_constant__ MlScal ab) {
  int64_t i0, st;
  const int l = ml_level(F, i0, st);
  const double a = ab.a[l], b = ab.b[l], one = 1.0;
  const double* __restrict__ xl = x.p[l];
  double* __restrict__ p1 = o1.p[l];
  double* __restrict__ p2 = o2.p[l];
  for (int64_t i = i0; i < F.n[l]; i += st) {
    const double v = a * xl[i] + b * xl[i];
    p1[i] = v;
    p2[i] = one * v + b * v;
  }
}

// p_l = r_l + beta (p_l - omega v_l)
__global__ void k_bicg_direction_ml(const __grid_constant__ MlFlat F, const __grid_constant__ MlPtrs r, const __grid_constant__ MlOut p, const __grid_constant__ MlPtrs v, double beta,
                                    double omega) {
  int64_t i0, st;
  const int l = ml_level(F, i0, st);
  const double* __restrict__ rl = r.p[l];
  double* __restrict__ pl = p.p[l];
  const double* __restrict__ vl = v.p[l];
  for (int64_t i = i0; i < F.n[l]; i += st) pl[i] = rl[i] + beta * (pl[i] - omega * vl[i]);
}

// x_l += a y_l + b z_l
__global__ void k_add2_ml(const __grid_constant__ MlFlat F, const __grid_constant__ MlOut x, double a, const __grid_constant__ MlPtrs y, double b, const __grid_constant__ MlPtrs z) {
  int64_t i0, st;
  const int l = ml_level(F, i0, st);
  double* __restrict__ xl = x.p[l];
  const double* __restrict__ yl = y.p[l];
  const double* __restrict__ zl = z.p[l];
  for (int64_t i = i0; i < F.n[l]; i += st) xl[i] += a * yl[i] + b * zl[i];
}

// valid-cell reductions over segments (a level and its vectors): chunk ranges [c0[s], c0[s+1])
constexpr int ML_CPB = 4;  // cell chunks per block of the dot product
struct MlCells {
  int ns;
  const DevBox* boxes[ML_MAX_SEG];
  const Chunk* chunks[ML_MAX_SEG];
  const double* x[ML_MAX_SEG];
  const double* y[ML_MAX_SEG];
  int nch[ML_MAX_SEG];   // cell chunks of the segment's level
  int c0[ML_MAX_SEG + 1];  // first block of each segment
};

__device__ __forceinline__ int ml_seg(const MlCells& M) {
  int s = 0;
  while (s + 1 < M.ns && (int)blockIdx.x >= M.c0[s + 1]) ++s;
  return s;
}

// Partial sums of x y: block b of a segment adds the cells of its cell chunks
// [ML_CPB b, ML_CPB (b + 1)), each thread one cell per chunk (the chunks' loads in flight
// together), then the warp and block sums in a fixed order.  Deterministic; the partials
// differ from one block per chunk only in the order of the additions.
__global__ void __launch_bounds__(KT) k_dot_partial_ml(const __grid_constant__ MlCells M, double* partials) {
  __shared__ double red[KT / 32];
  const int sg = ml_seg(M);
  const int b = blockIdx.x - M.c0[sg];
  double v = 0.0;
#pragma unroll
  for (int u = 0; u < ML_CPB; ++u) {
    const int c = ML_CPB * b + u;
    if (c >= M.nch[sg]) break;
    const Chunk ch = M.chunks[sg][c];
    const DevBox B = M.boxes[sg][ch.item];
    const int t = ch.start + threadIdx.x;
    if (t < B.nx * B.ny * B.nz) {
      const int i = t % B.nx, j = (t / B.nx) % B.ny, k = t / (B.nx * B.ny);
      const int64_t q = elem_index(B, i, j, k);
      v += M.x[sg][q] * M.y[sg][q];
    }
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < KT / 32; ++w) s += red[w];
    partials[blockIdx.x] = s;
  }
}

// block s adds segment s's partials (k_reduce_sum's order) into out[s]
__global__ void __launch_bounds__(KT) k_reduce_sum_ml(const __grid_constant__ MlCells M, const double* __restrict__ partials,
                                                      double* out) {
  __shared__ double red[KT / 32];
  const int sg = blockIdx.x;
  const double* pp = partials + M.c0[sg];
  const int n = M.c0[sg + 1] - M.c0[sg];
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += KT) v += pp[i];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < KT / 32; ++w) s += red[w];
    out[sg] = s;
  }
}

// max |x| over the valid cells of segment s into maxbits[s] (IEEE bits, integer max)
__global__ void __launch_bounds__(KT) k_norm_max_ml(const __grid_constant__ MlCells M, unsigned long long* maxbits) {
  __shared__ unsigned long long red[KT / 32];
  const int sg = ml_seg(M);
  const Chunk ch = M.chunks[sg][blockIdx.x - M.c0[sg]];
  const DevBox B = M.boxes[sg][ch.item];
  const int t = ch.start + threadIdx.x;
  unsigned long long v = 0;
  if (t < B.nx * B.ny * B.nz) {
    const int i = t % B.nx, j = (t / B.nx) % B.ny, k = t / (B.nx * B.ny);
    v = (unsigned long long)__double_as_longlong(M.x[sg][elem_index(B, i, j, k)]) & 0x7fffffffffffffffULL;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long w = __shfl_down_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < KT / 32 ? red[threadIdx.x] : 0ULL;
    for (int o = 16; o > 0; o >>= 1) {
      const unsigned long long w = __shfl_down_sync(0xffffffffu, v, o);
      v = w > v ? w : v;
    }
    if (threadIdx.x == 0 && v) atomicMax(maxbits + sg, v);
  }
}

// segments of chunks_per_block cell chunks per block
MlCells ml_cells(int ns, const LevelDev* const* L, const double* const* x, const double* const* y,
                 int chunks_per_block) {
  MlCells M{};
  M.ns = ns;
  M.c0[0] = 0;
  for (int s = 0; s < ns; ++s) {
    M.boxes[s] = L[s]->boxes;
    M.chunks[s] = L[s]->cell_chunks;
    M.x[s] = x[s];
    M.y[s] = y ? y[s] : nullptr;
    M.nch[s] = L[s]->n_cell_chunks;
    M.c0[s + 1] = M.c0[s] + (L[s]->n_cell_chunks + chunks_per_block - 1) / chunks_per_block;
  }
  return M;
}

}  // namespace

void launch_apply(const LevelDev& L, const double* in, const Coefs& c64, double* out, cudaStream_t s) {
  if (!L.n_cell_chunks) return;
  count_launches(1);
  k_apply<<<L.n_cell_chunks, KT, 0, s>>>(L.boxes, L.cell_chunks, in, (const double*)c64.wx, (const double*)c64.wy,
                                         (const double*)c64.wz, (const double*)c64.D, out);
}

void launch_bicg_direction(int64_t n, const double* r, double* p, const double* v, double beta, double omega,
                           cudaStream_t s) {
  if (n <= 0) return;
  count_launches(1);
  k_bicg_direction<<<flat_grid(n), KT, 0, s>>>(n, r, p, v, beta, omega);
}

void launch_add2(int64_t n, double* x, double a, const double* y, double b, const double* z, cudaStream_t s) {
  if (n <= 0) return;
  count_launches(1);
  k_add2<<<flat_grid(n), KT, 0, s>>>(n, x, a, y, b, z);
}

namespace {
template <class P>
P ml_pack(int nl, const double* const* v) {
  P o{};
  for (int l = 0; l < nl; ++l) o.p[l] = const_cast<double*>(v[l]);
  return o;
}
}  // namespace

void launch_axpby_ml(int nl, const int64_t* n, const double* a, const double* const* x, const double* b,
                     const double* const* y, double* const* out, cudaStream_t s) {
  if (nl <= 0) return;
  const MlFlat F = ml_flat(nl, n);
  MlScal ab{};
  for (int l = 0; l < nl; ++l) {
    ab.a[l] = a[l];
    ab.b[l] = b[l];
  }
  count_launches(1);
  k_axpby_ml<<<F.b0[nl], KT, 0, s>>>(F, ml_pack<MlPtrs>(nl, x), ml_pack<MlPtrs>(nl, y),
                                       ml_pack<MlOut>(nl, (const double* const*)out), ab);
}

void launch_scale2_ml(int nl, const int64_t* n, const double* a, const double* const* x, double* const* o1,
                      double* const* o2, cudaStream_t s) {
  if (nl <= 0) return;
  const MlFlat F = ml_flat(nl, n);
  MlScal ab{};
  for (int l = 0; l < nl; ++l) {
    ab.a[l] = a[l];
    ab.b[l] = 0.0;
  }
  count_launches(1);
  k_scale2_ml<<<F.b0[nl], KT, 0, s>>>(F, ml_pack<MlPtrs>(nl, x), ml_pack<MlOut>(nl, (const double* const*)o1),
                                        ml_pack<MlOut>(nl, (const double* const*)o2), ab);
}

void launch_bicg_direction_ml(int nl, const int64_t* n, const double* const* r, double* const* p,
                              const double* const* v, double beta, double omega, cudaStream_t s) {
  if (nl <= 0) return;
  const MlFlat F = ml_flat(nl, n);
  count_launches(1);
  k_bicg_direction_ml<<<F.b0[nl], KT, 0, s>>>(F, ml_pack<MlPtrs>(nl, r), ml_pack<MlOut>(nl, (const double* const*)p),
                                                ml_pack<MlPtrs>(nl, v), beta, omega);
}

void launch_add2_ml(int nl, const int64_t* n, double* const* x, double a, const double* const* y, double b,
                    const double* const* z, cudaStream_t s) {
  if (nl <= 0) return;
  const MlFlat F = ml_flat(nl, n);
  count_launches(1);
  k_add2_ml<<<F.b0[nl], KT, 0, s>>>(F, ml_pack<MlOut>(nl, (const double* const*)x), a, ml_pack<MlPtrs>(nl, y), b,
                                      ml_pack<MlPtrs>(nl, z));
}

void launch_dot_ml(int ns, const LevelDev* const* L, const double* const* x, const double* const* y,
                   double* partials, double* out, cudaStream_t s) {
  if (ns <= 0) return;
  const MlCells M = ml_cells(ns, L, x, y, ML_CPB);
  if (M.c0[ns] == 0) return;
  count_launches(2);
  k_dot_partial_ml<<<M.c0[ns], KT, 0, s>>>(M, partials);
  k_reduce_sum_ml<<<ns, KT, 0, s>>>(M, partials, out);
}

void launch_norm_max_ml(int ns, const LevelDev* const* L, const double* const* x, unsigned long long* maxbits,
                        cudaStream_t s) {
  if (ns <= 0) return;
  const MlCells M = ml_cells(ns, L, x, nullptr, 1);
  if (M.c0[ns] == 0) return;
  count_launches(1);
  k_norm_max_ml<<<M.c0[ns], KT, 0, s>>>(M, maxbits);
}

}  // namespace gmg
