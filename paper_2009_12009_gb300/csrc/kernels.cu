// kernels.cu -- sm_103a kernels of the multigrid V-cycle.
//
// Every kernel reads a work list of Chunk entries (box, first item) built once on the
// host, so one launch covers all boxes of a level (the fused launch of Sec.
// "Communication" applied to every step, not only to ghost exchange).  Arithmetic is
// double for double fields and float for float / bfloat16 fields.
#include <cuda_bf16.h>

#include <algorithm>
#include <type_traits>
#include <utility>

#include "dev_util.cuh"

namespace gmg {
namespace {

// |v| as ordered bits: for non-negative doubles the IEEE bit pattern is monotone, and a
// NaN (all exponent bits set, nonzero mantissa) compares above +inf, so the max of the
// bits is the max of |v| with NaN propagating.  Integer max keeps the FP64 pipe free.
__device__ __forceinline__ unsigned long long abs_bits(double v) {
  return (unsigned long long)__double_as_longlong(v) & 0x7fffffffffffffffULL;
}

__device__ __forceinline__ void block_max_atomic(unsigned long long v, unsigned long long* out) {
  __shared__ unsigned long long red[BLOCK / 32];
  for (int o = 16; o > 0; o >>= 1) {
    unsigned long long w = __shfl_down_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < (BLOCK / 32) ? red[threadIdx.x] : 0ULL;
    for (int o = 16; o > 0; o >>= 1) {
      unsigned long long w = __shfl_down_sync(0xffffffffu, v, o);
      v = w > v ? w : v;
    }
    if (threadIdx.x == 0 && v) atomicMax(out, v);
  }
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[BLOCK / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < BLOCK / 32; ++w) s += red[w];
  return s;  // valid in thread 0
}

// ---------------------------------------------------------------- ghost exchange

template <class T>
__global__ void __launch_bounds__(BLOCK) k_fill(const DevBox* __restrict__ boxes, const GhostRect* __restrict__ rects,
                                                const Chunk* __restrict__ chunks, T* f, int colour, int copy_mode,
                                                const int* __restrict__ active) {
  pdl_enter();
  const Chunk ch = chunks[blockIdx.x];
  const GhostRect g = rects[ch.item];
  if (copy_mode == 1 && g.kind != 0) return;
  const DevBox Bd = boxes[g.dst_box];
  if (active && !active[Bd.solve]) return;
  const DevBox Bs = boxes[g.src_box];
  const int64_t d0 = elem_index(Bd, g.dst[0], g.dst[1], g.dst[2]);
  const int64_t s0 = elem_index(Bs, g.src[0], g.src[1], g.src[2]);
  const int64_t du = axis_stride(Bd, g.d1), dv = axis_stride(Bd, g.d2);
  const int64_t su = axis_stride(Bs, g.d1), sv = axis_stride(Bs, g.d2);
  const int n = g.n1 * g.n2;
  const int end = min(n, ch.start + GHOST_CHUNK);
  for (int e = ch.start + threadIdx.x; e < end; e += BLOCK) {
    const int u = e % g.n1, v = e / g.n1;
    if (colour >= 0 && ((g.par0 + u + v) & 1) != colour) continue;
    const auto val = ld(f + s0 + u * su + v * sv);
    if (g.kind == 2)  // quadratic wall: a third of the second cell inward (0 for the transpose)
      st(f + d0 + u * du + v * dv, copy_mode == 2 ? (decltype(val))0 : val * (decltype(val))(1.0 / 3.0));
    else
      st(f + d0 + u * du + v * dv, g.sign < 0 ? -val : val);
  }
}

// ------------------------------------------------------------ red-black smoother

// resident blocks per SM the smoothers' register count must allow: 8 (32 registers) for float
// and bfloat16, whose passes are bound by latency more than by bytes; no bound for double
// (measured: held to 40 registers its finest-level pass took 167.8 us instead of 152.9)
template <class T> struct SmoothMinB { static constexpr int value = 8; };
template <> struct SmoothMinB<double> { static constexpr int value = 0; };

// One colour of Gauss-Seidel: each thread owns a pair of x-adjacent cells and updates
// the one whose global (i+j+k) parity is `colour`:
//   phi = invD * (rhs + sum_f w_f phi_nbr)          (7 FMA-pipe operations)
template <class T>
__global__ void __launch_bounds__(BLOCK, SmoothMinB<T>::value)
    k_smooth(const DevBox* __restrict__ boxes, const Chunk* __restrict__ chunks,
                                                  T* phi, const T* __restrict__ rhs,
                                                  const typename CoefOf<T>::type* __restrict__ wx,
                                                  const typename CoefOf<T>::type* __restrict__ wy,
                                                  const typename CoefOf<T>::type* __restrict__ wz,
                                                  const typename CoefOf<T>::type* __restrict__ invD, int colour,
                                                  const int* __restrict__ active,
                                                  const PushFace* __restrict__ push, int rev, int sp) {
  pdl_enter();
  using A = typename Arith<T>::type;
  const Chunk ch = chunks[rev ? gridDim.x - 1 - blockIdx.x : blockIdx.x];
  const DevBox B = boxes[ch.item];
  if (active && !active[B.solve]) return;
  const int t = ch.start + threadIdx.x;
  if (t >= ((B.nx + 1) >> 1) * B.ny * B.nz) return;
  int i, j, k;
  pair_decode(B, t, i, j, k);
  i += (B.lo[0] + B.lo[1] + B.lo[2] + j + k + colour) & 1;
  if (i >= B.nx) return;
  const int64_t q = elem_index(B, i, j, k);
  const int64_t sx = B.sx, sy = B.sy;
  const int64_t qs = sp ? split_pair_slot(q - (i & 1), i & ~1, colour, B.nx) : q;
  A s = ldg(rhs + ((sp & SPLIT_RHS) ? qs : q));
  s = fma((A)ldg(wx + q), (A)ld(phi + q - 1), s);
  s = fma((A)ldg(wx + q + 1), (A)ld(phi + q + 1), s);
  s = fma((A)ldg(wy + q), (A)ld(phi + q - sx), s);
  s = fma((A)ldg(wy + q + sx), (A)ld(phi + q + sx), s);
  s = fma((A)ldg(wz + q), (A)ld(phi + q - sy), s);
  s = fma((A)ldg(wz + q + sy), (A)ld(phi + q + sy), s);
  s = s * (A)ldg(invD + ((sp & SPLIT_INVD) ? qs : q));
  st(phi + q, s);
  if (push) push_ghosts(B, ch.item, boxes, push, phi, i, j, k, s);
}

// The last colour pass of a coarse level's post-smoothing fused with the piecewise-constant
// interpolation of its correction onto the finer level (Sec. "Operations between levels"):
// the thread updates the cell of its pair of the colour as k_smooth does, then adds both
// cells of the pair -- the other colour's value is final -- to their 8 children each in the
// box's one child box (child: per coarse box; the level pair is used only where every box
// has one, of exactly twice its extent), pushing the children's new values into the fine
// ghosts that copy them (fpush).  The values of the colour pass followed by k_prolong_add,
// one pass over the fine level fewer.
template <class T>
__global__ void __launch_bounds__(BLOCK)
    k_smooth_prolong(const DevBox* __restrict__ boxes, const Chunk* __restrict__ chunks, T* phi,
                     const T* __restrict__ rhs, const typename CoefOf<T>::type* __restrict__ wx,
                     const typename CoefOf<T>::type* __restrict__ wy, const typename CoefOf<T>::type* __restrict__ wz,
                     const typename CoefOf<T>::type* __restrict__ invD, int colour, const int* __restrict__ active,
                     const PushFace* __restrict__ push, int rev, T* fine, const DevBox* __restrict__ fboxes,
                     const int* __restrict__ child, const PushFace* __restrict__ fpush) {
  pdl_enter();
  using A = typename Arith<T>::type;
  const Chunk ch = chunks[rev ? gridDim.x - 1 - blockIdx.x : blockIdx.x];
  const DevBox B = boxes[ch.item];
  if (active && !active[B.solve]) return;
  const int t = ch.start + threadIdx.x;
  if (t >= ((B.nx + 1) >> 1) * B.ny * B.nz) return;
  int i0, j, k;
  pair_decode(B, t, i0, j, k);
  const int par = (B.lo[0] + B.lo[1] + B.lo[2] + i0 + j + k + colour) & 1;
  const int i = i0 + par;
  const int64_t q0 = elem_index(B, i0, j, k);
  const int64_t sx = B.sx, sy = B.sy;
  if (i < B.nx) {
    const int64_t q = q0 + par;
    A s = ldg(rhs + q);
    s = fma((A)ldg(wx + q), (A)ld(phi + q - 1), s);
    s = fma((A)ldg(wx + q + 1), (A)ld(phi + q + 1), s);
    s = fma((A)ldg(wy + q), (A)ld(phi + q - sx), s);
    s = fma((A)ldg(wy + q + sx), (A)ld(phi + q + sx), s);
    s = fma((A)ldg(wz + q), (A)ld(phi + q - sy), s);
    s = fma((A)ldg(wz + q + sy), (A)ld(phi + q + sy), s);
    s = s * (A)ldg(invD + q);
    st(phi + q, s);
    if (push) push_ghosts(B, ch.item, boxes, push, phi, i, j, k, s);
  }
  const int fb = child[ch.item];
  const DevBox F = fboxes[fb];
  for (int c = 0; c < 2 && i0 + c < B.nx; ++c) {
    const A e = ld(phi + q0 + c);  // (as stored)
    const int fi = 2 * (i0 + c);
    for (int dk = 0; dk < 2; ++dk)
      for (int dj = 0; dj < 2; ++dj) {
        const int fj = 2 * j + dj, fk = 2 * k + dk;
        const int64_t qf = elem_index(F, fi, fj, fk);
        const A v0 = (A)ld(fine + qf) + e;
        const A v1 = (A)ld(fine + qf + 1) + e;
        st(fine + qf, v0);
        st(fine + qf + 1, v1);
        if (fpush) {
          push_ghosts(F, fb, fboxes, fpush, fine, fi, fj, fk, v0);
          push_ghosts(F, fb, fboxes, fpush, fine, fi + 1, fj, fk, v1);
        }
      }
  }
}

// a value of type T's arithmetic type rounded as T stores it
__device__ __forceinline__ double as_stored(double v, const double*) { return v; }
__device__ __forceinline__ float as_stored(float v, const float*) { return v; }
__device__ __forceinline__ float as_stored(float v, const bf16*) { return __bfloat162float(__float2bfloat16_rn(v)); }

// The first (red) pass of post-smoothing fused with the interpolation of the coarse
// correction ec (piecewise constant, Sec. "Operations between levels"): a red cell reads
// each neighbour as the interpolation would have left it -- its value plus its parent's
// coarse value, rounded as stored, ghosts included (their parents are the coarse ghosts,
// which must be current) -- and is updated as k_smooth does.  The black cells are not
// written: the black pass that follows overwrites them without reading them, so the
// interpolation pass over the level goes away and the red cells get the values of the
// interpolation followed by the colour pass, bit for bit.  A black cell next to a wall does
// read its own image there, so its interpolated value goes into its wall ghosts (which no
// red cell reads); the level must push its ghosts (an exchange would copy the old value).
template <class T>
__global__ void __launch_bounds__(BLOCK)
    k_smooth_pro(const DevBox* __restrict__ boxes, const Chunk* __restrict__ chunks, T* phi, const T* __restrict__ rhs,
                 const typename CoefOf<T>::type* __restrict__ wx, const typename CoefOf<T>::type* __restrict__ wy,
                 const typename CoefOf<T>::type* __restrict__ wz, const typename CoefOf<T>::type* __restrict__ invD,
                 int colour, const int* __restrict__ active, const PushFace* __restrict__ push, int rev, int sp,
                 const T* __restrict__ ec, const DevBox* __restrict__ cboxes, const int* __restrict__ parent) {
  pdl_enter();
  using A = typename Arith<T>::type;
  const Chunk ch = chunks[rev ? gridDim.x - 1 - blockIdx.x : blockIdx.x];
  const DevBox B = boxes[ch.item];
  if (active && !active[B.solve]) return;
  const int t = ch.start + threadIdx.x;
  if (t >= ((B.nx + 1) >> 1) * B.ny * B.nz) return;
  int i0, j, k;
  pair_decode(B, t, i0, j, k);
  const int par = (B.lo[0] + B.lo[1] + B.lo[2] + i0 + j + k + colour) & 1;
  const int i = i0 + par, ib = i0 + 1 - par;  // the cell of the colour and the other one
  const DevBox P = cboxes[parent[ch.item]];
  // parent (coarse) element of the fine cell at global (a0, a1, a2); floor halving
  auto pe = [&](int a0, int a1, int a2) -> A {
    return (A)ld(ec + elem_index(P, (a0 >> 1) - P.lo[0], (a1 >> 1) - P.lo[1], (a2 >> 1) - P.lo[2]));
  };
  if (push && ib < B.nx) {
    const int64_t qb = elem_index(B, ib, j, k);
    push_walls(B, ch.item, boxes, push, phi, ib, j, k,
               as_stored((A)ld(phi + qb) + pe(B.lo[0] + ib, B.lo[1] + j, B.lo[2] + k), phi));
  }
  if (i >= B.nx) return;
  const int64_t q = elem_index(B, i, j, k);
  const int64_t sx = B.sx, sy = B.sy;
  const int64_t qs = sp ? split_pair_slot(q - (i & 1), i & ~1, colour, B.nx) : q;
  const int g0 = B.lo[0] + i, g1 = B.lo[1] + j, g2 = B.lo[2] + k;
  // the cell's own parent serves the three neighbours in its 2x2x2 block; each other one is
  // one coarse stride away (towards the side the neighbour lies on)
  const int64_t qp = elem_index(P, (g0 >> 1) - P.lo[0], (g1 >> 1) - P.lo[1], (g2 >> 1) - P.lo[2]);
  const int64_t psx = P.sx, psy = P.sy;
  const A pc = ld(ec + qp);
  const A pxm = (g0 & 1) ? pc : (A)ld(ec + qp - 1);
  const A pxp = (g0 & 1) ? (A)ld(ec + qp + 1) : pc;
  const A pym = (g1 & 1) ? pc : (A)ld(ec + qp - psx);
  const A pyp = (g1 & 1) ? (A)ld(ec + qp + psx) : pc;
  const A pzm = (g2 & 1) ? pc : (A)ld(ec + qp - psy);
  const A pzp = (g2 & 1) ? (A)ld(ec + qp + psy) : pc;
  const A vxm = as_stored((A)ld(phi + q - 1) + pxm, phi);
  const A vxp = as_stored((A)ld(phi + q + 1) + pxp, phi);
  const A vym = as_stored((A)ld(phi + q - sx) + pym, phi);
  const A vyp = as_stored((A)ld(phi + q + sx) + pyp, phi);
  const A vzm = as_stored((A)ld(phi + q - sy) + pzm, phi);
  const A vzp = as_stored((A)ld(phi + q + sy) + pzp, phi);
  A s = ldg(rhs + ((sp & SPLIT_RHS) ? qs : q));
  s = fma((A)ldg(wx + q), vxm, s);
  s = fma((A)ldg(wx + q + 1), vxp, s);
  s = fma((A)ldg(wy + q), vym, s);
  s = fma((A)ldg(wy + q + sx), vyp, s);
  s = fma((A)ldg(wz + q), vzm, s);
  s = fma((A)ldg(wz + q + sy), vzp, s);
  s = s * (A)ldg(invD + ((sp & SPLIT_INVD) ? qs : q));
  st(phi + q, s);
  if (push) push_ghosts(B, ch.item, boxes, push, phi, i, j, k, s);
}

// The last colour pass of a V-cycle's post-smoothing on the finest level fused with the
// solution update: the thread updates the cell of the colour as k_smooth does (storing e),
// then adds both cells' corrections of its pair to phi -- the other cell's e is final
// (the other colour went before) -- and pushes phi's new values into the ghosts that copy
// them (push_phi non-null).  The same values as the colour pass followed by
// k_add_correction (each correction added as stored), one pass fewer over phi and e.
template <class T>
__global__ void __launch_bounds__(BLOCK, SmoothMinB<T>::value)
    k_smooth_update(const DevBox* __restrict__ boxes, const Chunk* __restrict__ chunks, T* e, const T* __restrict__ rhs,
                    const typename CoefOf<T>::type* __restrict__ wx, const typename CoefOf<T>::type* __restrict__ wy,
                    const typename CoefOf<T>::type* __restrict__ wz, const typename CoefOf<T>::type* __restrict__ invD,
                    int colour, const int* __restrict__ active, double* phi, const PushFace* __restrict__ push_phi, int rev,
                    int sp) {
  pdl_enter();
  using A = typename Arith<T>::type;
  const Chunk ch = chunks[rev ? gridDim.x - 1 - blockIdx.x : blockIdx.x];
  const DevBox B = boxes[ch.item];
  if (active && !active[B.solve]) return;
  const int t = ch.start + threadIdx.x;
  if (t >= ((B.nx + 1) >> 1) * B.ny * B.nz) return;
  int i0, j, k;
  pair_decode(B, t, i0, j, k);
  const int par = (B.lo[0] + B.lo[1] + B.lo[2] + i0 + j + k + colour) & 1;
  const int i = i0 + par;
  const int64_t q0 = elem_index(B, i0, j, k);
  const int64_t sx = B.sx, sy = B.sy;
  if (i < B.nx) {
    const int64_t q = q0 + par;
    const int64_t qs = sp ? split_pair_slot(q0, i0, colour, B.nx) : q;
    A s = ldg(rhs + ((sp & SPLIT_RHS) ? qs : q));
    s = fma((A)ldg(wx + q), (A)ld(e + q - 1), s);
    s = fma((A)ldg(wx + q + 1), (A)ld(e + q + 1), s);
    s = fma((A)ldg(wy + q), (A)ld(e + q - sx), s);
    s = fma((A)ldg(wy + q + sx), (A)ld(e + q + sx), s);
    s = fma((A)ldg(wz + q), (A)ld(e + q - sy), s);
    s = fma((A)ldg(wz + q + sy), (A)ld(e + q + sy), s);
    s = s * (A)ldg(invD + ((sp & SPLIT_INVD) ? qs : q));
    st(e + q, s);
  }
  if (i0 + 1 < B.nx) {
    double2 p = *reinterpret_cast<const double2*>(phi + q0);
    p.x += (double)ld(e + q0);
    p.y += (double)ld(e + q0 + 1);
    *reinterpret_cast<double2*>(phi + q0) = p;
    if (push_phi) {
      push_ghosts(B, ch.item, boxes, push_phi, phi, i0, j, k, p.x);
      push_ghosts(B, ch.item, boxes, push_phi, phi, i0 + 1, j, k, p.y);
    }
  } else {
    const double v = phi[q0] + (double)ld(e + q0);
    phi[q0] = v;
    if (push_phi) push_ghosts(B, ch.item, boxes, push_phi, phi, i0, j, k, v);
  }
}

// Four consecutive cells (x), 16-byte aligned: 128-bit loads for float, 64-bit for bfloat16.
__device__ __forceinline__ void ld4(const float* p, float v[4]) {
  const float4 a = *reinterpret_cast<const float4*>(p);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void ldg4(const float* p, float v[4]) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
}
__device__ __forceinline__ void ld4(const bf16* p, float v[4]) {
  const uint2 u = *reinterpret_cast<const uint2*>(p);
  const float2 a = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.x));
  const float2 b = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(&u.y));
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void ldg4(const bf16* p, float v[4]) { ld4(p, v); }
// two consecutive elements from an even element (a 64-bit load for float, 32-bit for bfloat16)
__device__ __forceinline__ void ld2e(const float* p, float& a, float& b) {
  const float2 v = __ldg(reinterpret_cast<const float2*>(p));
  a = v.x;
  b = v.y;
}
__device__ __forceinline__ void ld2e(const bf16* p, float& a, float& b) {
  const float2 v = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
  a = v.x;
  b = v.y;
}

// One red-black colour with one thread per 4 consecutive cells of a row (boxes whose width
// is a multiple of 4; float and bfloat16 fields): the thread reads the 4-cell segments of
// phi (with its four neighbour segments), rhs and the coefficients with vector loads and
// updates the two cells of the colour -- the arithmetic and order of k_smooth, so the
// results are bitwise the same.
template <class T>
__global__ void __launch_bounds__(BLOCK, 4) k_smooth4(const DevBox* __restrict__ boxes, const Chunk* __restrict__ chunks,
                                                   T* phi, const T* __restrict__ rhs, const float* __restrict__ wx,
                                                   const float* __restrict__ wy, const float* __restrict__ wz,
                                                   const float* __restrict__ invD, int colour,
                                                   const int* __restrict__ active, const PushFace* __restrict__ push, int rev,
                                                   int sp) {
  pdl_enter();
  const Chunk ch = chunks[rev ? gridDim.x - 1 - blockIdx.x : blockIdx.x];
  const DevBox B = boxes[ch.item];
  if (active && !active[B.solve]) return;
  const int nq = B.nx >> 2;
  const int t = ch.start + threadIdx.x;
  if (t >= nq * B.ny * B.nz) return;
  const int g = t % nq, r = t / nq;
  const int j = r % B.ny, k = r / B.ny, i0 = 4 * g;
  const int64_t q0 = elem_index(B, i0, j, k);
  const int64_t sx = B.sx, sy = B.sy;
  float p[4], pym[4], pyp[4], pzm[4], pzp[4], wxl[4], wyl[4], wyh[4], wzl[4], wzh[4];
  ld4(phi + q0, p);
  ld4(phi + q0 - sx, pym);
  ld4(phi + q0 + sx, pyp);
  ld4(phi + q0 - sy, pzm);
  ld4(phi + q0 + sy, pzp);
  const float pl = ld(phi + q0 - 1), pr = ld(phi + q0 + 4);
  const int c0 = (B.lo[0] + B.lo[1] + B.lo[2] + i0 + j + k + colour) & 1;
  // rhs and 1/D of the segment's two cells of the colour (c0 and c0 + 2); colour-split: two
  // consecutive slots of the colour's half, the first at an even element (widths are
  // multiples of 4 here)
  float ra, rb, da, db;
  if (sp & SPLIT_RHS) {
    ld2e(rhs + split_pair_slot(q0, i0, colour, B.nx), ra, rb);
  } else {
    float rh[4];
    ldg4(rhs + q0, rh);
    ra = c0 ? rh[1] : rh[0];
    rb = c0 ? rh[3] : rh[2];
  }
  ldg4(wx + q0, wxl);
  const float wx4 = __ldg(wx + q0 + 4);
  ldg4(wy + q0, wyl);
  ldg4(wy + q0 + sx, wyh);
  ldg4(wz + q0, wzl);
  ldg4(wz + q0 + sy, wzh);
  if (sp & SPLIT_INVD) {
    ld2e(invD + split_pair_slot(q0, i0, colour, B.nx), da, db);
  } else {
    float id[4];
    ldg4(invD + q0, id);
    da = c0 ? id[1] : id[0];
    db = c0 ? id[3] : id[2];
  }
  // cells m and m + 2 of the segment, m = c0 (constant indices keep the arrays in registers)
  auto update = [&](auto mc, float rv, float dv) {
    constexpr int m = decltype(mc)::value;
    float s = rv;
    s = fmaf(wxl[m], m == 0 ? pl : p[m == 0 ? 0 : m - 1], s);
    s = fmaf(m == 3 ? wx4 : wxl[m == 3 ? 3 : m + 1], m == 3 ? pr : p[m == 3 ? 3 : m + 1], s);
    s = fmaf(wyl[m], pym[m], s);
    s = fmaf(wyh[m], pyp[m], s);
    s = fmaf(wzl[m], pzm[m], s);
    s = fmaf(wzh[m], pzp[m], s);
    s = s * dv;
    st(phi + q0 + m, s);
    if (push) push_ghosts(B, ch.item, boxes, push, phi, i0 + m, j, k, s);
  };
  if (c0 == 0) {
    update(std::integral_constant<int, 0>(), ra, da);
    update(std::integral_constant<int, 2>(), rb, db);
  } else {
    update(std::integral_constant<int, 1>(), ra, da);
    update(std::integral_constant<int, 3>(), rb, db);
  }
}

// One colour of Gauss-Seidel on double fields with 128-bit loads: each thread reads the
// aligned cell pair (i0, i0 + 1) of phi in its own row and in the rows and planes around it,
// and the pair's rhs, 1/D and face weights, as double2 loads, and updates the pair's cell of
// the colour with k_smooth's operands in k_smooth's order (bitwise the same values).
__global__ void __launch_bounds__(BLOCK)
    k_smooth_d2(const DevBox* __restrict__ boxes, const Chunk* __restrict__ chunks, double* phi,
                const double* __restrict__ rhs, const double* __restrict__ wx, const double* __restrict__ wy,
                const double* __restrict__ wz, const double* __restrict__ invD, int colour,
                const int* __restrict__ active, const PushFace* __restrict__ push, int rev, int sp) {
  pdl_enter();
  const Chunk ch = chunks[rev ? gridDim.x - 1 - blockIdx.x : blockIdx.x];
  const DevBox B = boxes[ch.item];
  if (active && !active[B.solve]) return;
  const int t = ch.start + threadIdx.x;
  if (t >= ((B.nx + 1) >> 1) * B.ny * B.nz) return;
  int i0, j, k;
  pair_decode(B, t, i0, j, k);
  const int off = (B.lo[0] + B.lo[1] + B.lo[2] + i0 + j + k + colour) & 1;
  if (i0 + 1 >= B.nx) {  // (a last single cell of an odd row: the scalar kernel's path)
    if (off) return;
  }
  const int64_t q0 = elem_index(B, i0, j, k);  // even: 16-byte aligned
  const int64_t q = q0 + off;
  const int64_t sx = B.sx, sy = B.sy;
  auto ld2 = [](const double* p) { return *reinterpret_cast<const double2*>(p); };
  auto ldg2 = [](const double* p) { return __ldg(reinterpret_cast<const double2*>(p)); };
  auto pick = [off](double2 v) { return off ? v.y : v.x; };
  const double2 own = ld2(phi + q0);
  const double outer = off ? phi[q0 + 2] : phi[q0 - 1];
  const double2 ym = ld2(phi + q0 - sx), yp = ld2(phi + q0 + sx);
  const double2 zm = ld2(phi + q0 - sy), zp = ld2(phi + q0 + sy);
  const double2 z2 = make_double2(0.0, 0.0);
  const double2 r2 = (sp & SPLIT_RHS) ? z2 : ldg2(rhs + q0), d2 = (sp & SPLIT_INVD) ? z2 : ldg2(invD + q0);
  const double2 wx2 = ldg2(wx + q0);
  const double2 wyl = ldg2(wy + q0), wyh = ldg2(wy + q0 + sx), wzl = ldg2(wz + q0), wzh = ldg2(wz + q0 + sy);
  const double wxr = off ? __ldg(wx + q0 + 2) : wx2.y;
  const int64_t qs = sp ? split_pair_slot(q0, i0, colour, B.nx) : q;
  double s = (sp & SPLIT_RHS) ? __ldg(rhs + qs) : pick(r2);
  s = fma(off ? wx2.y : wx2.x, off ? own.x : outer, s);
  s = fma(wxr, off ? outer : own.y, s);
  s = fma(pick(wyl), pick(ym), s);
  s = fma(pick(wyh), pick(yp), s);
  s = fma(pick(wzl), pick(zm), s);
  s = fma(pick(wzh), pick(zp), s);
  s = s * ((sp & SPLIT_INVD) ? __ldg(invD + qs) : pick(d2));
  phi[q] = s;
  if (push) push_ghosts(B, ch.item, boxes, push, phi, i0 + off, j, k, s);
}

// ------------------------------------------------------------------- residual

// whether global cell g of a level lies next to one of its problem's walls
__device__ __forceinline__ bool next_to_wall(const DevGeom& G, int g0, int g1, int g2) {
  return (G.wall_lo[0] && g0 == G.dlo[0]) || (G.wall_hi[0] && g0 == G.dhi[0]) || (G.wall_lo[1] && g1 == G.dlo[1]) ||
         (G.wall_hi[1] && g1 == G.dhi[1]) || (G.wall_lo[2] && g2 == G.dlo[2]) || (G.wall_hi[2] && g2 == G.dhi[2]);
}


template <class T, class C>
__device__ __forceinline__ typename Arith<T>::type resid_at(const T* phi, const T* rhs, const C* wx, const C* wy,
                                                           const C* wz, const C* D, int64_t q, int64_t sx, int64_t sy,
                                                           typename Arith<T>::type shift, int64_t rq) {
  using A = typename Arith<T>::type;
  A v = (A)ldg(rhs + rq) - shift;
  v = fma(-(A)ldg(D + q), (A)ld(phi + q), v);
  v = fma((A)ldg(wx + q), (A)ld(phi + q - 1), v);
  v = fma((A)ldg(wx + q + 1), (A)ld(phi + q + 1), v);
  v = fma((A)ldg(wy + q), (A)ld(phi + q - sx), v);
  v = fma((A)ldg(wy + q + sx), (A)ld(phi + q + sx), v);
  v = fma((A)ldg(wz + q), (A)ld(phi + q - sy), v);
  v = fma((A)ldg(wz + q + sy), (A)ld(phi + q + sy), v);
  return v;
}

// (MINB: resident blocks per SM the register count must allow; 6 for the FP64 residual,
// whose loads then have more warps to overlap them; 0, no bound, elsewhere)
template <class T, class R, int MINB, bool RS>
__global__ void __launch_bounds__(BLOCK, MINB) k_residual(const DevBox* __restrict__ boxes,
                                                          const DevGeom* __restrict__ geoms,
                                                    const Chunk* __restrict__ chunks,
                                                    const T* __restrict__ phi, const T* __restrict__ rhs,
                                                    const typename CoefOf<T>::type* __restrict__ wx,
                                                    const typename CoefOf<T>::type* __restrict__ wy,
                                                    const typename CoefOf<T>::type* __restrict__ wz,
                                                    const typename CoefOf<T>::type* __restrict__ D, R* r,
                                                    unsigned long long* maxbits, const double* shift_p, R* e,
                                                    const typename CoefOf<R>::type* __restrict__ invDe,
                                                    const PushFace* __restrict__ push, int settled, int rev) {
  constexpr bool rsplit = RS;  // r (and invDe) colour-split
  pdl_enter();
  using A = typename Arith<T>::type;
  using AR = typename Arith<R>::type;
  const Chunk ch = chunks[rev ? gridDim.x - 1 - blockIdx.x : blockIdx.x];
  const DevBox B = boxes[ch.item];
  const int t = ch.start + threadIdx.x;
  const A shift = shift_p ? (A)shift_p[B.solve] : (A)0;
  unsigned long long mx = 0;
  if (settled >= 0 && t < ((B.nx + 1) >> 1) * B.ny * B.nz) {
    // the cell of the pair not of the settled colour is computed; the settled one's r is 0
    // unless it lies next to a wall.  e: r / D on red, 0 on black.
    int i0, j, k;
    pair_decode(B, t, i0, j, k);
    const int64_t q0 = elem_index(B, i0, j, k);
    const int c0 = (B.lo[0] + B.lo[1] + B.lo[2] + i0 + j + k) & 1;  // colour of the pair's first cell
    const int cc = c0 == settled ? 1 : 0;                          // offset of the computed cell
    const int cs = 1 - cc;                                          // offset of the settled cell
    if (i0 + cc < B.nx) {
      const A v = shift_p ? resid_at(phi, rhs, wx, wy, wz, D, q0 + cc, B.sx, B.sy, shift, q0 + cc)
                          : resid_at(phi, rhs, wx, wy, wz, D, q0 + cc, B.sx, B.sy, (A)0, q0 + cc);
      st(r + (rsplit ? split_pair_slot(q0, i0, (c0 + cc) & 1, B.nx) : q0 + cc), v);
      mx = abs_bits((double)v);
    }
    if (i0 + cs < B.nx) {
      A v = 0;
      if (next_to_wall(geoms[B.solve], B.lo[0] + i0 + cs, B.lo[1] + j, B.lo[2] + k)) {
        v = shift_p ? resid_at(phi, rhs, wx, wy, wz, D, q0 + cs, B.sx, B.sy, shift, q0 + cs)
                    : resid_at(phi, rhs, wx, wy, wz, D, q0 + cs, B.sx, B.sy, (A)0, q0 + cs);
        const unsigned long long bb = abs_bits((double)v);
        mx = bb > mx ? bb : mx;
      }
      st(r + (rsplit ? split_pair_slot(q0, i0, (c0 + cs) & 1, B.nx) : q0 + cs), v);
    }
    if (e) {
      for (int c = 0; c < 2; ++c) {
        if (i0 + c >= B.nx) break;
        const bool red = ((c0 + c) & 1) == 0;
        const int64_t rs = rsplit ? split_pair_slot(q0, i0, (c0 + c) & 1, B.nx) : q0 + c;
        const AR ev = red ? (AR)ld(r + rs) * (AR)ldg(invDe + rs) : (AR)0;
        st(e + q0 + c, ev);
        if (push) push_ghosts(B, ch.item, boxes, push, e, i0 + c, j, k, ev);
      }
    }
  } else if (t < ((B.nx + 1) >> 1) * B.ny * B.nz) {
    int i0, j, k;
    pair_decode(B, t, i0, j, k);
    const int64_t q0 = elem_index(B, i0, j, k);
    for (int c = 0; c < 2; ++c) {
      if (i0 + c >= B.nx) break;
      // (no shift: one FP64 operation per cell less, the kernel being bound by the FP64 pipe)
      const A v = shift_p ? resid_at(phi, rhs, wx, wy, wz, D, q0 + c, B.sx, B.sy, shift, q0 + c)
                          : resid_at(phi, rhs, wx, wy, wz, D, q0 + c, B.sx, B.sy, (A)0, q0 + c);
      const int64_t rs = rsplit ? split_pair_slot(q0, i0, (B.lo[0] + B.lo[1] + B.lo[2] + i0 + c + j + k) & 1, B.nx) : q0 + c;
      if (r) st(r + rs, v);
      const unsigned long long bb = abs_bits((double)v);
      mx = bb > mx ? bb : mx;
      if (e) {
        // the first red half-sweep of the next V-cycle on e = 0: every neighbour term is
        // zero, so a red cell becomes r / D (r as stored), a black cell stays 0
        const bool red = ((B.lo[0] + B.lo[1] + B.lo[2] + i0 + c + j + k) & 1) == 0;
        const AR ev = red ? (AR)ld(r + rs) * (AR)ldg(invDe + rs) : (AR)0;
        st(e + q0 + c, ev);
        if (push) push_ghosts(B, ch.item, boxes, push, e, i0 + c, j, k, ev);
      }
    }
  }
  if (maxbits) block_max_atomic(mx, maxbits + B.solve);
}

// the restriction of the residual of the 8 children of coarse cell (ci, cj, ck) of fine box F
template <class T>
__device__ __forceinline__ typename Arith<T>::type resid_sum8(const DevBox& F, const T* phi, const T* rhs,
                                                              const typename CoefOf<T>::type* wx,
                                                              const typename CoefOf<T>::type* wy,
                                                              const typename CoefOf<T>::type* wz,
                                                              const typename CoefOf<T>::type* D, int ci, int cj,
                                                              int ck, bool split) {
  using A = typename Arith<T>::type;
  A s = 0;
  for (int dk = 0; dk < 2; ++dk)
    for (int dj = 0; dj < 2; ++dj) {
      const int i = 2 * ci, j = 2 * cj + dj, k = 2 * ck + dk;
      const int64_t q = elem_index(F, i, j, k);
      s += resid_at(phi, rhs, wx, wy, wz, D, q, F.sx, F.sy, (A)0, cell_slot(split, F, i, j, k, q));
      s += resid_at(phi, rhs, wx, wy, wz, D, q + 1, F.sx, F.sy, (A)0, cell_slot(split, F, i + 1, j, k, q + 1));
    }
  return s;
}

// residual of the 8 children of one coarse cell, averaged into the coarse level
template <class T, class R>
__global__ void __launch_bounds__(BLOCK, 5)
    k_resid_restrict(const DevBox* __restrict__ fboxes, const DevGeom* __restrict__ fgeoms,
                     const DevBox* __restrict__ cboxes,
                     const int* __restrict__ parent, const Chunk* __restrict__ chunks, const T* __restrict__ phi,
                     const T* __restrict__ rhs, const typename CoefOf<T>::type* __restrict__ wx,
                     const typename CoefOf<T>::type* __restrict__ wy, const typename CoefOf<T>::type* __restrict__ wz,
                     const typename CoefOf<T>::type* __restrict__ D, R* rc, const int* __restrict__ active,
                     int settled_black, int rev, int split, R* ec, const typename CoefOf<R>::type* __restrict__ invDc,
                     const PushFace* __restrict__ cpush) {
  pdl_enter();
  using A = typename Arith<T>::type;
  const Chunk ch = chunks[rev ? gridDim.x - 1 - blockIdx.x : blockIdx.x];
  const DevBox F = fboxes[ch.item];
  if (active && !active[F.solve]) return;
  const DevBox P = cboxes[parent[ch.item]];
  const int ncx = F.nx >> 1, ncy = F.ny >> 1, ncz = F.nz >> 1;
  const int t = ch.start + threadIdx.x;
  if (t >= ncx * ncy * ncz) return;
  const int ci = t % ncx, cj = (t / ncx) % ncy, ck = t / (ncx * ncy);
  A s = 0;
  if (settled_black) {
    // the 4 red children; the black ones count 0 (see launch_resid_restrict) unless the
    // coarse cell's children touch a wall
    const int par = (F.lo[0] + F.lo[1] + F.lo[2]) & 1;  // colour of the box's first cell
    for (int dk = 0; dk < 2; ++dk)
      for (int dj = 0; dj < 2; ++dj) {
        const int dx = (par + dj + dk) & 1;  // the red child of the row pair
        const int i = 2 * ci + dx, j = 2 * cj + dj, k = 2 * ck + dk;
        const int64_t q = elem_index(F, i, j, k);
        s += resid_at(phi, rhs, wx, wy, wz, D, q, F.sx, F.sy, (A)0, cell_slot(split, F, i, j, k, q));
      }
    const DevGeom G = fgeoms[F.solve];
    const int g0 = F.lo[0] + 2 * ci, g1 = F.lo[1] + 2 * cj, g2 = F.lo[2] + 2 * ck;
    if (next_to_wall(G, g0, g1, g2) || next_to_wall(G, g0 + 1, g1 + 1, g2 + 1)) {
      for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj) {
          const int dx = 1 - ((par + dj + dk) & 1);  // the black child of the row pair
          if (!next_to_wall(G, g0 + dx, g1 + dj, g2 + dk)) continue;  // (its residual is 0)
          const int i = 2 * ci + dx, j = 2 * cj + dj, k = 2 * ck + dk;
          const int64_t q = elem_index(F, i, j, k);
          s += resid_at(phi, rhs, wx, wy, wz, D, q, F.sx, F.sy, (A)0, cell_slot(split, F, i, j, k, q));
        }
    }
  } else {
    s = resid_sum8(F, phi, rhs, wx, wy, wz, D, ci, cj, ck, split != 0);
  }
  const int I = (F.lo[0] >> 1) + ci - P.lo[0];
  const int J = (F.lo[1] >> 1) + cj - P.lo[1];
  const int K = (F.lo[2] >> 1) + ck - P.lo[2];
  const int64_t qc = elem_index(P, I, J, K);
  st(rc + qc, s * (A)0.125);
  if (ec) {
    // the coarse level's first red half-sweep on e = 0: every neighbour term is zero, so a
    // red cell becomes r / D (r as stored), a black cell stays 0
    using AR = typename Arith<R>::type;
    const bool red = ((P.lo[0] + P.lo[1] + P.lo[2] + I + J + K) & 1) == 0;
    const AR ev = red ? (AR)ld(rc + qc) * (AR)ldg(invDc + qc) : (AR)0;
    st(ec + qc, ev);
    if (cpush) push_ghosts(P, parent[ch.item], cboxes, cpush, ec, I, J, K, ev);
  }
}

template <class T>
__global__ void __launch_bounds__(BLOCK)
    k_restrict(const DevBox* __restrict__ fboxes, const DevBox* __restrict__ cboxes, const int* __restrict__ parent,
               const Chunk* __restrict__ chunks, const T* __restrict__ fine, T* coarse) {
  using A = typename Arith<T>::type;
  const Chunk ch = chunks[blockIdx.x];
  const DevBox F = fboxes[ch.item];
  const DevBox P = cboxes[parent[ch.item]];
  const int ncx = F.nx >> 1, ncy = F.ny >> 1, ncz = F.nz >> 1;
  const int t = ch.start + threadIdx.x;
  if (t >= ncx * ncy * ncz) return;
  const int ci = t % ncx, cj = (t / ncx) % ncy, ck = t / (ncx * ncy);
  A s = 0;
  for (int dk = 0; dk < 2; ++dk)
    for (int dj = 0; dj < 2; ++dj) {
      const int64_t q = elem_index(F, 2 * ci, 2 * cj + dj, 2 * ck + dk);
      s += (A)ld(fine + q);
      s += (A)ld(fine + q + 1);
    }
  const int I = (F.lo[0] >> 1) + ci - P.lo[0];
  const int J = (F.lo[1] >> 1) + cj - P.lo[1];
  const int K = (F.lo[2] >> 1) + ck - P.lo[2];
  st(coarse + elem_index(P, I, J, K), s * (A)0.125);
}

// (MINB as for k_residual: 8 for FP64, no bound otherwise)
template <class T, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB)
    k_prolong_add(const DevBox* __restrict__ fboxes, const DevBox* __restrict__ cboxes, const int* __restrict__ parent,
                  const Chunk* __restrict__ chunks, const T* __restrict__ coarse, T* fine,
                  const int* __restrict__ active, const PushFace* __restrict__ push, int rev) {
  pdl_enter();
  using A = typename Arith<T>::type;
  const Chunk ch = chunks[rev ? gridDim.x - 1 - blockIdx.x : blockIdx.x];
  const DevBox F = fboxes[ch.item];
  if (active && !active[F.solve]) return;
  const DevBox P = cboxes[parent[ch.item]];
  const int ncx = F.nx >> 1, ncy = F.ny >> 1, ncz = F.nz >> 1;
  const int t = ch.start + threadIdx.x;
  if (t >= ncx * ncy * ncz) return;
  const int ci = t % ncx, cj = (t / ncx) % ncy, ck = t / (ncx * ncy);
  const int I = (F.lo[0] >> 1) + ci - P.lo[0];
  const int J = (F.lo[1] >> 1) + cj - P.lo[1];
  const int K = (F.lo[2] >> 1) + ck - P.lo[2];
  const A e = ld(coarse + elem_index(P, I, J, K));
  for (int dk = 0; dk < 2; ++dk)
    for (int dj = 0; dj < 2; ++dj) {
      const int64_t q = elem_index(F, 2 * ci, 2 * cj + dj, 2 * ck + dk);
      A v0, v1;
      if constexpr (std::is_same<T, double>::value) {  // the pair (even element) as one 16-byte access
        double2 f = *reinterpret_cast<const double2*>(fine + q);
        v0 = f.x + e;
        v1 = f.y + e;
        *reinterpret_cast<double2*>(fine + q) = make_double2(v0, v1);
      } else {
        v0 = (A)ld(fine + q) + e;
        v1 = (A)ld(fine + q + 1) + e;
        st(fine + q, v0);
        st(fine + q + 1, v1);
      }
      if (push) {
        push_ghosts(F, ch.item, fboxes, push, fine, 2 * ci, 2 * cj + dj, 2 * ck + dk, v0);
        push_ghosts(F, ch.item, fboxes, push, fine, 2 * ci + 1, 2 * cj + dj, 2 * ck + dk, v1);
      }
    }
}

__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }

// Trilinear interpolation of the coarse correction, added to the fine one: one thread per
// coarse cell reads its 3x3x3 neighbourhood (ghosts included) and writes its 8 children.  A
// child's centre lies a quarter of a coarse cell from the parent's centre towards side
// s_d = +1 (odd local index) or -1 per axis; weights 3/4 on the parent's coordinate and 1/4 on
// the neighbour's, the eight terms summed z outermost, then y, then x, with unfused
// products (the oracle's arithmetic, so FP64 results are bitwise the oracle's).
template <class T, int MINB>
__global__ void __launch_bounds__(BLOCK, MINB)
    k_prolong_tri(const DevBox* __restrict__ fboxes, const DevBox* __restrict__ cboxes, const int* __restrict__ parent,
                  const Chunk* __restrict__ chunks, const T* __restrict__ coarse, T* fine,
                  const int* __restrict__ active, const PushFace* __restrict__ push, int rev) {
  pdl_enter();
  using A = typename Arith<T>::type;
  const Chunk ch = chunks[rev ? gridDim.x - 1 - blockIdx.x : blockIdx.x];
  const DevBox F = fboxes[ch.item];
  if (active && !active[F.solve]) return;
  const DevBox P = cboxes[parent[ch.item]];
  const int ncx = F.nx >> 1, ncy = F.ny >> 1, ncz = F.nz >> 1;
  const int t = ch.start + threadIdx.x;
  if (t >= ncx * ncy * ncz) return;
  const int ci = t % ncx, cj = (t / ncx) % ncy, ck = t / (ncx * ncy);
  const int I = (F.lo[0] >> 1) + ci - P.lo[0];
  const int J = (F.lo[1] >> 1) + cj - P.lo[1];
  const int K = (F.lo[2] >> 1) + ck - P.lo[2];
  A E[3][3][3];
#pragma unroll
  for (int dz = 0; dz < 3; ++dz)
#pragma unroll
    for (int dy = 0; dy < 3; ++dy)
#pragma unroll
      for (int dx = 0; dx < 3; ++dx) E[dz][dy][dx] = ld(coarse + elem_index(P, I + dx - 1, J + dy - 1, K + dz - 1));
  const A w[2] = {(A)0.75, (A)0.25};
#pragma unroll
  for (int oz = 0; oz < 2; ++oz)
#pragma unroll
    for (int oy = 0; oy < 2; ++oy) {
      A v[2];
#pragma unroll
      for (int ox = 0; ox < 2; ++ox) {
        const int sx = ox ? 1 : -1, sy = oy ? 1 : -1, sz = oz ? 1 : -1;
        A acc = 0;
#pragma unroll
        for (int cz = 0; cz < 2; ++cz)
#pragma unroll
          for (int cy = 0; cy < 2; ++cy)
#pragma unroll
            for (int cx = 0; cx < 2; ++cx)
              acc = add_rn(acc, mul_rn(w[cx] * w[cy] * w[cz], E[1 + cz * sz][1 + cy * sy][1 + cx * sx]));
        v[ox] = acc;
      }
      const int64_t q = elem_index(F, 2 * ci, 2 * cj + oy, 2 * ck + oz);
      const A v0 = add_rn((A)ld(fine + q), v[0]), v1 = add_rn((A)ld(fine + q + 1), v[1]);
      st(fine + q, v0);
      st(fine + q + 1, v1);
      if (push) {
        push_ghosts(F, ch.item, fboxes, push, fine, 2 * ci, 2 * cj + oy, 2 * ck + oz, v0);
        push_ghosts(F, ch.item, fboxes, push, fine, 2 * ci + 1, 2 * cj + oy, 2 * ck + oz, v1);
      }
    }
}

// f[dst] = sign * f[src] over a flat list (edge and corner ghosts)
template <class T>
__global__ void __launch_bounds__(BLOCK) k_fill_list(const BotGhost* __restrict__ g, int n, T* f) {
  pdl_enter();
  const int t = blockIdx.x * BLOCK + threadIdx.x;
  if (t >= n) return;
  const BotGhost e = g[t];
  const auto v = ld(f + e.src);
  st(f + e.dst, e.sign < 0 ? -v : v);
}

// ----------------------------------------------------------- cell-wise helpers

template <class T>
__global__ void __launch_bounds__(BLOCK) k_add_correction(const DevBox* __restrict__ boxes,
                                                          const Chunk* __restrict__ chunks, double* phi,
                                                          const T* __restrict__ e, const int* __restrict__ active,
                                                          const PushFace* __restrict__ push) {
  pdl_enter();
  // one thread per x-adjacent cell pair (chunks of pair items): the pair of phi is one
  // 16-byte access (the first cell of a pair sits at an even element)
  const Chunk ch = chunks[blockIdx.x];
  const DevBox B = boxes[ch.item];
  if (active && !active[B.solve]) return;
  const int t = ch.start + threadIdx.x;
  if (t >= ((B.nx + 1) >> 1) * B.ny * B.nz) return;
  int i0, j, k;
  pair_decode(B, t, i0, j, k);
  const int64_t q = elem_index(B, i0, j, k);
  if (i0 + 1 < B.nx) {
    double2 p = *reinterpret_cast<const double2*>(phi + q);
    p.x += (double)ld(e + q);
    p.y += (double)ld(e + q + 1);
    *reinterpret_cast<double2*>(phi + q) = p;
    if (push) {
      push_ghosts(B, ch.item, boxes, push, phi, i0, j, k, p.x);
      push_ghosts(B, ch.item, boxes, push, phi, i0 + 1, j, k, p.y);
    }
  } else {
    const double v = phi[q] + (double)ld(e + q);
    phi[q] = v;
    if (push) push_ghosts(B, ch.item, boxes, push, phi, i0, j, k, v);
  }
}

template <class T>
__global__ void __launch_bounds__(BLOCK) k_pack(const DevBox* __restrict__ boxes, const Chunk* __restrict__ chunks,
                                                int3 dlo, int3 dn, const double* __restrict__ dense, T* boxed) {
  const Chunk ch = chunks[blockIdx.x];
  const DevBox B = boxes[ch.item];
  const int t = ch.start + threadIdx.x;
  if (t >= B.nx * B.ny * B.nz) return;
  const int i = t % B.nx, j = (t / B.nx) % B.ny, k = t / (B.nx * B.ny);
  const int64_t g = (int64_t)(B.lo[0] + i - dlo.x) + (int64_t)dn.x * ((B.lo[1] + j - dlo.y) + (int64_t)dn.y * (B.lo[2] + k - dlo.z));
  st(boxed + elem_index(B, i, j, k), dense[g]);
}

template <class T>
__global__ void __launch_bounds__(BLOCK) k_unpack(const DevBox* __restrict__ boxes, const Chunk* __restrict__ chunks,
                                                  int3 dlo, int3 dn, const T* __restrict__ boxed, double* dense) {
  const Chunk ch = chunks[blockIdx.x];
  const DevBox B = boxes[ch.item];
  const int t = ch.start + threadIdx.x;
  if (t >= B.nx * B.ny * B.nz) return;
  const int i = t % B.nx, j = (t / B.nx) % B.ny, k = t / (B.nx * B.ny);
  const int64_t g = (int64_t)(B.lo[0] + i - dlo.x) + (int64_t)dn.x * ((B.lo[1] + j - dlo.y) + (int64_t)dn.y * (B.lo[2] + k - dlo.z));
  dense[g] = (double)ld(boxed + elem_index(B, i, j, k));
}

__global__ void __launch_bounds__(BLOCK) k_norm_max(const DevBox* __restrict__ boxes, const Chunk* __restrict__ chunks,
                                                    const double* __restrict__ x, unsigned long long* maxbits) {
  const Chunk ch = chunks[blockIdx.x];
  const DevBox B = boxes[ch.item];
  const int t = ch.start + threadIdx.x;
  unsigned long long mx = 0;
  if (t < B.nx * B.ny * B.nz) {
    const int i = t % B.nx, j = (t / B.nx) % B.ny, k = t / (B.nx * B.ny);
    mx = abs_bits(x[elem_index(B, i, j, k)]);
  }
  block_max_atomic(mx, maxbits + B.solve);
}

__global__ void __launch_bounds__(BLOCK) k_sum_partial(const DevBox* __restrict__ boxes, const Chunk* __restrict__ chunks,
                                                       const double* __restrict__ x, double* partials) {
  const Chunk ch = chunks[blockIdx.x];
  const DevBox B = boxes[ch.item];
  const int t = ch.start + threadIdx.x;
  double v = 0.0;
  if (t < B.nx * B.ny * B.nz) {
    const int i = t % B.nx, j = (t / B.nx) % B.ny, k = t / (B.nx * B.ny);
    v = x[elem_index(B, i, j, k)];
  }
  const double s = block_sum(v);
  if (threadIdx.x == 0) partials[blockIdx.x] = s;
}

// block s reduces the partial sums of solve s's chunk range [range[s], range[s+1]) in a
// fixed order and writes the mean (sum * inv_count[s])
__global__ void __launch_bounds__(BLOCK) k_sum_final(const double* __restrict__ partials,
                                                     const int* __restrict__ range,
                                                     const double* __restrict__ inv_count, double* out) {
  const int s = blockIdx.x;
  double v = 0.0;
  for (int i = range[s] + threadIdx.x; i < range[s + 1]; i += BLOCK) v += partials[i];
  const double t = block_sum(v);
  if (threadIdx.x == 0) out[s] = t * inv_count[s];
}

__global__ void __launch_bounds__(BLOCK) k_add_scalar(const DevBox* __restrict__ boxes, const Chunk* __restrict__ chunks,
                                                      double* x, const double* c, double scale) {
  const Chunk ch = chunks[blockIdx.x];
  const DevBox B = boxes[ch.item];
  const int t = ch.start + threadIdx.x;
  if (t >= B.nx * B.ny * B.nz) return;
  const int i = t % B.nx, j = (t / B.nx) % B.ny, k = t / (B.nx * B.ny);
  x[elem_index(B, i, j, k)] += scale * c[B.solve];
}

__global__ void __launch_bounds__(BLOCK) k_scale_valid(const DevBox* __restrict__ boxes,
                                                       const Chunk* __restrict__ chunks, double* x, double scale) {
  const Chunk ch = chunks[blockIdx.x];
  const DevBox B = boxes[ch.item];
  const int t = ch.start + threadIdx.x;
  if (t >= B.nx * B.ny * B.nz) return;
  const int i = t % B.nx, j = (t / B.nx) % B.ny, k = t / (B.nx * B.ny);
  x[elem_index(B, i, j, k)] *= scale;
}

__global__ void __launch_bounds__(BLOCK) k_copy_valid(const DevBox* __restrict__ boxes, const Chunk* __restrict__ chunks,
                                                      double* dst, const double* __restrict__ src) {
  const Chunk ch = chunks[blockIdx.x];
  const DevBox B = boxes[ch.item];
  const int t = ch.start + threadIdx.x;
  if (t >= B.nx * B.ny * B.nz) return;
  const int i = t % B.nx, j = (t / B.nx) % B.ny, k = t / (B.nx * B.ny);
  const int64_t q = elem_index(B, i, j, k);
  dst[q] = src[q];
}

// ------------------------------------------------------------- coefficients

__global__ void __launch_bounds__(BLOCK) k_acoef(const DevBox* __restrict__ boxes, const Chunk* __restrict__ chunks,
                                                 double a, const double* __restrict__ alpha, double* acoef) {
  const Chunk ch = chunks[blockIdx.x];
  const DevBox B = boxes[ch.item];
  const int t = ch.start + threadIdx.x;
  if (t >= B.nx * B.ny * B.nz) return;
  const int i = t % B.nx, j = (t / B.nx) % B.ny, k = t / (B.nx * B.ny);
  const int64_t q = elem_index(B, i, j, k);
  acoef[q] = alpha ? a * alpha[q] : a;
}

// Face beta from cell beta (Sec. "Linear Solvers": beta on faces): harmonic mean of the
// two cells; on a wall face (Dirichlet or Neumann) the interior cell's value.  Each thread writes the
// low face of its cell in every direction and, for the last cell of a row/column, the
// high face too.  The ghosts of beta must hold the neighbouring boxes' values.
__global__ void __launch_bounds__(BLOCK)
    k_faces_from_cell(const DevBox* __restrict__ boxes, const DevGeom* __restrict__ geoms,
                      const Chunk* __restrict__ chunks, const double* __restrict__ beta, double* bx, double* by,
                      double* bz) {
  const Chunk ch = chunks[blockIdx.x];
  const DevBox B = boxes[ch.item];
  const DevGeom G = geoms[B.solve];
  const int t = ch.start + threadIdx.x;
  if (t >= B.nx * B.ny * B.nz) return;
  const int loc[3] = {t % B.nx, (t / B.nx) % B.ny, t / (B.nx * B.ny)};
  const int n[3] = {B.nx, B.ny, B.nz};
  const int64_t q = elem_index(B, loc[0], loc[1], loc[2]);
  double* w[3] = {bx, by, bz};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int64_t st_d = d == 0 ? 1 : (d == 1 ? (int64_t)B.sx : B.sy);
    for (int side = 0; side < 2; ++side) {
      if (side == 1 && loc[d] != n[d] - 1) continue;
      const int64_t qf = q + side * st_d;         // face slot (low face of cell qf)
      const int gf = B.lo[d] + loc[d] + side;      // global face index
      const double bl = beta[qf - st_d], br = beta[qf];
      double v;
      if (G.wall_lo[d] && gf == G.dlo[d]) v = br;
      else if (G.wall_hi[d] && gf == G.dhi[d] + 1) v = bl;
      else v = 2.0 * bl * br / (bl + br);
      w[d][qf] = v;
    }
  }
}

__global__ void __launch_bounds__(BLOCK)
    k_faces_scale(const DevBox* __restrict__ boxes, const DevGeom* __restrict__ geoms, const Chunk* __restrict__ chunks,
                  double b, const double* __restrict__ bx, const double* __restrict__ by, const double* __restrict__ bz,
                  double* wx, double* wy, double* wz) {
  const Chunk ch = chunks[blockIdx.x];
  const DevBox B = boxes[ch.item];
  const DevGeom G = geoms[B.solve];
  const int t = ch.start + threadIdx.x;
  if (t >= B.nx * B.ny * B.nz) return;
  const int loc[3] = {t % B.nx, (t / B.nx) % B.ny, t / (B.nx * B.ny)};
  const int n[3] = {B.nx, B.ny, B.nz};
  const int64_t q = elem_index(B, loc[0], loc[1], loc[2]);
  const double* src[3] = {bx, by, bz};
  double* w[3] = {wx, wy, wz};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int64_t st_d = d == 0 ? 1 : (d == 1 ? (int64_t)B.sx : B.sy);
    for (int side = 0; side < 2; ++side) {
      if (side == 1 && loc[d] != n[d] - 1) continue;
      const int64_t qf = q + side * st_d;
      w[d][qf] = b * src[d][qf] * G.ih2[d];
    }
  }
}

// Coarse coefficients (Sec. "Operations between levels": average of fine data): coarse
// a*alpha = mean of the 8 children; coarse beta face = mean of the 4 fine faces, i.e.
// coarse w = (sum of the 4 fine w) / 16 because h doubles.
__global__ void __launch_bounds__(BLOCK)
    k_coarsen_coefs(const DevBox* __restrict__ fboxes, const DevBox* __restrict__ cboxes, const int* __restrict__ parent,
                    const Chunk* __restrict__ chunks, const double* __restrict__ acf, const double* __restrict__ wxf,
                    const double* __restrict__ wyf, const double* __restrict__ wzf, double* acc, double* wxc,
                    double* wyc, double* wzc) {
  const Chunk ch = chunks[blockIdx.x];
  const DevBox F = fboxes[ch.item];
  const DevBox P = cboxes[parent[ch.item]];
  const int nc[3] = {F.nx >> 1, F.ny >> 1, F.nz >> 1};
  const int t = ch.start + threadIdx.x;
  if (t >= nc[0] * nc[1] * nc[2]) return;
  const int c[3] = {t % nc[0], (t / nc[0]) % nc[1], t / (nc[0] * nc[1])};
  const int64_t qc = elem_index(P, (F.lo[0] >> 1) + c[0] - P.lo[0], (F.lo[1] >> 1) + c[1] - P.lo[1],
                                (F.lo[2] >> 1) + c[2] - P.lo[2]);
  const int64_t qf = elem_index(F, 2 * c[0], 2 * c[1], 2 * c[2]);
  const int64_t fs[3] = {1, (int64_t)F.sx, F.sy};
  const int64_t cs[3] = {1, (int64_t)P.sx, P.sy};
  double s = 0.0;
  for (int dk = 0; dk < 2; ++dk)
    for (int dj = 0; dj < 2; ++dj)
      for (int di = 0; di < 2; ++di) s += acf[qf + di + dj * fs[1] + dk * fs[2]];
  acc[qc] = s * 0.125;
  const double* wf[3] = {wxf, wyf, wzf};
  double* wc[3] = {wxc, wyc, wzc};
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
    for (int side = 0; side < 2; ++side) {
      if (side == 1 && c[d] != nc[d] - 1) continue;
      const int64_t f0 = qf + 2 * side * fs[d];
      const double v = wf[d][f0] + wf[d][f0 + fs[d1]] + wf[d][f0 + fs[d2]] + wf[d][f0 + fs[d1] + fs[d2]];
      wc[d][qc + side * cs[d]] = v * 0.0625;
    }
  }
}

// D = a alpha + sum_f w_f, plus 2 w_f for each face on a quadratic Dirichlet wall (the
// rule's -2 phi_0 term of the ghost, moved into the row's diagonal; the box must have two
// cells along the normal, else the linear rule holds there)
__global__ void __launch_bounds__(BLOCK) k_diag(const DevBox* __restrict__ boxes, const DevGeom* __restrict__ geoms,
                                                const Chunk* __restrict__ chunks,
                                                const double* __restrict__ acoef, const double* __restrict__ wx,
                                                const double* __restrict__ wy, const double* __restrict__ wz,
                                                double* D, double* invD, int split) {
  const Chunk ch = chunks[blockIdx.x];
  const DevBox B = boxes[ch.item];
  const int t = ch.start + threadIdx.x;
  if (t >= B.nx * B.ny * B.nz) return;
  const int i = t % B.nx, j = (t / B.nx) % B.ny, k = t / (B.nx * B.ny);
  const int64_t q = elem_index(B, i, j, k);
  const double s = ((wx[q] + wx[q + 1]) + (wy[q] + wy[q + B.sx])) + (wz[q] + wz[q + B.sy]);
  double d = acoef[q] + s;
  const DevGeom G = geoms[B.solve];
  const int c[3] = {i, j, k}, n[3] = {B.nx, B.ny, B.nz};
  const double* w[3] = {wx, wy, wz};
  for (int a = 0; a < 3; ++a) {
    if (n[a] < 2) continue;
    const int64_t sa = axis_stride(B, a);
    if (G.wall_lo[a] == 3 && c[a] == 0 && B.lo[a] == G.dlo[a]) d += 2.0 * w[a][q];
    if (G.wall_hi[a] == 3 && c[a] == n[a] - 1 && B.lo[a] + n[a] - 1 == G.dhi[a]) d += 2.0 * w[a][q + sa];
  }
  D[q] = d;
  invD[cell_slot(split & SPLIT_INVD, B, i, j, k, q)] = 1.0 / d;
}

template <class S, class T>
__global__ void k_convert(const S* __restrict__ src, T* dst, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    st(dst + i, ld(src + i));
}

inline unsigned grid_of(int n) { return (unsigned)(n > 0 ? n : 0); }

bool g_pdl = false;

// <<<grid, block, smem, s>>>(args...) with the programmatic-serialization attribute when
// dependent launch is on (the kernel must begin with pdl_enter())
template <class... P, class... A>
void launch_pdl(void (*k)(P...), unsigned grid, unsigned block, size_t smem, cudaStream_t s, A&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = g_pdl ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k, std::forward<A>(args)...);
}

}  // namespace

static int64_t g_launches = 0;
void set_pdl(bool on) { g_pdl = on; }
bool pdl_enabled() { return g_pdl; }
int64_t kernel_launch_count() { return g_launches; }
void count_launches(int n) { g_launches += n; }

// ================================================================= launchers

#define GMG_DISPATCH(dt, KERNEL_CALL)                  \
  switch (dt) {                                         \
    case DT_F64: { using T = double; KERNEL_CALL; } break; \
    case DT_F32: { using T = float; KERNEL_CALL; } break;  \
    default: { using T = bf16; KERNEL_CALL; } break;       \
  }

void launch_fill(int dt, const LevelDev& L, void* f, int colour, int copy_mode, cudaStream_t s) {
  if (!L.n_ghost_chunks) return;
  ++g_launches;
  GMG_DISPATCH(dt, launch_pdl(k_fill<T>, grid_of(L.n_ghost_chunks), BLOCK, 0, s, L.boxes, L.ghosts, L.ghost_chunks,
                               (T*)f, colour, copy_mode, L.active));
}

// the split flags of a smoother launch: 1/D as the level keeps it, the right-hand side split
// only when it is the level's own buffer
int smooth_split(const LevelDev& L, bool own_rhs) {
  return (own_rhs ? (L.split & SPLIT_RHS) : 0) | (L.split & SPLIT_INVD);
}

void launch_smooth_update(int dt, const LevelDev& L, void* e, const void* rhs, const Coefs& c, int colour,
                          double* phi, bool push_phi, cudaStream_t s, bool own_rhs) {
  if (!L.n_pair_chunks) return;
  ++g_launches;
  const PushFace* pf = push_phi ? L.push_faces : nullptr;
  const int sp = smooth_split(L, own_rhs);
  GMG_DISPATCH(dt, launch_pdl(k_smooth_update<T>, grid_of(L.n_pair_chunks), BLOCK, 0, s, L.boxes, L.pair_chunks,
                              (T*)e, (const T*)rhs, (const typename CoefOf<T>::type*)c.wx,
                              (const typename CoefOf<T>::type*)c.wy, (const typename CoefOf<T>::type*)c.wz,
                              (const typename CoefOf<T>::type*)c.invD, colour, L.active, phi, pf, L.rev, sp));
}

void launch_smooth(int dt, const LevelDev& L, void* phi, const void* rhs, const Coefs& c, int colour, cudaStream_t s,
                   bool push, bool vec, bool own_rhs) {
  if (!L.n_pair_chunks) return;
  ++g_launches;
  const PushFace* pf = push ? L.push_faces : nullptr;
  const int sp = smooth_split(L, own_rhs);
  if (vec && dt == DT_F64) {
    launch_pdl(k_smooth_d2, grid_of(L.n_pair_chunks), BLOCK, 0, s, L.boxes, L.pair_chunks, (double*)phi,
               (const double*)rhs, (const double*)c.wx, (const double*)c.wy, (const double*)c.wz,
               (const double*)c.invD, colour, L.active, pf, L.rev, sp);
    return;
  }
  if (vec && dt != DT_F64 && L.quad_chunks && L.n_quad_chunks > 0) {
    const float *wx = (const float*)c.wx, *wy = (const float*)c.wy, *wz = (const float*)c.wz;
    const float* invD = (const float*)c.invD;
    if (dt == DT_F32)
      launch_pdl(k_smooth4<float>, grid_of(L.n_quad_chunks), BLOCK, 0, s, L.boxes, L.quad_chunks, (float*)phi,
                 (const float*)rhs, wx, wy, wz, invD, colour, L.active, pf, L.rev, sp);
    else
      launch_pdl(k_smooth4<bf16>, grid_of(L.n_quad_chunks), BLOCK, 0, s, L.boxes, L.quad_chunks, (bf16*)phi,
                 (const bf16*)rhs, wx, wy, wz, invD, colour, L.active, pf, L.rev, sp);
    return;
  }
  GMG_DISPATCH(dt, launch_pdl(k_smooth<T>, grid_of(L.n_pair_chunks), BLOCK, 0, s, L.boxes, L.pair_chunks, (T*)phi,
                              (const T*)rhs, (const typename CoefOf<T>::type*)c.wx,
                              (const typename CoefOf<T>::type*)c.wy, (const typename CoefOf<T>::type*)c.wz,
                              (const typename CoefOf<T>::type*)c.invD, colour, L.active, pf, L.rev, sp));
}

void launch_smooth_pro(int dt, const LevelDev& L, const LevelDev& Lc, void* phi, const void* rhs, const Coefs& c,
                       int colour, const void* ec, cudaStream_t s, bool push, bool own_rhs) {
  if (!L.n_pair_chunks) return;
  ++g_launches;
  const PushFace* pf = push ? L.push_faces : nullptr;
  const int sp = smooth_split(L, own_rhs);
  GMG_DISPATCH(dt, launch_pdl(k_smooth_pro<T>, grid_of(L.n_pair_chunks), BLOCK, 0, s, L.boxes, L.pair_chunks, (T*)phi,
                              (const T*)rhs, (const typename CoefOf<T>::type*)c.wx,
                              (const typename CoefOf<T>::type*)c.wy, (const typename CoefOf<T>::type*)c.wz,
                              (const typename CoefOf<T>::type*)c.invD, colour, L.active, pf, L.rev, sp, (const T*)ec,
                              Lc.boxes, L.parent));
}

void launch_smooth_prolong(int dt, const LevelDev& L, const LevelDev& Lf, void* phi, const void* rhs, const Coefs& c,
                           int colour, void* fine, cudaStream_t s, bool push, bool fpush) {
  if (!L.n_pair_chunks) return;
  ++g_launches;
  const PushFace* pf = push ? L.push_faces : nullptr;
  const PushFace* ff = fpush ? Lf.push_faces : nullptr;
  GMG_DISPATCH(dt, launch_pdl(k_smooth_prolong<T>, grid_of(L.n_pair_chunks), BLOCK, 0, s, L.boxes, L.pair_chunks,
                              (T*)phi, (const T*)rhs, (const typename CoefOf<T>::type*)c.wx,
                              (const typename CoefOf<T>::type*)c.wy, (const typename CoefOf<T>::type*)c.wz,
                              (const typename CoefOf<T>::type*)c.invD, colour, L.active, pf, L.rev, (T*)fine,
                              Lf.boxes, L.child, ff));
}

// residual work list: pair items over every box (the bottom level included)
void launch_residual(int dt, int rdt, const LevelDev& L, const void* phi, const void* rhs, const Coefs& c, void* r,
                     unsigned long long* maxbits, const double* shift, cudaStream_t s, void* e, const void* invDe,
                     bool push, int settled, bool own_r) {
  const int rsplit = own_r ? L.split : 0;
  if (settled >= 0 && (dt != DT_F64 || rdt != DT_F64 || !r)) settled = -1;  // (defined for FP64 only)
  if (!L.n_pair_all_chunks) return;
  ++g_launches;
  const PushFace* pf = push ? L.push_faces : nullptr;
#define GMG_RESID_LAUNCH(TR, RS)                                                                          \
  launch_pdl(k_residual<T, TR, std::is_same<T, double>::value && std::is_same<TR, double>::value ? 6 : 0, RS>, \
             grid_of(L.n_pair_all_chunks), BLOCK, 0, s, L.boxes, L.geoms, L.pair_all_chunks, (const T*)phi,   \
             (const T*)rhs, (const typename CoefOf<T>::type*)c.wx, (const typename CoefOf<T>::type*)c.wy,      \
             (const typename CoefOf<T>::type*)c.wz, (const typename CoefOf<T>::type*)c.D, (TR*)r, maxbits,     \
             shift, (TR*)e, (const typename CoefOf<TR>::type*)invDe, pf, settled, L.rev)
#define GMG_RESID(TR)                                                                                     \
  GMG_DISPATCH(dt, rsplit ? GMG_RESID_LAUNCH(TR, true) : GMG_RESID_LAUNCH(TR, false))
  switch (rdt) {
    case DT_F64: GMG_RESID(double); break;
    case DT_F32: GMG_RESID(float); break;
    default: GMG_RESID(bf16); break;
  }
#undef GMG_RESID
#undef GMG_RESID_LAUNCH

}

void launch_resid_restrict(int dt, const LevelDev& f, const LevelDev& c, const void* phi, const void* rhs,
                           const Coefs& cf, void* rc, cudaStream_t s, bool settled_black, bool own_rhs, void* ec,
                           const void* invDc, bool cpush) {
  if (!f.n_coarse_chunks) return;
  ++g_launches;
  const int split = own_rhs ? (f.split & SPLIT_RHS) : 0;
  const PushFace* pf = (ec && cpush) ? c.push_faces : nullptr;
  GMG_DISPATCH(dt, launch_pdl(k_resid_restrict<T, T>, grid_of(f.n_coarse_chunks), BLOCK, 0, s, f.boxes, f.geoms, c.boxes,
                              f.parent, f.coarse_chunks, (const T*)phi, (const T*)rhs,
                              (const typename CoefOf<T>::type*)cf.wx, (const typename CoefOf<T>::type*)cf.wy,
                              (const typename CoefOf<T>::type*)cf.wz, (const typename CoefOf<T>::type*)cf.D, (T*)rc,
                              f.active, settled_black ? 1 : 0, f.rev, split, (T*)ec,
                              (const typename CoefOf<T>::type*)invDc, pf));

}

void launch_restrict(int dt, const LevelDev& f, const LevelDev& c, const void* fine, void* coarse, cudaStream_t s) {
  if (!f.n_coarse_chunks) return;
  ++g_launches;
  GMG_DISPATCH(dt, (k_restrict<T><<<grid_of(f.n_coarse_chunks), BLOCK, 0, s>>>(f.boxes, c.boxes, f.parent,
                                                                                 f.coarse_chunks, (const T*)fine,
                                                                                 (T*)coarse)));
}

void launch_prolong_add(int dt, const LevelDev& f, const LevelDev& c, const void* coarse, void* fine, cudaStream_t s,
                        bool push) {
  if (!f.n_coarse_chunks) return;
  ++g_launches;
  const PushFace* pf = push ? f.push_faces : nullptr;
  GMG_DISPATCH(dt, launch_pdl(k_prolong_add<T, std::is_same<T, double>::value ? 8 : 0>, grid_of(f.n_coarse_chunks),
                              BLOCK, 0, s, f.boxes, c.boxes,
                              f.parent, f.coarse_chunks, (const T*)coarse, (T*)fine, f.active, pf, f.rev));
}

void launch_prolong_tri(int dt, const LevelDev& f, const LevelDev& c, const void* coarse, void* fine, cudaStream_t s,
                        bool push) {
  if (!f.n_coarse_chunks) return;
  ++g_launches;
  const PushFace* pf = push ? f.push_faces : nullptr;
  GMG_DISPATCH(dt, launch_pdl(k_prolong_tri<T, std::is_same<T, double>::value ? 4 : 0>, grid_of(f.n_coarse_chunks),
                              BLOCK, 0, s, f.boxes, c.boxes, f.parent, f.coarse_chunks, (const T*)coarse, (T*)fine,
                              f.active, pf, f.rev));
}

void launch_fill_ec(int dt, const LevelDev& L, void* f, cudaStream_t s) {
  if (!L.n_ec_ghosts) return;
  ++g_launches;
  GMG_DISPATCH(dt, launch_pdl(k_fill_list<T>, (unsigned)((L.n_ec_ghosts + BLOCK - 1) / BLOCK), BLOCK, 0, s,
                              L.ec_ghosts, L.n_ec_ghosts, (T*)f));
}

void launch_add_correction(int dt, const LevelDev& L, double* phi, const void* e, cudaStream_t s, bool push) {
  if (!L.n_pair_all_chunks) return;
  ++g_launches;
  const PushFace* pf = push ? L.push_faces : nullptr;
  GMG_DISPATCH(dt, launch_pdl(k_add_correction<T>, grid_of(L.n_pair_all_chunks), BLOCK, 0, s, L.boxes,
                              L.pair_all_chunks, phi, (const T*)e, L.active, pf));
}

void launch_pack(int dt, const LevelDev& L, const int dlo[3], const int dn[3], const double* dense, void* boxed,
                 cudaStream_t s) {
  if (!L.n_cell_chunks) return;
  ++g_launches;
  int3 lo = make_int3(dlo[0], dlo[1], dlo[2]), n = make_int3(dn[0], dn[1], dn[2]);
  GMG_DISPATCH(dt, (k_pack<T><<<grid_of(L.n_cell_chunks), BLOCK, 0, s>>>(L.boxes, L.cell_chunks, lo, n, dense,
                                                                          (T*)boxed)));
}

void launch_unpack(int dt, const LevelDev& L, const int dlo[3], const int dn[3], const void* boxed, double* dense,
                   cudaStream_t s) {
  if (!L.n_cell_chunks) return;
  ++g_launches;
  int3 lo = make_int3(dlo[0], dlo[1], dlo[2]), n = make_int3(dn[0], dn[1], dn[2]);
  GMG_DISPATCH(dt, (k_unpack<T><<<grid_of(L.n_cell_chunks), BLOCK, 0, s>>>(L.boxes, L.cell_chunks, lo, n,
                                                                            (const T*)boxed, dense)));
}

void launch_norm_max(const LevelDev& L, const double* x, unsigned long long* maxbits, cudaStream_t s) {
  if (!L.n_cell_chunks) return;
  ++g_launches;
  k_norm_max<<<grid_of(L.n_cell_chunks), BLOCK, 0, s>>>(L.boxes, L.cell_chunks, x, maxbits);
}

void launch_sum(const LevelDev& L, const double* x, double* partials, double* out, cudaStream_t s) {
  if (!L.n_cell_chunks) return;
  ++g_launches;
  ++g_launches;
  k_sum_partial<<<grid_of(L.n_cell_chunks), BLOCK, 0, s>>>(L.boxes, L.cell_chunks, x, partials);
  k_sum_final<<<grid_of(L.nsolves), BLOCK, 0, s>>>(partials, L.solve_chunk_range, L.inv_count, out);
}

void launch_add_scalar(const LevelDev& L, double* x, const double* c, double scale, cudaStream_t s) {
  if (!L.n_cell_chunks) return;
  ++g_launches;
  k_add_scalar<<<grid_of(L.n_cell_chunks), BLOCK, 0, s>>>(L.boxes, L.cell_chunks, x, c, scale);
}

void launch_scale_valid(const LevelDev& L, double* x, double scale, cudaStream_t s) {
  if (!L.n_cell_chunks) return;
  ++g_launches;
  k_scale_valid<<<grid_of(L.n_cell_chunks), BLOCK, 0, s>>>(L.boxes, L.cell_chunks, x, scale);
}

void launch_copy_valid(const LevelDev& L, double* dst, const double* src, cudaStream_t s) {
  if (!L.n_cell_chunks) return;
  ++g_launches;
  k_copy_valid<<<grid_of(L.n_cell_chunks), BLOCK, 0, s>>>(L.boxes, L.cell_chunks, dst, src);
}

void launch_acoef(const LevelDev& L, double a, const double* alpha, double* acoef, cudaStream_t s) {
  if (!L.n_cell_chunks) return;
  ++g_launches;
  k_acoef<<<grid_of(L.n_cell_chunks), BLOCK, 0, s>>>(L.boxes, L.cell_chunks, a, alpha, acoef);
}

void launch_faces_from_cell(const LevelDev& L, const double* beta, double* bx, double* by, double* bz, cudaStream_t s) {
  if (!L.n_cell_chunks) return;
  ++g_launches;
  k_faces_from_cell<<<grid_of(L.n_cell_chunks), BLOCK, 0, s>>>(L.boxes, L.geoms, L.cell_chunks, beta, bx, by, bz);
}

void launch_faces_scale(const LevelDev& L, double b, const double* bx, const double* by, const double* bz, double* wx,
                        double* wy, double* wz, cudaStream_t s) {
  if (!L.n_cell_chunks) return;
  ++g_launches;
  k_faces_scale<<<grid_of(L.n_cell_chunks), BLOCK, 0, s>>>(L.boxes, L.geoms, L.cell_chunks, b, bx, by, bz, wx, wy,
                                                           wz);
}

void launch_coarsen_coefs(const LevelDev& f, const LevelDev& c, const double* acf, const double* wxf,
                          const double* wyf, const double* wzf, double* acc, double* wxc, double* wyc, double* wzc,
                          cudaStream_t s) {
  if (!f.n_coarse_chunks) return;
  ++g_launches;
  k_coarsen_coefs<<<grid_of(f.n_coarse_chunks), BLOCK, 0, s>>>(f.boxes, c.boxes, f.parent, f.coarse_chunks, acf, wxf,
                                                               wyf, wzf, acc, wxc, wyc, wzc);
}

// dst (type T, the level's own right-hand side layout: colour-split if split) = src (double,
// the ordinary layout) on every valid cell
template <class S, class T>
__global__ void __launch_bounds__(BLOCK) k_to_rhs(const DevBox* __restrict__ boxes, const Chunk* __restrict__ chunks,
                                                  const S* __restrict__ src, T* dst, int split) {
  const Chunk ch = chunks[blockIdx.x];
  const DevBox B = boxes[ch.item];
  const int t = ch.start + threadIdx.x;
  if (t >= B.nx * B.ny * B.nz) return;
  const int i = t % B.nx, j = (t / B.nx) % B.ny, k = t / (B.nx * B.ny);
  const int64_t q = elem_index(B, i, j, k);
  if (std::is_same<S, T>::value)
    dst[cell_slot(split & SPLIT_RHS, B, i, j, k, q)] = *reinterpret_cast<const T*>(src + q);
  else
    st(dst + cell_slot(split & SPLIT_RHS, B, i, j, k, q), ld(src + q));
}

void launch_to_rhs(int dt, const LevelDev& L, const double* src, void* dst, cudaStream_t s) {
  if (!(L.split & SPLIT_RHS)) {
    launch_convert(DT_F64, dt, src, dst, L.nelem, s);
    return;
  }
  if (!L.n_cell_chunks) return;
  ++g_launches;
  GMG_DISPATCH(dt, (k_to_rhs<double, T><<<grid_of(L.n_cell_chunks), BLOCK, 0, s>>>(L.boxes, L.cell_chunks, src,
                                                                                     (T*)dst, L.split)));
}

void launch_copy_to_rhs(int dt, const LevelDev& L, const void* src, void* dst, cudaStream_t s) {
  if (!(L.split & SPLIT_RHS)) {
    cudaMemcpyAsync(dst, src, (size_t)L.nelem * (dt == DT_F64 ? 8 : (dt == DT_F32 ? 4 : 2)), cudaMemcpyDeviceToDevice,
                    s);
    return;
  }
  if (!L.n_cell_chunks) return;
  ++g_launches;
  GMG_DISPATCH(dt, (k_to_rhs<T, T><<<grid_of(L.n_cell_chunks), BLOCK, 0, s>>>(L.boxes, L.cell_chunks, (const T*)src,
                                                                                (T*)dst, L.split)));
}

void launch_diag(const LevelDev& L, const double* acoef, const double* wx, const double* wy, const double* wz,
                 double* D, double* invD, cudaStream_t s) {
  if (!L.n_cell_chunks) return;
  ++g_launches;
  k_diag<<<grid_of(L.n_cell_chunks), BLOCK, 0, s>>>(L.boxes, L.geoms, L.cell_chunks, acoef, wx, wy, wz, D, invD,
                                                    L.split);
}

void launch_convert(int dt, int dt2, const void* src, void* dst, int64_t n, cudaStream_t s) {
  if (n <= 0) return;
  ++g_launches;
  const unsigned g = (unsigned)std::min<int64_t>((n + BLOCK - 1) / BLOCK, 152 * 16);
#define GMG_CVT(TD) GMG_DISPATCH(dt, (k_convert<T, TD><<<g, BLOCK, 0, s>>>((const T*)src, (TD*)dst, n)))
  switch (dt2) {
    case DT_F64: GMG_CVT(double); break;
    case DT_F32: GMG_CVT(float); break;
    default: GMG_CVT(bf16); break;
  }
#undef GMG_CVT
}

void launch_to_float(const double* src, float* dst, int64_t n, cudaStream_t s) {
  launch_convert(DT_F64, DT_F32, src, dst, n, s);
}

}  // namespace gmg
