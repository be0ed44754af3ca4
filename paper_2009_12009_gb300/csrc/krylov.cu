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

}  // namespace gmg
