// bottom.cu -- bottom solve of the V-cycle (Sec. "Linear Solvers": Krylov bottom
// solver): unpreconditioned BiCGStab (van der Vorst 1992) or conjugate gradients (Hestenes
// and Stiefel 1952) in FP64, x0 = 0, one thread block per bottom problem running the whole
// iteration on the device (no host round trip per iteration).  Stops at ||r||_inf <= tol * ||r0||_inf, after maxit iterations,
// or on breakdown.  Singular problems (no Dirichlet wall, a = 0) project the right-hand side
// and the result onto zero mean.  Dot products are reduced in a fixed order, so the
// result is deterministic.
#include <cuda_bf16.h>

#include <utility>

#include "kernels.h"

namespace gmg {
namespace {

using bf16 = __nv_bfloat16;
constexpr int BT = 512;  // threads of the bottom block

__device__ __forceinline__ double ldd(const double* p) { return *p; }
__device__ __forceinline__ double ldd(const float* p) { return (double)*p; }
__device__ __forceinline__ double ldd(const bf16* p) { return (double)__bfloat162float(*p); }
__device__ __forceinline__ void std_(double* p, double v) { *p = v; }
__device__ __forceinline__ void std_(float* p, double v) { *p = (float)v; }
__device__ __forceinline__ void std_(bf16* p, double v) { *p = __float2bfloat16_rn((float)v); }

// block-wide sum, result broadcast to every thread (fixed reduction order)
__device__ double bsum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < BT / 32; ++w) s += sh[w];
    sh[BT / 32] = s;
  }
  __syncthreads();
  return sh[BT / 32];
}

__device__ double bmax(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < BT / 32; ++w) s = fmax(s, sh[w]);
    sh[BT / 32] = s;
  }
  __syncthreads();
  return sh[BT / 32];
}

struct BotCtx {
  const BotCell* cells;
  const BotGhost* ghosts;
  int ncell, nghost;
  const double *wx, *wy, *wz, *D;
};

// out = A in on the problem's cells (ghosts of `in` filled first)
__device__ void bot_apply(const BotCtx& c, double* in, double* out) {
  for (int g = threadIdx.x; g < c.nghost; g += BT) {
    const BotGhost G = c.ghosts[g];
    in[G.dst] = G.sign * in[G.src];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < c.ncell; i += BT) {
    const BotCell C = c.cells[i];
    const int64_t q = C.q, sx = C.sx, sy = C.sy;
    double v = c.D[q] * in[q];
    v = fma(-c.wx[q], in[q - 1], v);
    v = fma(-c.wx[q + 1], in[q + 1], v);
    v = fma(-c.wy[q], in[q - sx], v);
    v = fma(-c.wy[q + sx], in[q + sx], v);
    v = fma(-c.wz[q], in[q - sy], v);
    v = fma(-c.wz[q + sy], in[q + sy], v);
    out[q] = v;
  }
  __syncthreads();
}

__device__ double bot_dot(const BotCtx& c, const double* x, const double* y, double* sh) {
  double s = 0.0;
  for (int i = threadIdx.x; i < c.ncell; i += BT) s += x[c.cells[i].q] * y[c.cells[i].q];
  return bsum(s, sh);
}

__device__ double bot_norm(const BotCtx& c, const double* x, double* sh) {
  double s = 0.0;
  for (int i = threadIdx.x; i < c.ncell; i += BT) s = fmax(s, fabs(x[c.cells[i].q]));
  return bmax(s, sh);
}

__device__ double bot_sum(const BotCtx& c, const double* x, double* sh) {
  double s = 0.0;
  for (int i = threadIdx.x; i < c.ncell; i += BT) s += x[c.cells[i].q];
  return bsum(s, sh);
}

template <class T>
__global__ void __launch_bounds__(BT) k_bottom(const BotDesc* __restrict__ descs, const BotCell* __restrict__ cells,
                                               const BotGhost* __restrict__ ghosts, const T* __restrict__ rhs, T* xout,
                                               const double* __restrict__ wx, const double* __restrict__ wy,
                                               const double* __restrict__ wz, const double* __restrict__ D,
                                               double* work, int64_t nelem, int maxit, double tol, int* iters,
                                               const int* __restrict__ active, int cg) {
  __shared__ double sh[BT / 32 + 1];
  // programmatic dependent launch: wait for the predecessor before any global access
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const BotDesc P = descs[blockIdx.x];
  if (active && !active[P.solve]) return;
  BotCtx c{cells + P.cell0, ghosts + P.ghost0, P.ncell, P.nghost, wx, wy, wz, D};
  double* r = work;
  double* rh = work + nelem;
  double* p = work + 2 * nelem;
  double* v = work + 3 * nelem;
  double* s = work + 4 * nelem;
  double* t = work + 5 * nelem;
  double* x = work + 6 * nelem;
  for (int i = threadIdx.x; i < c.ncell; i += BT) {
    const int64_t q = c.cells[i].q;
    r[q] = ldd(rhs + q);
    p[q] = 0.0;
    v[q] = 0.0;
    x[q] = 0.0;
  }
  __syncthreads();
  if (P.singular) {
    const double mean = bot_sum(c, r, sh) / (double)c.ncell;
    for (int i = threadIdx.x; i < c.ncell; i += BT) r[c.cells[i].q] -= mean;
    __syncthreads();
  }
  for (int i = threadIdx.x; i < c.ncell; i += BT) rh[c.cells[i].q] = r[c.cells[i].q];
  __syncthreads();
  const double r0 = bot_norm(c, r, sh);
  double rho_old = 1.0, alpha = 1.0, omega = 1.0;
  int it = 0;
  if (cg && r0 > 0.0) {
    // conjugate gradients: p = r; alpha = (r,r)/(p,Ap); x += alpha p; r -= alpha Ap;
    // beta = (r',r')/(r,r); p = r' + beta p; breakdown when (p,Ap) is not positive
    for (int i = threadIdx.x; i < c.ncell; i += BT) p[c.cells[i].q] = r[c.cells[i].q];
    __syncthreads();
    double rho = bot_dot(c, r, r, sh);
    for (it = 1; it <= maxit; ++it) {
      bot_apply(c, p, v);
      const double pv = bot_dot(c, p, v, sh);
      if (!(pv > 0.0)) { --it; break; }
      const double al = rho / pv;
      for (int i = threadIdx.x; i < c.ncell; i += BT) {
        const int64_t q = c.cells[i].q;
        x[q] += al * p[q];
        r[q] -= al * v[q];
      }
      __syncthreads();
      if (bot_norm(c, r, sh) <= tol * r0) break;
      const double rho_new = bot_dot(c, r, r, sh);
      const double be = rho_new / rho;
      rho = rho_new;
      for (int i = threadIdx.x; i < c.ncell; i += BT) {
        const int64_t q = c.cells[i].q;
        p[q] = r[q] + be * p[q];
      }
      __syncthreads();
    }
    if (it > maxit) it = maxit;
  } else if (r0 > 0.0) {
    for (it = 1; it <= maxit; ++it) {
      const double rho = bot_dot(c, rh, r, sh);
      if (fabs(rho) < 1e-300) { --it; break; }
      const double beta = (rho / rho_old) * (alpha / omega);
      for (int i = threadIdx.x; i < c.ncell; i += BT) {
        const int64_t q = c.cells[i].q;
        p[q] = r[q] + beta * (p[q] - omega * v[q]);
      }
      __syncthreads();
      bot_apply(c, p, v);
      const double rv = bot_dot(c, rh, v, sh);
      if (fabs(rv) < 1e-300) { --it; break; }
      alpha = rho / rv;
      for (int i = threadIdx.x; i < c.ncell; i += BT) {
        const int64_t q = c.cells[i].q;
        s[q] = r[q] - alpha * v[q];
      }
      __syncthreads();
      if (bot_norm(c, s, sh) <= tol * r0) {
        for (int i = threadIdx.x; i < c.ncell; i += BT) x[c.cells[i].q] += alpha * p[c.cells[i].q];
        __syncthreads();
        break;
      }
      bot_apply(c, s, t);
      const double tt = bot_dot(c, t, t, sh);
      if (tt == 0.0) {
        for (int i = threadIdx.x; i < c.ncell; i += BT) x[c.cells[i].q] += alpha * p[c.cells[i].q];
        __syncthreads();
        break;
      }
      omega = bot_dot(c, t, s, sh) / tt;
      for (int i = threadIdx.x; i < c.ncell; i += BT) {
        const int64_t q = c.cells[i].q;
        x[q] += alpha * p[q] + omega * s[q];
        r[q] = s[q] - omega * t[q];
      }
      __syncthreads();
      if (bot_norm(c, r, sh) <= tol * r0) break;
      rho_old = rho;
    }
    if (it > maxit) it = maxit;
  }
  double shift = 0.0;
  if (P.singular) shift = bot_sum(c, x, sh) / (double)c.ncell;
  for (int i = threadIdx.x; i < c.ncell; i += BT) {
    const int64_t q = c.cells[i].q;
    std_(xout + q, x[q] - shift);
  }
  if (threadIdx.x == 0 && iters) iters[P.solve] = it;
}

}  // namespace

template <class T, class... A>
static void launch_bottom_kernel(int nblocks, cudaStream_t s, A&&... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(nblocks);
  cfg.blockDim = dim3(BT);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  cudaLaunchKernelEx(&cfg, k_bottom<T>, std::forward<A>(args)...);
}

void launch_bottom(int dt, const LevelDev& L, const void* rhs, void* x, const Coefs& c, const BottomArgs& a,
                   cudaStream_t s) {
  if (!L.n_bot) return;
  count_launches(1);
  const double* wx = (const double*)c.wx;
  const double* wy = (const double*)c.wy;
  const double* wz = (const double*)c.wz;
  const double* D = (const double*)c.D;
  switch (dt) {
    case DT_F64:
      launch_bottom_kernel<double>(L.n_bot, s, L.bot_descs, L.bot_cells, L.bot_ghosts, (const double*)rhs, (double*)x,
                                   wx, wy, wz, D, a.work, L.nelem, a.maxit, a.tol, a.iters, L.active, a.cg);
      break;
    case DT_F32:
      launch_bottom_kernel<float>(L.n_bot, s, L.bot_descs, L.bot_cells, L.bot_ghosts, (const float*)rhs, (float*)x,
                                  wx, wy, wz, D, a.work, L.nelem, a.maxit, a.tol, a.iters, L.active, a.cg);
      break;
    default:
      launch_bottom_kernel<bf16>(L.n_bot, s, L.bot_descs, L.bot_cells, L.bot_ghosts, (const bf16*)rhs, (bf16*)x, wx,
                                 wy, wz, D, a.work, L.nelem, a.maxit, a.tol, a.iters, L.active, a.cg);
      break;
  }
}

}  // namespace gmg
