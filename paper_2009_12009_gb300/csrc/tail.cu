// tail.cu -- the coarse end of the V-cycle (Sec. "Linear Solvers": geometric multigrid
// with a Krylov bottom solve), one thread block per problem.
//
// Below a few thousand cells a level's grid launches are pure latency: a ghost exchange or
// a colour sweep moves kilobytes but costs a launch and a dependent-load chain each.  Here
// one block runs every remaining step of its problem -- ghost fills, red-black sweeps,
// residual restriction, the BiCGStab bottom solve, interpolation and post-smoothing --
// with a block barrier between steps, from the first level with at most TAIL_MAX_CELLS
// cells down to the bottom and back.  The arithmetic of every step is that of the grid
// kernels (kernels.cu, bottom.cu), in the same order per cell; only the order of the
// bottom solve's dot-product additions differs.
//
// Two forms: k_vtail reads and writes the levels' global arrays at every step;
// k_vtail_dense (the default where the levels fit) first copies each level into shared
// memory as one padded array over the problem's domain and runs every step there, bitwise
// the same values.  Both leave the ghosts of their first level current when they return.
#include <cuda_bf16.h>

#include "kernels.h"

namespace gmg {
namespace {

using bf16 = __nv_bfloat16;
constexpr int TT = 512;  // threads of a tail block

template <class T> struct Ar { using type = float; };
template <> struct Ar<double> { using type = double; };
template <class T> struct Cf { using type = float; };
template <> struct Cf<double> { using type = double; };

__device__ __forceinline__ double tld(const double* p) { return *p; }
__device__ __forceinline__ float tld(const float* p) { return *p; }
__device__ __forceinline__ float tld(const bf16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ void tst(double* p, double v) { *p = v; }
__device__ __forceinline__ void tst(float* p, float v) { *p = v; }
__device__ __forceinline__ void tst(bf16* p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void tst_d(double* p, double v) { *p = v; }
__device__ __forceinline__ void tst_d(float* p, double v) { *p = (float)v; }
__device__ __forceinline__ void tst_d(bf16* p, double v) { *p = __float2bfloat16_rn((float)v); }

// block-wide sum / max, broadcast to every thread; fixed reduction order
__device__ double tsum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < TT / 32 ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) sh[TT / 32] = w;
  }
  __syncthreads();
  return sh[TT / 32];
}

__device__ double tmax(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    double w = threadIdx.x < TT / 32 ? sh[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) w = fmax(w, __shfl_down_sync(0xffffffffu, w, o));
    if (threadIdx.x == 0) sh[TT / 32] = w;
  }
  __syncthreads();
  return sh[TT / 32];
}

// ghosts of one parity (or both: parity -1) of field f
template <class T>
__device__ void t_fill(const TailLevel& L, const BotGhost* __restrict__ ghosts, T* f, int parity) {
  const int g0 = L.ghost0 + (parity == 1 ? L.nghost[0] : 0);
  const int n = parity < 0 ? L.nghost[0] + L.nghost[1] : (parity ? L.nghost[1] : L.nghost[0]);
  for (int i = threadIdx.x; i < n; i += TT) {
    const BotGhost G = ghosts[g0 + i];
    const auto v = tld(f + G.src);
    tst(f + G.dst, G.sign < 0 ? -v : v);
  }
}

// one Gauss-Seidel update of the cell at q: phi = invD * (rhs + sum_f w_f phi_nbr), as k_smooth
template <class T, class C>
__device__ __forceinline__ void gs_cell(T* phi, const T* rhs, const C* wx, const C* wy, const C* wz, const C* invD,
                                        int64_t q, int64_t sx, int64_t sy) {
  using A = typename Ar<T>::type;
  A s = tld(rhs + q);
  s = fma((A)wx[q], (A)tld(phi + q - 1), s);
  s = fma((A)wx[q + 1], (A)tld(phi + q + 1), s);
  s = fma((A)wy[q], (A)tld(phi + q - sx), s);
  s = fma((A)wy[q + sx], (A)tld(phi + q + sx), s);
  s = fma((A)wz[q], (A)tld(phi + q - sy), s);
  s = fma((A)wz[q + sy], (A)tld(phi + q + sy), s);
  tst(phi + q, s * (A)invD[q]);
}

// one Gauss-Seidel colour of a level
template <class T>
__device__ void t_smooth(const TailLevel& L, const BotCell* __restrict__ cells, T* phi, const T* rhs,
                         const typename Cf<T>::type* wx, const typename Cf<T>::type* wy,
                         const typename Cf<T>::type* wz, const typename Cf<T>::type* invD, int colour) {
  const int c0 = L.cell0 + (colour ? L.ncell[0] : 0);
  const int nc = colour ? L.ncell[1] : L.ncell[0];
  for (int i = threadIdx.x; i < nc; i += TT) {
    const BotCell C = cells[c0 + i];
    gs_cell(phi, rhs, wx, wy, wz, invD, C.q, (int64_t)C.sx, C.sy);
  }
}

template <class T, class C>
__device__ __forceinline__ typename Ar<T>::type t_resid(const T* phi, const T* rhs, const C* wx, const C* wy,
                                                        const C* wz, const C* D, int64_t q, int64_t sx, int64_t sy) {
  using A = typename Ar<T>::type;
  A v = (A)tld(rhs + q);
  v = fma(-(A)D[q], (A)tld(phi + q), v);
  v = fma((A)wx[q], (A)tld(phi + q - 1), v);
  v = fma((A)wx[q + 1], (A)tld(phi + q + 1), v);
  v = fma((A)wy[q], (A)tld(phi + q - sx), v);
  v = fma((A)wy[q + sx], (A)tld(phi + q + sx), v);
  v = fma((A)wz[q], (A)tld(phi + q - sy), v);
  v = fma((A)wz[q + sy], (A)tld(phi + q + sy), v);
  return v;
}

// xor-butterfly warp reductions.  Only the lanes below span (a power of two) hold values --
// the others hold 0 -- so the steps across wider distances, which would add those zeros, are
// left out; the lanes below span then hold the same bits (a + b == b + a) and lane 0's
// result is broadcast, so that every lane of the warp returns the same value (the callers'
// loop exits and warp barriers depend on it).
__device__ __forceinline__ double wsum(double v, int span) {
  for (int o = 16; o > 0; o >>= 1)
    if (o < span) v += __shfl_xor_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);
}
__device__ __forceinline__ double wmax(double v, int span) {
  for (int o = 16; o > 0; o >>= 1)
    if (o < span) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return __shfl_sync(0xffffffffu, v, 0);
}
// two independent sums at once (their steps interleave; each sum is the one wsum gives)
__device__ __forceinline__ void wsum2(double& a, double& b, int span) {
  for (int o = 16; o > 0; o >>= 1)
    if (o < span) {
      const double x = __shfl_xor_sync(0xffffffffu, a, o), y = __shfl_xor_sync(0xffffffffu, b, o);
      a += x;
      b += y;
    }
  a = __shfl_sync(0xffffffffu, a, 0);
  b = __shfl_sync(0xffffffffu, b, 0);
}
// a sum and a max at once
__device__ __forceinline__ void wsum_max(double& a, double& m, int span) {
  for (int o = 16; o > 0; o >>= 1)
    if (o < span) {
      const double x = __shfl_xor_sync(0xffffffffu, a, o), y = __shfl_xor_sync(0xffffffffu, m, o);
      a += x;
      m = fmax(m, y);
    }
  a = __shfl_sync(0xffffffffu, a, 0);
  m = __shfl_sync(0xffffffffu, m, 0);
}

constexpr int WS = TAIL_WARP_CELLS;  // cell slots of the warp bottom solve

// Shared memory of the warp bottom solve: p and s (the vectors the operator is applied to)
// in the problem's own element layout from bot_base, with ghosts; the other vectors, the
// coefficients and the cell offsets per cell slot.
struct WarpBottomSmem {
  double p[TAIL_WARP_SPAN], s[TAIL_WARP_SPAN];
  double D[WS], wxm[WS], wxp[WS], wym[WS], wyp[WS], wzm[WS], wzp[WS];
  double r[WS], rh[WS], v[WS], t[WS], x[WS];
  int q[WS], sx[WS], sy[WS];
};

// BiCGStab (van der Vorst 1992) of a small bottom problem in warp 0 (lanes own cell slots
// lane, lane + 32, ...): the steps and stopping rules of the block version, with warp
// barriers instead of block barriers and the operator applied from shared memory.
template <class T>
__device__ void warp_bottom(const TailDesc& Dd, const BotCell* __restrict__ cells, int nc,
                            const BotGhost* __restrict__ ghosts, int ng, const double* wx, const double* wy,
                            const double* wz, const double* Dg, const T* rhs, T* e, int maxit, double tol,
                            int* iters, WarpBottomSmem& W, int cg) {
  const int lane = threadIdx.x;
  const int64_t base = Dd.bot_base;
  for (int i = lane; i < nc; i += 32) {
    const BotCell C = cells[i];
    const int64_t q = C.q;
    W.q[i] = (int)(q - base);
    W.sx[i] = C.sx;
    W.sy[i] = (int)C.sy;
    W.D[i] = Dg[q];
    W.wxm[i] = wx[q];
    W.wxp[i] = wx[q + 1];
    W.wym[i] = wy[q];
    W.wyp[i] = wy[q + C.sx];
    W.wzm[i] = wz[q];
    W.wzp[i] = wz[q + C.sy];
    W.r[i] = (double)tld(rhs + q);
    W.p[W.q[i]] = 0.0;
    W.v[i] = 0.0;
    W.x[i] = 0.0;
  }
  __syncwarp();
  auto apply = [&](double* in, double* out) {  // out[slot] = (A in)[cell]
    __syncwarp();
    for (int g = lane; g < ng; g += 32) {
      const BotGhost G = ghosts[g];
      in[G.dst - base] = G.sign * in[G.src - base];
    }
    __syncwarp();
    for (int i = lane; i < nc; i += 32) {
      const int q = W.q[i], sx = W.sx[i], sy = W.sy[i];
      double w = W.D[i] * in[q];
      w = fma(-W.wxm[i], in[q - 1], w);
      w = fma(-W.wxp[i], in[q + 1], w);
      w = fma(-W.wym[i], in[q - sx], w);
      w = fma(-W.wyp[i], in[q + sx], w);
      w = fma(-W.wzm[i], in[q - sy], w);
      w = fma(-W.wzp[i], in[q + sy], w);
      out[i] = w;
    }
  };
  const int span = nc >= 32 ? 32 : (nc > 16 ? 32 : nc > 8 ? 16 : nc > 4 ? 8 : nc > 2 ? 4 : nc > 1 ? 2 : 1);
  auto dot = [&](const double* a, const double* b) {
    double acc = 0.0;
    for (int i = lane; i < nc; i += 32) acc += a[i] * b[i];
    return wsum(acc, span);
  };
  auto norm = [&](const double* a) {
    double acc = 0.0;
    for (int i = lane; i < nc; i += 32) acc = fmax(acc, fabs(a[i]));
    return wmax(acc, span);
  };
  if (Dd.singular) {
    double acc = 0.0;
    for (int i = lane; i < nc; i += 32) acc += W.r[i];
    const double mean = wsum(acc, span) / (double)nc;
    for (int i = lane; i < nc; i += 32) W.r[i] -= mean;
  }
  for (int i = lane; i < nc; i += 32) W.rh[i] = W.r[i];
  const double r0 = norm(W.r);
  double rho_old = 1.0, alpha = 1.0, omega = 1.0;
  int it = 0;
  // s-values of the cells (slot order) live in W.s at the cells' element offsets
  auto sval = [&](int i) -> double& { return W.s[W.q[i]]; };
  auto pval = [&](int i) -> double& { return W.p[W.q[i]]; };
  if (cg && r0 > 0.0) {
    // conjugate gradients (the steps of the block version): v = A p in W.v
    __syncwarp();
    for (int i = lane; i < nc; i += 32) pval(i) = W.r[i];
    double rho = dot(W.r, W.r);
    for (it = 1; it <= maxit; ++it) {
      apply(W.p, W.v);
      __syncwarp();
      double pv = 0.0;
      for (int i = lane; i < nc; i += 32) pv += pval(i) * W.v[i];
      pv = wsum(pv, span);
      if (!(pv > 0.0)) { --it; break; }
      const double al = rho / pv;
      for (int i = lane; i < nc; i += 32) {
        W.x[i] += al * pval(i);
        W.r[i] -= al * W.v[i];
      }
      if (norm(W.r) <= tol * r0) break;
      const double rho_new = dot(W.r, W.r);
      const double be = rho_new / rho;
      rho = rho_new;
      __syncwarp();
      for (int i = lane; i < nc; i += 32) pval(i) = W.r[i] + be * pval(i);
    }
    if (it > maxit) it = maxit;
  } else if (r0 > 0.0) {
    // (rho of the next iteration is taken with the residual's norm, from the same r)
    double rho = dot(W.rh, W.r);
    for (it = 1; it <= maxit; ++it) {
      if (fabs(rho) < 1e-300) { --it; break; }
      const double beta = (rho / rho_old) * (alpha / omega);
      __syncwarp();
      for (int i = lane; i < nc; i += 32) pval(i) = W.r[i] + beta * (pval(i) - omega * W.v[i]);
      apply(W.p, W.v);
      const double rv = dot(W.rh, W.v);
      if (fabs(rv) < 1e-300) { --it; break; }
      alpha = rho / rv;
      __syncwarp();
      for (int i = lane; i < nc; i += 32) sval(i) = W.r[i] - alpha * W.v[i];
      double ns = 0.0;
      for (int i = lane; i < nc; i += 32) ns = fmax(ns, fabs(sval(i)));
      if (wmax(ns, span) <= tol * r0) {
        for (int i = lane; i < nc; i += 32) W.x[i] += alpha * pval(i);
        break;
      }
      apply(W.s, W.t);
      double tt = 0.0, ts = 0.0;
      for (int i = lane; i < nc; i += 32) {
        tt += W.t[i] * W.t[i];
        ts += W.t[i] * sval(i);
      }
      wsum2(tt, ts, span);
      if (tt == 0.0) {
        for (int i = lane; i < nc; i += 32) W.x[i] += alpha * pval(i);
        break;
      }
      omega = ts / tt;
      double rn = 0.0, nr = 0.0;
      for (int i = lane; i < nc; i += 32) {
        W.x[i] += alpha * pval(i) + omega * sval(i);
        W.r[i] = sval(i) - omega * W.t[i];
        rn += W.rh[i] * W.r[i];
        nr = fmax(nr, fabs(W.r[i]));
      }
      wsum_max(rn, nr, span);
      if (nr <= tol * r0) break;
      rho_old = rho;
      rho = rn;
    }
    if (it > maxit) it = maxit;
  }
  double shift = 0.0;
  if (Dd.singular) {
    double acc = 0.0;
    for (int i = lane; i < nc; i += 32) acc += W.x[i];
    shift = wsum(acc, span) / (double)nc;
  }
  for (int i = lane; i < nc; i += 32) tst_d(e + (base + W.q[i]), W.x[i] - shift);
  if (lane == 0 && iters) *iters = it;
}

// every level's buffers in the V-cycle's element type
template <class T>
struct TailPtrs {
  T* e[TAIL_MAXLEV];
  T* r[TAIL_MAXLEV];
  const typename Cf<T>::type* wx[TAIL_MAXLEV];
  const typename Cf<T>::type* wy[TAIL_MAXLEV];
  const typename Cf<T>::type* wz[TAIL_MAXLEV];
  const typename Cf<T>::type* D[TAIL_MAXLEV];
  const typename Cf<T>::type* invD[TAIL_MAXLEV];
};

// The bottom of one problem's coarse end: BiCGStab (van der Vorst 1992) or conjugate
// gradients in FP64 on its bottom level from x0 = 0, reading the bottom's right-hand side
// from P.r[mb] and writing the correction to P.e[mb] (global memory); every thread of the
// block calls it.
template <class T>
__device__ void tail_bottom(const TailArgs& a, const TailPtrs<T>& P, const TailDesc& Dd, double* sh,
                            WarpBottomSmem& wb) {
  const TailLevel Lb = a.levels[Dd.lev0 + Dd.mb - Dd.m0];
  if (Lb.ncell[0] + Lb.ncell[1] <= TAIL_WARP_CELLS && Dd.bot_span <= TAIL_WARP_SPAN) {
    const int m = Dd.mb;
    if (threadIdx.x < 32)
      warp_bottom(Dd, a.cells + Lb.cell0, Lb.ncell[0] + Lb.ncell[1], a.ghosts + Lb.ghost0,
                  Lb.nghost[0] + Lb.nghost[1], a.wx64[m], a.wy64[m], a.wz64[m], a.D64[m], P.r[m], P.e[m], a.maxit,
                  a.tol, a.iters ? a.iters + Dd.solve : nullptr, wb, a.cg);
    __syncthreads();
  } else {
    const int m = Dd.mb;
    const TailLevel L = a.levels[Dd.lev0 + m - Dd.m0];
    const BotCell* cells = a.cells + L.cell0;
    const int nc = L.ncell[0] + L.ncell[1];
    const BotGhost* ghosts = a.ghosts + L.ghost0;
    const int ng = L.nghost[0] + L.nghost[1];
    const double *wx = a.wx64[m], *wy = a.wy64[m], *wz = a.wz64[m], *D = a.D64[m];
    const int64_t ne = a.nelem[m];
    double* r = a.work[m];
    double* rh = r + ne;
    double* p = r + 2 * ne;
    double* v = r + 3 * ne;
    double* s = r + 4 * ne;
    double* t = r + 5 * ne;
    double* x = r + 6 * ne;
    const T* rhs = P.r[m];
    auto apply = [&](double* in, double* out) {
      for (int g = threadIdx.x; g < ng; g += TT) {
        const BotGhost G = ghosts[g];
        in[G.dst] = G.sign * in[G.src];
      }
      __syncthreads();
      for (int i = threadIdx.x; i < nc; i += TT) {
        const BotCell C = cells[i];
        const int64_t q = C.q, sx = C.sx, sy = C.sy;
        double w = D[q] * in[q];
        w = fma(-wx[q], in[q - 1], w);
        w = fma(-wx[q + 1], in[q + 1], w);
        w = fma(-wy[q], in[q - sx], w);
        w = fma(-wy[q + sx], in[q + sx], w);
        w = fma(-wz[q], in[q - sy], w);
        w = fma(-wz[q + sy], in[q + sy], w);
        out[q] = w;
      }
      __syncthreads();
    };
    auto dot = [&](const double* y, const double* z) {
      double acc = 0.0;
      for (int i = threadIdx.x; i < nc; i += TT) acc += y[cells[i].q] * z[cells[i].q];
      return tsum(acc, sh);
    };
    auto norm = [&](const double* y) {
      double acc = 0.0;
      for (int i = threadIdx.x; i < nc; i += TT) acc = fmax(acc, fabs(y[cells[i].q]));
      return tmax(acc, sh);
    };
    auto sum = [&](const double* y) {
      double acc = 0.0;
      for (int i = threadIdx.x; i < nc; i += TT) acc += y[cells[i].q];
      return tsum(acc, sh);
    };
    for (int i = threadIdx.x; i < nc; i += TT) {
      const int64_t q = cells[i].q;
      r[q] = (double)tld(rhs + q);
      p[q] = 0.0;
      v[q] = 0.0;
      x[q] = 0.0;
    }
    __syncthreads();
    if (Dd.singular) {
      const double mean = sum(r) / (double)nc;
      for (int i = threadIdx.x; i < nc; i += TT) r[cells[i].q] -= mean;
      __syncthreads();
    }
    for (int i = threadIdx.x; i < nc; i += TT) rh[cells[i].q] = r[cells[i].q];
    __syncthreads();
    const double r0 = norm(r);
    double rho_old = 1.0, alpha = 1.0, omega = 1.0;
    int it = 0;
    if (a.cg && r0 > 0.0) {  // conjugate gradients, v = A p
      for (int i = threadIdx.x; i < nc; i += TT) p[cells[i].q] = r[cells[i].q];
      __syncthreads();
      double rho = dot(r, r);
      for (it = 1; it <= a.maxit; ++it) {
        apply(p, v);
        const double pv = dot(p, v);
        if (!(pv > 0.0)) { --it; break; }
        const double al = rho / pv;
        for (int i = threadIdx.x; i < nc; i += TT) {
          const int64_t q = cells[i].q;
          x[q] += al * p[q];
          r[q] -= al * v[q];
        }
        __syncthreads();
        if (norm(r) <= a.tol * r0) break;
        const double rho_new = dot(r, r);
        const double be = rho_new / rho;
        rho = rho_new;
        for (int i = threadIdx.x; i < nc; i += TT) {
          const int64_t q = cells[i].q;
          p[q] = r[q] + be * p[q];
        }
        __syncthreads();
      }
      if (it > a.maxit) it = a.maxit;
    } else if (r0 > 0.0) {
      for (it = 1; it <= a.maxit; ++it) {
        const double rho = dot(rh, r);
        if (fabs(rho) < 1e-300) { --it; break; }
        const double beta = (rho / rho_old) * (alpha / omega);
        for (int i = threadIdx.x; i < nc; i += TT) {
          const int64_t q = cells[i].q;
          p[q] = r[q] + beta * (p[q] - omega * v[q]);
        }
        __syncthreads();
        apply(p, v);
        const double rv = dot(rh, v);
        if (fabs(rv) < 1e-300) { --it; break; }
        alpha = rho / rv;
        for (int i = threadIdx.x; i < nc; i += TT) {
          const int64_t q = cells[i].q;
          s[q] = r[q] - alpha * v[q];
        }
        __syncthreads();
        if (norm(s) <= a.tol * r0) {
          for (int i = threadIdx.x; i < nc; i += TT) x[cells[i].q] += alpha * p[cells[i].q];
          __syncthreads();
          break;
        }
        apply(s, t);
        const double tt = dot(t, t);
        if (tt == 0.0) {
          for (int i = threadIdx.x; i < nc; i += TT) x[cells[i].q] += alpha * p[cells[i].q];
          __syncthreads();
          break;
        }
        omega = dot(t, s) / tt;
        for (int i = threadIdx.x; i < nc; i += TT) {
          const int64_t q = cells[i].q;
          x[q] += alpha * p[q] + omega * s[q];
          r[q] = s[q] - omega * t[q];
        }
        __syncthreads();
        if (norm(r) <= a.tol * r0) break;
        rho_old = rho;
      }
      if (it > a.maxit) it = a.maxit;
    }
    double shift = 0.0;
    if (Dd.singular) shift = sum(x) / (double)nc;
    T* e = P.e[m];
    for (int i = threadIdx.x; i < nc; i += TT) {
      const int64_t q = cells[i].q;
      tst_d(e + q, x[q] - shift);
    }
    if (threadIdx.x == 0 && a.iters) a.iters[Dd.solve] = it;
    __syncthreads();
  }
}

template <class T>
__global__ void __launch_bounds__(TT, 1) k_vtail(const __grid_constant__ TailArgs a, const __grid_constant__ TailPtrs<T> P) {
  using A = typename Ar<T>::type;
  // programmatic dependent launch: wait for the predecessor before any global access
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  __shared__ double sh[TT / 32 + 1];
  const TailDesc Dd = a.descs[blockIdx.x];
  if (a.active && !a.active[Dd.solve]) return;
  // ---- down: pre-smooth, restrict the residual
  for (int m = Dd.m0; m < Dd.mb; ++m) {
    const TailLevel L = a.levels[Dd.lev0 + m - Dd.m0];
    T* e = P.e[m];
    const T* r = P.r[m];
    for (int i = threadIdx.x; i < L.ncell[0] + L.ncell[1]; i += TT) tst(e + a.cells[L.cell0 + i].q, (A)0);
    __syncthreads();
    for (int it = 0; it < a.nu1; ++it)
      for (int colour = 0; colour < 2; ++colour) {
        t_fill(L, a.ghosts, e, 1 - colour);
        __syncthreads();
        t_smooth(L, a.cells, e, r, P.wx[m], P.wy[m], P.wz[m], P.invD[m], colour);
        __syncthreads();
      }
    t_fill(L, a.ghosts, e, -1);
    __syncthreads();
    T* rc = P.r[m + 1];
    for (int i = threadIdx.x; i < L.nxfer; i += TT) {
      const TailXfer X = a.xfer[L.xfer0 + i];
      A s = 0;
      for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj) {
          const int64_t q = X.qf + (int64_t)dj * X.sx + (int64_t)dk * X.sy;
          s += t_resid(e, r, P.wx[m], P.wy[m], P.wz[m], P.D[m], q, X.sx, X.sy);
          s += t_resid(e, r, P.wx[m], P.wy[m], P.wz[m], P.D[m], q + 1, X.sx, X.sy);
        }
      tst(rc + X.qc, s * (A)0.125);
    }
    __syncthreads();
  }
  // ---- bottom
  __shared__ WarpBottomSmem wb;
  tail_bottom(a, P, Dd, sh, wb);
  // ---- up: interpolate, post-smooth
  for (int m = Dd.mb - 1; m >= Dd.m0; --m) {
    const TailLevel L = a.levels[Dd.lev0 + m - Dd.m0];
    T* e = P.e[m];
    const T* r = P.r[m];
    const T* ec = P.e[m + 1];
    for (int i = threadIdx.x; i < L.nxfer; i += TT) {
      const TailXfer X = a.xfer[L.xfer0 + i];
      const A c = tld(ec + X.qc);
      for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj) {
          const int64_t q = X.qf + (int64_t)dj * X.sx + (int64_t)dk * X.sy;
          tst(e + q, (A)tld(e + q) + c);
          tst(e + q + 1, (A)tld(e + q + 1) + c);
        }
    }
    __syncthreads();
    for (int it = 0; it < a.nu2; ++it)
      for (int cc = 0; cc < 2; ++cc) {
        const int colour = a.post_rev ? 1 - cc : cc;
        t_fill(L, a.ghosts, e, 1 - colour);
        __syncthreads();
        t_smooth(L, a.cells, e, r, P.wx[m], P.wy[m], P.wz[m], P.invD[m], colour);
        __syncthreads();
      }
  }
  // the first level's ghosts current on exit (the interpolation from it may read them)
  t_fill(a.levels[Dd.lev0], a.ghosts, P.e[Dd.m0], -1);
}

// ---------------------------------------------------------------- dense coarse end
// The same V-cycle steps with every tail level held in shared memory: each level of the
// problem as one padded array over its domain (the boxes of a problem tile it, so a ghost
// between two boxes is the neighbouring cell itself and only the ghosts outside the domain
// are filled), loaded once at the start -- coefficients of the smoothed levels and the
// right-hand side of the first -- so that every later step reads on-chip memory.  Per cell
// the arithmetic is that of k_vtail in the same order (the face weights a box stores for
// its high faces are those its neighbour stores for the same faces), and the bottom solve is
// k_vtail's: its right-hand side goes out to global memory and its correction comes back.

// one level's arrays in the dense layout
template <class T>
struct DenseLev {
  T* e;
  T* r;
  typename Cf<T>::type *wx, *wy, *wz, *invD, *D;
};

template <class T>
__device__ DenseLev<T> dense_lev(unsigned char* base, const TailArgs& a, const TailDesc& Dd, int m) {
  using CF = typename Cf<T>::type;
  int64_t off = 0;
  for (int q = Dd.m0; q < m; ++q)
    off += tail_level_bytes(a.levels[Dd.lev0 + q - Dd.m0].dne, (int)sizeof(T), (int)sizeof(CF), q < Dd.mb);
  const int ne = a.levels[Dd.lev0 + m - Dd.m0].dne;
  const int64_t eb = ((int64_t)ne * sizeof(T) + 15) & ~(int64_t)15;
  const int64_t cb = ((int64_t)ne * sizeof(CF) + 15) & ~(int64_t)15;
  DenseLev<T> d;
  d.e = (T*)(base + off);
  d.r = (T*)(base + off + eb);
  CF* w = (CF*)(base + off + 2 * eb);
  d.wx = w;
  d.wy = (CF*)((unsigned char*)w + cb);
  d.wz = (CF*)((unsigned char*)w + 2 * cb);
  d.invD = (CF*)((unsigned char*)w + 3 * cb);
  d.D = (CF*)((unsigned char*)w + 4 * cb);
  return d;
}

// the work item of thread t in a loop over a level's cells: items 4l + w (warp w < 4, lane
// l) first, so that a short list spreads over the four warp schedulers (the FP64 pipe of
// each is narrow); a bijection on [0, TT)
__device__ __forceinline__ int spread(int t) { return ((t >> 5) & 3) + 4 * (t & 31) + 128 * (t >> 7); }

__device__ __forceinline__ double neg(double v) { return -v; }
__device__ __forceinline__ float neg(float v) { return -v; }
__device__ __forceinline__ bf16 neg(bf16 v) { return __hneg(v); }
__device__ __forceinline__ double to_t(double v, const double*) { return v; }
__device__ __forceinline__ float to_t(float v, const float*) { return v; }
__device__ __forceinline__ bf16 to_t(float v, const bf16*) { return __float2bfloat16_rn(v); }

// The value v just stored at slot q also goes into the ghosts outside the domain that copy
// it (fl: the cell's TAIL_LO_* / TAIL_HI_* flags): the wall ghost beside it (+/- v), or the
// periodic image past the other end -- what a fill from the cell gives them.
template <class T>
__device__ __forceinline__ void d_push(T* e, int q, int fl, const TailLevel& L, T v) {
  if (!(fl & (TAIL_LO_X | TAIL_LO_Y | TAIL_LO_Z | TAIL_HI_X | TAIL_HI_Y | TAIL_HI_Z))) return;
  const int st[3] = {1, L.dsx, L.dsy};
  const int n[3] = {L.dsx - 2, L.dsy / L.dsx - 2, L.dne / L.dsy - 2};
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    if (fl & (TAIL_LO_X << a)) {
      const int f = L.face[2 * a];
      if (f == 2) e[q + n[a] * st[a]] = v;
      else if (f != 0) e[q - st[a]] = f < 0 ? neg(v) : v;
    }
    if (fl & (TAIL_HI_X << a)) {
      const int f = L.face[2 * a + 1];
      if (f == 2) e[q - n[a] * st[a]] = v;
      else if (f != 0) e[q + st[a]] = f < 0 ? neg(v) : v;
    }
  }
}

// one colour of a level in the dense layout (gs_cell's arithmetic), pushing boundary values
template <class T>
__device__ void d_smooth(const TailLevel& L, const BotCell* __restrict__ cells, const DenseLev<T>& d, int colour) {
  using A = typename Ar<T>::type;
  const int c0 = L.cell0 + (colour ? L.ncell[0] : 0);
  const int nc = colour ? L.ncell[1] : L.ncell[0];
  const int sx = L.dsx, sy = L.dsy;
  for (int i = spread(threadIdx.x); i < nc; i += TT) {
    const int fl = cells[c0 + i].pad;
    const int q = fl & TAIL_SLOT_MASK;
    A s = tld(d.r + q);
    s = fma((A)d.wx[q], (A)tld(d.e + q - 1), s);
    s = fma((A)d.wx[q + 1], (A)tld(d.e + q + 1), s);
    s = fma((A)d.wy[q], (A)tld(d.e + q - sx), s);
    s = fma((A)d.wy[q + sx], (A)tld(d.e + q + sx), s);
    s = fma((A)d.wz[q], (A)tld(d.e + q - sy), s);
    s = fma((A)d.wz[q + sy], (A)tld(d.e + q + sy), s);
    const T v = to_t(s * (A)d.invD[q], d.e);
    d.e[q] = v;
    d_push(d.e, q, fl, L, v);
  }
}

template <class T>
__global__ void __launch_bounds__(TT, 1) k_vtail_dense(const __grid_constant__ TailArgs a,
                                                      const __grid_constant__ TailPtrs<T> P) {
  using A = typename Ar<T>::type;
  extern __shared__ __align__(16) unsigned char tail_smem[];
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  __shared__ double sh[TT / 32 + 1];
  __shared__ WarpBottomSmem wb;
  const TailDesc Dd = a.descs[blockIdx.x];
  if (a.active && !a.active[Dd.solve]) return;
  // ---- load: zero every level's e; coefficients of the smoothed levels, r of the first
  for (int m = Dd.m0; m <= Dd.mb; ++m) {
    const TailLevel L = a.levels[Dd.lev0 + m - Dd.m0];
    const DenseLev<T> d = dense_lev<T>(tail_smem, a, Dd, m);
    for (int i = threadIdx.x; i < L.dne; i += TT) tst(d.e + i, (A)0);
    if (m == Dd.mb) break;
    const int nc = L.ncell[0] + L.ncell[1];
    for (int i = threadIdx.x; i < nc; i += TT) {
      const BotCell C = a.cells[L.cell0 + i];
      const int q = C.pad & TAIL_SLOT_MASK;
      d.wx[q] = P.wx[m][C.q];
      d.wy[q] = P.wy[m][C.q];
      d.wz[q] = P.wz[m][C.q];
      d.invD[q] = P.invD[m][C.q];
      d.D[q] = P.D[m][C.q];
      if (C.pad & TAIL_HI_X) d.wx[q + 1] = P.wx[m][C.q + 1];
      if (C.pad & TAIL_HI_Y) d.wy[q + L.dsx] = P.wy[m][C.q + C.sx];
      if (C.pad & TAIL_HI_Z) d.wz[q + L.dsy] = P.wz[m][C.q + C.sy];
      if (m == Dd.m0) d.r[q] = P.r[m][C.q];
    }
  }
  __syncthreads();
  // the ghosts outside the domain as a fill from the zero correction gives them (+/- 0)
  for (int m = Dd.m0; m < Dd.mb; ++m) {
    const TailLevel L = a.levels[Dd.lev0 + m - Dd.m0];
    T* e = dense_lev<T>(tail_smem, a, Dd, m).e;
    for (int i = threadIdx.x; i < L.ndghost[0] + L.ndghost[1]; i += TT) {
      const BotGhost G = a.dghosts[L.dghost0 + i];
      tst(e + G.dst, G.sign < 0 ? -(A)0 : (A)0);
    }
  }
  __syncthreads();
  // ---- down: pre-smooth, restrict the residual
  for (int m = Dd.m0; m < Dd.mb; ++m) {
    const TailLevel L = a.levels[Dd.lev0 + m - Dd.m0];
    const DenseLev<T> d = dense_lev<T>(tail_smem, a, Dd, m);
    // (the ghosts are current: every value written went into them too)
    for (int it = 0; it < a.nu1; ++it)
      for (int colour = 0; colour < 2; ++colour) {
        d_smooth(L, a.cells, d, colour);
        __syncthreads();
      }
    T* rc = dense_lev<T>(tail_smem, a, Dd, m + 1).r;
    const int64_t sx = L.dsx, sy = L.dsy;
    // eight lanes per coarse cell, one child each (child k = 4 dk + 2 dj + di); the first
    // lane of the eight adds their residuals in k order, as one thread adding them would
    const int nitem = 8 * L.nxfer;
    for (int i0 = 0; i0 < nitem; i0 += TT) {
      const int i = i0 + threadIdx.x;
      const int k = i & 7;
      A v = 0;
      int qc = 0;
      if (i < nitem) {
        const TailXfer X = a.xfer[L.xfer0 + (i >> 3)];
        const int64_t q = X.dqf + (k & 1) + ((k >> 1) & 1) * sx + (k >> 2) * sy;
        v = t_resid(d.e, d.r, d.wx, d.wy, d.wz, d.D, q, sx, sy);
        qc = X.dqc;
      }
      const int g = (threadIdx.x & 31) & ~7;
      A s = 0;
#pragma unroll
      for (int u = 0; u < 8; ++u) s += __shfl_sync(0xffffffffu, v, g + u);
      if (i < nitem && k == 0) tst(rc + qc, s * (A)0.125);
    }
    __syncthreads();
  }
  // ---- bottom: its right-hand side out to global memory, the solve, its correction back
  {
    const TailLevel Lb = a.levels[Dd.lev0 + Dd.mb - Dd.m0];
    const DenseLev<T> d = dense_lev<T>(tail_smem, a, Dd, Dd.mb);
    const int nc = Lb.ncell[0] + Lb.ncell[1];
    T* rb = P.r[Dd.mb];
    if (Dd.mb > Dd.m0)  // (a tail that is only its bottom level reads its rhs in place)
      for (int i = threadIdx.x; i < nc; i += TT) {
        const BotCell C = a.cells[Lb.cell0 + i];
        rb[C.q] = d.r[C.pad & TAIL_SLOT_MASK];
      }
    __syncthreads();
    tail_bottom(a, P, Dd, sh, wb);
    const T* eb = P.e[Dd.mb];
    for (int i = threadIdx.x; i < nc; i += TT) {
      const BotCell C = a.cells[Lb.cell0 + i];
      d.e[C.pad & TAIL_SLOT_MASK] = eb[C.q];
    }
    __syncthreads();
  }
  // ---- up: interpolate, post-smooth
  for (int m = Dd.mb - 1; m >= Dd.m0; --m) {
    const TailLevel L = a.levels[Dd.lev0 + m - Dd.m0];
    const DenseLev<T> d = dense_lev<T>(tail_smem, a, Dd, m);
    const T* ec = dense_lev<T>(tail_smem, a, Dd, m + 1).e;
    const int sx = L.dsx, sy = L.dsy;
    // one thread per fine cell (child k = 4 dk + 2 dj + di of coarse cell i >> 3)
    for (int i = threadIdx.x; i < 8 * L.nxfer; i += TT) {
      const TailXfer X = a.xfer[L.xfer0 + (i >> 3)];
      const int di = i & 1, dj = (i >> 1) & 1, dk = (i >> 2) & 1;
      const int q = X.dqf + di + dj * sx + dk * sy;
      const int fl = (X.dfl & (di ? TAIL_HI_X : TAIL_LO_X)) | (X.dfl & (dj ? TAIL_HI_Y : TAIL_LO_Y)) |
                     (X.dfl & (dk ? TAIL_HI_Z : TAIL_LO_Z));
      const T v = to_t((A)tld(d.e + q) + (A)tld(ec + X.dqc), d.e);
      d.e[q] = v;
      d_push(d.e, q, fl, L, v);
    }
    __syncthreads();
    for (int it = 0; it < a.nu2; ++it)
      for (int cc = 0; cc < 2; ++cc) {
        const int colour = a.post_rev ? 1 - cc : cc;
        d_smooth(L, a.cells, d, colour);
        __syncthreads();
      }
  }
  // ---- the first level's correction back to global memory (valid cells)
  {
    const TailLevel L = a.levels[0 + Dd.lev0];
    const DenseLev<T> d = dense_lev<T>(tail_smem, a, Dd, Dd.m0);
    T* e0 = P.e[Dd.m0];
    for (int i = threadIdx.x; i < L.ncell[0] + L.ncell[1]; i += TT) {
      const BotCell C = a.cells[L.cell0 + i];
      e0[C.q] = d.e[C.pad & TAIL_SLOT_MASK];
    }
    // and its ghosts (the box layout's), current on exit as k_vtail leaves them
    __syncthreads();
    t_fill(L, a.ghosts, e0, -1);
  }
}

template <class T>
void fill_ptrs(TailPtrs<T>& P, const TailLevelBufs* lv, int n) {
  for (int m = 0; m < TAIL_MAXLEV; ++m) {
    const bool ok = m < n;
    P.e[m] = ok ? (T*)lv[m].e : nullptr;
    P.r[m] = ok ? (T*)lv[m].r : nullptr;
    P.wx[m] = ok ? (const typename Cf<T>::type*)lv[m].wx : nullptr;
    P.wy[m] = ok ? (const typename Cf<T>::type*)lv[m].wy : nullptr;
    P.wz[m] = ok ? (const typename Cf<T>::type*)lv[m].wz : nullptr;
    P.D[m] = ok ? (const typename Cf<T>::type*)lv[m].D : nullptr;
    P.invD[m] = ok ? (const typename Cf<T>::type*)lv[m].invD : nullptr;
  }
}

}  // namespace

template <class T>
static void launch_tail_kernel(int nblocks, const TailArgs& a, const TailPtrs<T>& P, int dense_bytes,
                               cudaStream_t s) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(nblocks);
  cfg.blockDim = dim3(TT);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = pdl_enabled() ? 1 : 0;
  if (dense_bytes > 0) {
    // (the opt-in above 48 KB belongs to the current device: set before every launch)
    cudaFuncSetAttribute(k_vtail_dense<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, TAIL_SMEM_MAX);
    cfg.dynamicSmemBytes = (size_t)dense_bytes;
    cudaLaunchKernelEx(&cfg, k_vtail_dense<T>, a, P);
  } else {
    cudaLaunchKernelEx(&cfg, k_vtail<T>, a, P);
  }
}

void launch_vtail(int dt, int nblocks, const TailArgs& a, const TailLevelBufs* lv, int nlev, int dense_bytes,
                  cudaStream_t s) {
  if (nblocks <= 0) return;
  count_launches(1);
  switch (dt) {
    case DT_F64: {
      TailPtrs<double> P;
      fill_ptrs(P, lv, nlev);
      launch_tail_kernel(nblocks, a, P, dense_bytes, s);
      break;
    }
    case DT_F32: {
      TailPtrs<float> P;
      fill_ptrs(P, lv, nlev);
      launch_tail_kernel(nblocks, a, P, dense_bytes, s);
      break;
    }
    default: {
      TailPtrs<bf16> P;
      fill_ptrs(P, lv, nlev);
      launch_tail_kernel(nblocks, a, P, dense_bytes, s);
      break;
    }
  }
}

}  // namespace gmg
