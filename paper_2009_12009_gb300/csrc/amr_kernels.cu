// amr_kernels.cu -- kernels of the two-level composite operator (FP64).
//
// Sec. "Operations between levels": fine ghost cells on the coarse/fine boundary are
// interpolated from coarse data, coarse cells next to the fine level take the averaged
// fine fluxes (refluxing), covered coarse cells hold the average of the fine data.
//   fine ghost  phi_g = 8/15 phi_c* + 2/3 phi_f1 - 1/5 phi_f2,  phi_c* = sum_e cw_e phi_c[cq_e]
//   reflux      row of an uncovered coarse cell I with a face shared with a covered cell N:
//               the term w (phi_I - phi_N) of the coarse stencil is replaced by
//               sum over the 4 fine faces of cf (phi_g - phi_f),  cf = w_f * h_f / (4 h_c).
// The transpose of the composite operator is the (symmetric) level stencils plus the
// transpose of these two couplings, scattered with atomics over the interface only.
#include <algorithm>

#include "amr.h"

namespace gmg {
namespace {

constexpr int AT = 256;

__global__ void __launch_bounds__(AT) k_cf_fill(const CfGhost* __restrict__ g, int n, double* f,
                                                const double* __restrict__ c, int mode) {
  const int i = blockIdx.x * AT + threadIdx.x;
  if (i >= n) return;
  const CfGhost G = g[i];
  double v;
  if (mode == CF_COPY) {
    v = f[G.f1];
  } else if (mode == CF_ZERO) {
    v = 0.0;
  } else {
    double cs = 0.0;
    if (c)
      for (int e = 0; e < 5; ++e) cs += G.cw[e] * c[G.cq[e]];
    v = (8.0 / 15.0) * cs + (2.0 / 3.0) * f[G.f1] - 0.2 * f[G.f2];
  }
  f[G.dst] = v;
}

// out[I] = in[I] + std * w (c[I] - c[N]) - sum_4 cf (f[g] - f[f])   (one thread per coarse
// cell that has coarse/fine faces; its faces are processed in order: deterministic)
__global__ void __launch_bounds__(AT) k_reflux(const RefluxCell* __restrict__ cells, int n,
                                               const RefluxFace* __restrict__ faces, const double* __restrict__ wc0,
                                               const double* __restrict__ wc1, const double* __restrict__ wc2,
                                               const double* __restrict__ wf0, const double* __restrict__ wf1,
                                               const double* __restrict__ wf2, const double* __restrict__ c,
                                               const double* __restrict__ f, const double* in, double* out, int std_part,
                                               double ratio_h) {
  const int i = blockIdx.x * AT + threadIdx.x;
  if (i >= n) return;
  const RefluxCell R = cells[i];
  const double* wc[3] = {wc0, wc1, wc2};
  const double* wf[3] = {wf0, wf1, wf2};
  double v = in ? in[R.I] : 0.0;
  for (int k = 0; k < R.nface; ++k) {
    const RefluxFace F = faces[R.face0 + k];
    if (std_part) v += wc[F.d][F.cslot] * (c[R.I] - c[F.N]);
    for (int q = 0; q < 4; ++q) {
      const double cf = 0.25 * wf[F.d][F.fslot[q]] * ratio_h;
      v -= cf * (f[F.g[q]] - f[F.f[q]]);
    }
  }
  out[R.I] = v;
}

__global__ void __launch_bounds__(AT) k_zero_list(const int64_t* __restrict__ idx, int n, double* x) {
  const int i = blockIdx.x * AT + threadIdx.x;
  if (i < n) x[idx[i]] = 0.0;
}

// transpose of the fine rows' ghost coupling: row f1 holds -w_g phi_g
__global__ void __launch_bounds__(AT) k_cf_transpose(const CfGhost* __restrict__ g, int n,
                                                     const double* __restrict__ wf0, const double* __restrict__ wf1,
                                                     const double* __restrict__ wf2, const double* __restrict__ yf,
                                                     double* outc, double* outf) {
  const int i = blockIdx.x * AT + threadIdx.x;
  if (i >= n) return;
  const CfGhost G = g[i];
  const double* wf[3] = {wf0, wf1, wf2};
  const double s = -wf[G.d][G.fslot] * yf[G.f1];
  for (int e = 0; e < 5; ++e) atomicAdd(outc + G.cq[e], s * (8.0 / 15.0) * G.cw[e]);
  atomicAdd(outf + G.f1, s * (2.0 / 3.0));
  atomicAdd(outf + G.f2, s * (-0.2));
}

// transpose of the reflux rows: row I holds -w (phi_I - phi_N) + sum_4 cf (phi_g - phi_f)
__global__ void __launch_bounds__(AT) k_reflux_transpose(const RefluxCell* __restrict__ cells, int n,
                                                         const RefluxFace* __restrict__ faces,
                                                         const CfGhost* __restrict__ cfg,
                                                         const double* __restrict__ wc0, const double* __restrict__ wc1,
                                                         const double* __restrict__ wc2,
                                                         const double* __restrict__ wf0, const double* __restrict__ wf1,
                                                         const double* __restrict__ wf2, const double* __restrict__ yc,
                                                         double* outc, double* outf, double ratio_h) {
  const int i = blockIdx.x * AT + threadIdx.x;
  if (i >= n) return;
  const RefluxCell R = cells[i];
  const double* wc[3] = {wc0, wc1, wc2};
  const double* wf[3] = {wf0, wf1, wf2};
  const double y = yc[R.I];
  for (int k = 0; k < R.nface; ++k) {
    const RefluxFace F = faces[R.face0 + k];
    const double w = wc[F.d][F.cslot];
    atomicAdd(outc + R.I, -w * y);
    atomicAdd(outc + F.N, w * y);  // a covered column: cleared by the caller
    for (int q = 0; q < 4; ++q) {
      const double cf = 0.25 * wf[F.d][F.fslot[q]] * ratio_h;
      atomicAdd(outf + F.f[q], -cf * y);
      const CfGhost G = cfg[F.cf[q]];
      for (int e = 0; e < 5; ++e) atomicAdd(outc + G.cq[e], cf * y * (8.0 / 15.0) * G.cw[e]);
      atomicAdd(outf + G.f1, cf * y * (2.0 / 3.0));
      atomicAdd(outf + G.f2, cf * y * (-0.2));
    }
  }
}

__device__ __forceinline__ int64_t ax_stride(const DevBox& B, int d) {
  return d == 0 ? 1 : (d == 1 ? (int64_t)B.sx : B.sy);
}

// dL/dbeta at the cells of one level (coarse: uncovered cells only) from
// dL/dbeta_face = -lambda^T (dA/dbeta_face) phi, through the face rule that made the face
// beta (harmonic mean of two cells of the level; the one adjacent cell at a wall or at a
// coarse/fine face).  Ghosts of phi, lambda and beta must be filled; C/F ghosts of phi hold
// the interpolated values; wall ghosts of phi hold the wall rule (with the wall values, if
// any), so a wall face contributes lambda_q w (phi_ghost - phi_q) to its one row.  cfidx (fine level): per element, the C/F ghost index or -1.
// covered (coarse level): per element, 1 if covered.  lamc: coarse lambda (fine level: the
// coarse cell of a C/F ghost takes the reflux part).
__global__ void __launch_bounds__(AT)
    k_grad_beta(const DevBox* __restrict__ boxes, const DevGeom* __restrict__ geoms, const Chunk* __restrict__ chunks,
                const double* __restrict__ phi, const double* __restrict__ lam, const double* __restrict__ beta,
                double b, const int* __restrict__ cfidx, const CfGhost* __restrict__ cfg,
                const double* __restrict__ lamc, double hf_over_hc, const unsigned char* __restrict__ covered,
                double* out) {
  const Chunk ch = chunks[blockIdx.x];
  const DevBox B = boxes[ch.item];
  const DevGeom G = geoms[B.solve];
  const int t = ch.start + threadIdx.x;
  if (t >= B.nx * B.ny * B.nz) return;
  const int loc[3] = {t % B.nx, (t / B.nx) % B.ny, t / (B.nx * B.ny)};
  const int n[3] = {B.nx, B.ny, B.nz};
  const int64_t q = elem_index(B, loc[0], loc[1], loc[2]);
  if (covered && covered[q]) {
    out[q] = 0.0;
    return;
  }
  double acc = 0.0;
  const double pq = phi[q], lq = lam[q], bq = beta[q];
  for (int d = 0; d < 3; ++d) {
    const double ih2 = b * G.ih2[d];
    const int64_t sd = ax_stride(B, d);
    for (int side = 0; side < 2; ++side) {
      const int64_t nq = side ? q + sd : q - sd;
      const int nloc = loc[d] + (side ? 1 : -1);
      const bool ghost = nloc < 0 || nloc >= n[d];
      const int gface = B.lo[d] + loc[d] + side;  // global index of the face
      const bool wall = (side == 0 && G.wall_lo[d] && gface == G.dlo[d]) ||
                        (side == 1 && G.wall_hi[d] && gface == G.dhi[d] + 1);
      if (wall) {  // one row: q's, with w (phi_q - phi_g); beta_face = beta_q
        if ((side ? G.wall_hi[d] : G.wall_lo[d]) == 3 && n[d] >= 2)
          acc += lq * ih2 * ((phi[nq] - 2.0 * pq) - pq);  // quadratic: the ghost holds phi_1 / 3 (+ 8g/3)
        else
          acc += lq * ih2 * (phi[nq] - pq);
        continue;
      }
      if (ghost && cfidx && cfidx[nq] >= 0) {  // fine coarse/fine face: fine row + reflux row
        const CfGhost C = cfg[cfidx[nq]];
        const double pg = phi[nq];
        acc += -lq * ih2 * (pq - pg);
        acc += -lamc[C.cq[0]] * 0.25 * ih2 * hf_over_hc * (pg - pq);
        continue;
      }
      if (covered && covered[nq]) continue;  // coarse face under reflux: not in the operator
      const double pn = phi[nq], ln = lam[nq], bn = beta[nq];
      const double gf = -ih2 * (pq - pn) * (lq - ln);
      const double s = bq + bn;
      acc += gf * 2.0 * bn * bn / (s * s);
    }
  }
  out[q] = acc;
}

}  // namespace

static unsigned nblk(int n) { return (unsigned)((n + AT - 1) / AT); }

void launch_cf_fill(const AmrDev& A, double* f, const double* c, int mode, cudaStream_t s) {
  if (!A.ncf) return;
  count_launches(1);
  k_cf_fill<<<nblk(A.ncf), AT, 0, s>>>(A.cf, A.ncf, f, c, mode);
}

void launch_reflux(const AmrDev& A, const Coefs& cc, const Coefs& cf, const double* c, const double* f,
                   const double* in, double* out, int std_part, cudaStream_t s) {
  if (!A.nrcell) return;
  count_launches(1);
  k_reflux<<<nblk(A.nrcell), AT, 0, s>>>(A.rcells, A.nrcell, A.rfaces, (const double*)cc.wx, (const double*)cc.wy,
                                          (const double*)cc.wz, (const double*)cf.wx, (const double*)cf.wy,
                                          (const double*)cf.wz, c, f, in, out, std_part, A.hf_over_hc);
}

__global__ void __launch_bounds__(AT) k_avgdown_faces(const AvgFace* __restrict__ t, int n,
                                                      const double* __restrict__ fwx, const double* __restrict__ fwy,
                                                      const double* __restrict__ fwz, double* cwx, double* cwy,
                                                      double* cwz) {
  const int i = blockIdx.x * AT + threadIdx.x;
  if (i >= n) return;
  const AvgFace a = t[i];
  const double* fw = a.d == 0 ? fwx : (a.d == 1 ? fwy : fwz);
  double* cw = a.d == 0 ? cwx : (a.d == 1 ? cwy : cwz);
  const double sum = fw[a.f0] + fw[a.f0 + a.s2] + fw[a.f0 + a.s1] + fw[a.f0 + a.s1 + a.s2];
  cw[a.cslot] = sum * 0.0625;
}

__global__ void __launch_bounds__(AT) k_avgdown_cells(const AvgCell* __restrict__ t, int n,
                                                      const double* __restrict__ fa, double* ca) {
  const int i = blockIdx.x * AT + threadIdx.x;
  if (i >= n) return;
  const AvgCell a = t[i];
  double sum = 0.0;
  for (int e = 0; e < 8; ++e) sum += fa[a.f0 + (e & 1) + (int64_t)a.sx * ((e >> 1) & 1) + (int64_t)a.sy * (e >> 2)];
  ca[a.cq] = 0.125 * sum;
}

void launch_avgdown_coefs(const AmrDev& A, const double* facoef, const double* fwx, const double* fwy,
                          const double* fwz, double* cacoef, double* cwx, double* cwy, double* cwz, cudaStream_t s) {
  if (A.navg_face) {
    count_launches(1);
    k_avgdown_faces<<<nblk(A.navg_face), AT, 0, s>>>(A.avg_faces, A.navg_face, fwx, fwy, fwz, cwx, cwy, cwz);
  }
  if (A.navg_cell) {
    count_launches(1);
    k_avgdown_cells<<<nblk(A.navg_cell), AT, 0, s>>>(A.avg_cells, A.navg_cell, facoef, cacoef);
  }
}

void launch_zero_covered(const AmrDev& A, double* c, cudaStream_t s) {
  if (!A.ncov) return;
  count_launches(1);
  k_zero_list<<<nblk(A.ncov), AT, 0, s>>>(A.covered_list, A.ncov, c);
}

void launch_composite_transpose_couplings(const AmrDev& A, const Coefs& cc, const Coefs& cf, const double* yc,
                                          const double* yf, double* outc, double* outf, cudaStream_t s) {
  if (A.ncf) {
    count_launches(1);
    k_cf_transpose<<<nblk(A.ncf), AT, 0, s>>>(A.cf, A.ncf, (const double*)cf.wx, (const double*)cf.wy,
                                              (const double*)cf.wz, yf, outc, outf);
  }
  if (A.nrcell) {
    count_launches(1);
    k_reflux_transpose<<<nblk(A.nrcell), AT, 0, s>>>(A.rcells, A.nrcell, A.rfaces, A.cf, (const double*)cc.wx,
                                                     (const double*)cc.wy, (const double*)cc.wz, (const double*)cf.wx,
                                                     (const double*)cf.wy, (const double*)cf.wz, yc, outc, outf,
                                                     A.hf_over_hc);
  }
}

void launch_grad_beta(const LevelDev& L, const double* phi, const double* lam, const double* beta, double b,
                      const int* cfidx, const CfGhost* cfg, const double* lamc, double hf_over_hc,
                      const unsigned char* covered, double* out, cudaStream_t s) {
  if (!L.n_cell_chunks) return;
  count_launches(1);
  k_grad_beta<<<L.n_cell_chunks, AT, 0, s>>>(L.boxes, L.geoms, L.cell_chunks, phi, lam, beta, b, cfidx, cfg, lamc,
                                             hf_over_hc, covered, out);
}

}  // namespace gmg

// ------------------------------------------------------------- vector helpers

namespace gmg {
namespace {

__global__ void __launch_bounds__(AT) k_dot_partial(const DevBox* __restrict__ boxes, const Chunk* __restrict__ chunks,
                                                    const double* __restrict__ x, const double* __restrict__ y,
                                                    double* partials) {
  __shared__ double red[AT / 32];
  const Chunk ch = chunks[blockIdx.x];
  const DevBox B = boxes[ch.item];
  const int t = ch.start + threadIdx.x;
  double v = 0.0;
  if (t < B.nx * B.ny * B.nz) {
    const int i = t % B.nx, j = (t / B.nx) % B.ny, k = t / (B.nx * B.ny);
    const int64_t q = elem_index(B, i, j, k);
    v = x[q] * y[q];
  }
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < AT / 32; ++w) s += red[w];
    partials[blockIdx.x] = s;
  }
}

__global__ void __launch_bounds__(AT) k_reduce_sum(const double* __restrict__ partials, int n, double* out) {
  __shared__ double red[AT / 32];
  double v = 0.0;
  for (int i = threadIdx.x; i < n; i += AT) v += partials[i];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < AT / 32; ++w) s += red[w];
    *out = s;
  }
}

__global__ void k_axpby(int64_t n, double a, const double* __restrict__ x, double b, const double* __restrict__ y,
                        double* out) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    out[i] = a * x[i] + b * y[i];
}

}  // namespace

void launch_dot(const LevelDev& L, const double* x, const double* y, double* partials, double* out, cudaStream_t s) {
  if (!L.n_cell_chunks) return;
  count_launches(2);
  k_dot_partial<<<L.n_cell_chunks, AT, 0, s>>>(L.boxes, L.cell_chunks, x, y, partials);
  k_reduce_sum<<<1, AT, 0, s>>>(partials, L.n_cell_chunks, out);
}

void launch_axpby(int64_t n, double a, const double* x, double b, const double* y, double* out, cudaStream_t s) {
  if (n <= 0) return;
  count_launches(1);
  const unsigned g = (unsigned)std::min<int64_t>((n + AT - 1) / AT, 152 * 16);
  k_axpby<<<g, AT, 0, s>>>(n, a, x, b, y, out);
}

}  // namespace gmg
