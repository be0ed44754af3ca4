// sweep.cu -- one red-black Gauss-Seidel sweep (red half-sweep then black half-sweep) in
// one pass over memory.
//
// The two half-sweeps of a sweep each read every coefficient array in full (a sector holds
// cells of both colours), so two passes move twice the data one pass needs.  Here a block
// owns a region of a box (full x extent, a slab of rows and planes) and marches through
// its planes: at step j it updates the red cells of plane z0 + j, then the black cells of
// plane z0 + j - 1, whose red neighbours above, below and beside are then final.  Plane
// z0 + j - 1 was brought into L2 by the red step before, so the coefficient arrays come
// from DRAM once per sweep.
//
// A black cell on the boundary of its region needs red values of a neighbouring region
// (or box) that another block computes at an unknown time, and a red cell next to that
// boundary needs the black value there before it changes.  Such black cells are left
// untouched by the region pass and updated afterwards by the fix-up pass (after the red
// ghost exchange), so every update sees exactly the operands of the two-pass sweep: red
// cells the old black values, black cells the new red values.  Results are bitwise those
// of k_smooth colour 0 followed by k_smooth colour 1.
#include <cuda_bf16.h>

#include "kernels.h"

namespace gmg {
namespace {

using bf16 = __nv_bfloat16;
constexpr int SWT = 512;  // threads of a sweep block

template <class T> struct SA { using type = float; };
template <> struct SA<double> { using type = double; };
template <class T> struct SC { using type = float; };
template <> struct SC<double> { using type = double; };

__device__ __forceinline__ double sld(const double* p) { return *p; }
__device__ __forceinline__ float sld(const float* p) { return *p; }
__device__ __forceinline__ float sld(const bf16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ double sldg(const double* p) { return __ldg(p); }
__device__ __forceinline__ float sldg(const float* p) { return __ldg(p); }
__device__ __forceinline__ float sldg(const bf16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ void sst(double* p, double v) { *p = v; }
__device__ __forceinline__ void sst(float* p, float v) { *p = v; }
__device__ __forceinline__ void sst(bf16* p, float v) { *p = __float2bfloat16_rn(v); }

// the Gauss-Seidel update of cell q (the arithmetic and order of k_smooth)
template <class T>
__device__ __forceinline__ void gs_update(T* phi, const T* __restrict__ rhs, const typename SC<T>::type* __restrict__ wx,
                                          const typename SC<T>::type* __restrict__ wy,
                                          const typename SC<T>::type* __restrict__ wz,
                                          const typename SC<T>::type* __restrict__ invD, int64_t q, int64_t sx,
                                          int64_t sy) {
  using A = typename SA<T>::type;
  A s = sldg(rhs + q);
  s = fma((A)sldg(wx + q), (A)sld(phi + q - 1), s);
  s = fma((A)sldg(wx + q + 1), (A)sld(phi + q + 1), s);
  s = fma((A)sldg(wy + q), (A)sld(phi + q - sx), s);
  s = fma((A)sldg(wy + q + sx), (A)sld(phi + q + sx), s);
  s = fma((A)sldg(wz + q), (A)sld(phi + q - sy), s);
  s = fma((A)sldg(wz + q + sy), (A)sld(phi + q + sy), s);
  sst(phi + q, s * (A)sldg(invD + q));
}

// ---------------------------------------------------------------- TMA-staged region pass
//
// Each plane of a region is staged in shared memory by six 1-D bulk copies (TMA), one per
// array (phi, rhs, wx, wy, wz, 1/D): the rows [y0 - 1, y0 + ny] of the plane are one
// contiguous range of the ghosted layout (start 16-byte aligned, length a multiple of 16
// bytes).  Four slots rotate: while red plane k and black plane k - 1 are computed from
// slots k - 1, k, k + 1, plane k + 2 streams into the fourth (eight slots with thinner
// regions, or one thread waiting for all, measured slower: 287 / 321 us vs 176 us).  An mbarrier per
// slot counts the bytes in; every wait on it is bounded, and a wait that gives up raises
// err.
constexpr int NSLOT = 4;
constexpr long long WAIT_LIMIT = 1ll << 26;  // try_wait polls before a wait gives up

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait for phase `parity` of bar; false (and err set) if it did not complete
__device__ __forceinline__ bool mbar_wait(unsigned long long* bar, unsigned parity, int* err) {
  for (long long n = 0; n < WAIT_LIMIT; ++n)
    if (mbar_try_wait(bar, parity)) return true;
  atomicExch(err, 1);
  return false;
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// staged plane: phi and rhs (type T), then wx, wy, wz, 1/D (float), each `cap` elements
template <class T>
struct Slot {
  T* phi;
  T* rhs;
  float* w[4];  // wx, wy, wz, invD
};

template <class T>
__device__ __forceinline__ Slot<T> slot_at(unsigned char* base, int s, int cap) {
  const size_t sz = (size_t)cap * (2 * sizeof(T) + 4 * sizeof(float));
  unsigned char* p = base + (size_t)s * sz;
  Slot<T> S;
  S.phi = (T*)p;
  S.rhs = (T*)(p + (size_t)cap * sizeof(T));
  float* f = (float*)(p + (size_t)cap * 2 * sizeof(T));
  for (int a = 0; a < 4; ++a) S.w[a] = f + (size_t)a * cap;
  return S;
}

template <class T>
__global__ void __launch_bounds__(SWT, 1)
    k_sweep_tma(const DevBox* __restrict__ boxes, const SweepRegion* __restrict__ regions, int nreg, T* phi,
                const T* __restrict__ rhs, const float* __restrict__ wx, const float* __restrict__ wy,
                const float* __restrict__ wz, const float* __restrict__ invD, const int* __restrict__ active,
                int cap, int* err) {
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned long long* bar = (unsigned long long*)smem;
  unsigned char* slots = smem + 128;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NSLOT; ++s) mbar_init(&bar[s], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  unsigned uses[NSLOT] = {};  // copies issued into each slot (same in every thread)
  for (int r = blockIdx.x; r < nreg; r += gridDim.x) {
    const SweepRegion R = regions[r];
    const DevBox B = boxes[R.box];
    if (active && !active[B.solve]) continue;
    const int npx = (B.nx + 1) >> 1;
    const int np = npx * R.ny;
    const int par = B.lo[0] + B.lo[1] + B.lo[2];
    const int sx = B.sx;
    const int64_t sy = B.sy;
    const int ylast = R.y0 + R.ny - 1, zlast = R.z0 + R.nz - 1;
    const unsigned bytesT = (unsigned)((R.ny + 2) * sx * sizeof(T));
    const unsigned bytesF = (unsigned)((R.ny + 2) * sx * sizeof(float));
    // plane p of the region is z0 - 1 + p; its rows start at global element g0(k)
    auto g0 = [&](int k) { return B.off + (int64_t)sx * R.y0 + sy * (k + 1); };
    auto issue = [&](int p) {  // thread 0 only
      const int s = p % NSLOT;
      const int k = R.z0 - 1 + p;
      Slot<T> S = slot_at<T>(slots, s, cap);
      const int64_t g = g0(k);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(&bar[s], 2 * bytesT + 4 * bytesF);
      bulk_g2s(S.phi, phi + g, bytesT, &bar[s]);
      bulk_g2s(S.rhs, rhs + g, bytesT, &bar[s]);
      bulk_g2s(S.w[0], wx + g, bytesF, &bar[s]);
      bulk_g2s(S.w[1], wy + g, bytesF, &bar[s]);
      bulk_g2s(S.w[2], wz + g, bytesF, &bar[s]);
      bulk_g2s(S.w[3], invD + g, bytesF, &bar[s]);
    };
    const int nplanes = R.nz + 2;  // z0 - 1 .. zlast + 1
    // the first NSLOT planes now; then, at step j, plane j - 1 + NSLOT into the slot of plane
    // j - 1 (k - 2, no longer read from shared memory)
    if (threadIdx.x == 0)
      for (int p = 0; p < NSLOT && p < nplanes; ++p) issue(p);
    for (int p = 0; p < NSLOT && p < nplanes; ++p) uses[p % NSLOT]++;
    bool good = true;
    for (int p = 0; p < 2; ++p) good &= mbar_wait(&bar[p % NSLOT], (uses[p % NSLOT] - 1) & 1, err);
    for (int j = 0; j < R.nz; ++j) {
      const int k = R.z0 + j;
      if (j >= 1 && j - 1 + NSLOT < nplanes) {
        if (threadIdx.x == 0) issue(j - 1 + NSLOT);
        uses[(j - 1 + NSLOT) % NSLOT]++;
      }
      good &= mbar_wait(&bar[(j + 2) % NSLOT], (uses[(j + 2) % NSLOT] - 1) & 1, err);
      const Slot<T> Sm = slot_at<T>(slots, j % NSLOT, cap);        // plane k - 1
      const Slot<T> S0 = slot_at<T>(slots, (j + 1) % NSLOT, cap);  // plane k
      const Slot<T> Sp = slot_at<T>(slots, (j + 2) % NSLOT, cap);  // plane k + 1
      using A = float;
      const int64_t gk = g0(k);
      for (int t = threadIdx.x; t < np; t += SWT) {  // red cells of plane k
        const int y = R.y0 + t / npx;
        const int i = 2 * (t % npx) + ((par + y + k) & 1);
        if (i >= B.nx) continue;
        const int l = (y - R.y0 + 1) * sx + GX + i;
        A v = sld(S0.rhs + l);
        v = fma(S0.w[0][l], sld(S0.phi + l - 1), v);
        v = fma(S0.w[0][l + 1], sld(S0.phi + l + 1), v);
        v = fma(S0.w[1][l], sld(S0.phi + l - sx), v);
        v = fma(S0.w[1][l + sx], sld(S0.phi + l + sx), v);
        v = fma(S0.w[2][l], sld(Sm.phi + l), v);
        v = fma(Sp.w[2][l], sld(Sp.phi + l), v);
        v = v * S0.w[3][l];
        sst(S0.phi + l, v);
        sst(phi + gk + l, v);
      }
      __syncthreads();
      const int kb = k - 1;  // black cells of plane k - 1 inside the region
      if (kb > R.z0 && kb < zlast) {
        const int64_t gb = g0(kb);
        for (int t = threadIdx.x; t < np; t += SWT) {
          const int y = R.y0 + t / npx;
          const int i = 2 * (t % npx) + ((par + y + kb + 1) & 1);
          if (i <= 0 || i >= B.nx - 1 || y == R.y0 || y == ylast) continue;
          const int l = (y - R.y0 + 1) * sx + GX + i;
          A v = sld(Sm.rhs + l);
          v = fma(Sm.w[0][l], sld(Sm.phi + l - 1), v);
          v = fma(Sm.w[0][l + 1], sld(Sm.phi + l + 1), v);
          v = fma(Sm.w[1][l], sld(Sm.phi + l - sx), v);
          v = fma(Sm.w[1][l + sx], sld(Sm.phi + l + sx), v);
          v = fma(Sm.w[2][l], sld(phi + gb + l - sy), v);  // plane k - 2: red values in global memory
          v = fma(S0.w[2][l], sld(S0.phi + l), v);
          v = v * Sm.w[3][l];
          sst(Sm.phi + l, v);
          sst(phi + gb + l, v);
        }
      }
      __syncthreads();
    }
    // planes issued but not consumed by a step: none (the last issue is plane zlast + 1,
    // waited in the last step); drain defensively in case a wait gave up
    if (!good)
      for (int s = 0; s < NSLOT; ++s)
        if (uses[s]) mbar_wait(&bar[s], (uses[s] - 1) & 1, err);
    __syncthreads();
  }
}

// The black cells the region pass left: its first and last plane, its first and last row
// of the other planes, and the x-face cells of the remaining rows.
template <class T>
__global__ void __launch_bounds__(SWT)
    k_sweep_fixup(const DevBox* __restrict__ boxes, const SweepRegion* __restrict__ regions, T* phi,
                  const T* __restrict__ rhs, const typename SC<T>::type* __restrict__ wx,
                  const typename SC<T>::type* __restrict__ wy, const typename SC<T>::type* __restrict__ wz,
                  const typename SC<T>::type* __restrict__ invD, const int* __restrict__ active) {
  const SweepRegion R = regions[blockIdx.x];
  const DevBox B = boxes[R.box];
  if (active && !active[B.solve]) return;
  const int npx = (B.nx + 1) >> 1;
  const int par = B.lo[0] + B.lo[1] + B.lo[2];
  const int64_t sx = B.sx, sy = B.sy;
  const int nbp = R.nz >= 2 ? 2 : 1;          // boundary planes
  const int nip = R.nz - nbp;                  // interior planes
  const int nbr = R.ny >= 2 ? 2 : 1;           // boundary rows of an interior plane
  const int nir = R.ny - nbr;                  // interior rows
  const int nend = B.nx >= 2 ? 2 : 1;          // x-face cells of an interior row
  const int n_plane = npx * R.ny;              // pair items of a boundary plane
  const int n_iplane = nbr * npx + nir * nend; // items of an interior plane
  const int total = nbp * n_plane + nip * n_iplane;
  for (int t = threadIdx.x; t < total; t += SWT) {
    int i, y, k;
    if (t < nbp * n_plane) {
      const int pl = t / n_plane, u = t % n_plane;
      k = pl == 0 ? R.z0 : R.z0 + R.nz - 1;
      y = R.y0 + u / npx;
      i = 2 * (u % npx) + ((par + y + k + 1) & 1);
      if (i >= B.nx) continue;
    } else {
      const int u0 = t - nbp * n_plane;
      k = R.z0 + 1 + u0 / n_iplane;
      const int u = u0 % n_iplane;
      if (u < nbr * npx) {
        const int row = u / npx;
        y = row == 0 ? R.y0 : R.y0 + R.ny - 1;
        i = 2 * (u % npx) + ((par + y + k + 1) & 1);
        if (i >= B.nx) continue;
      } else {
        const int v = u - nbr * npx;
        y = R.y0 + 1 + v / nend;
        i = (v % nend) == 0 ? 0 : B.nx - 1;
        if (((par + i + y + k) & 1) != 1) continue;
      }
    }
    gs_update(phi, rhs, wx, wy, wz, invD, elem_index(B, i, y, k), sx, sy);
  }
}

}  // namespace

#define GMG_SWEEP_DISPATCH(dt, KERNEL)                                                                       \
  switch (dt) {                                                                                               \
    case DT_F64: KERNEL<double><<<n, SWT, 0, s>>>(L.boxes, regions, (double*)phi, (const double*)rhs,          \
                                                  (const double*)c.wx, (const double*)c.wy, (const double*)c.wz, \
                                                  (const double*)c.invD, L.active); break;                    \
    case DT_F32: KERNEL<float><<<n, SWT, 0, s>>>(L.boxes, regions, (float*)phi, (const float*)rhs,             \
                                                 (const float*)c.wx, (const float*)c.wy, (const float*)c.wz,    \
                                                 (const float*)c.invD, L.active); break;                       \
    default: KERNEL<bf16><<<n, SWT, 0, s>>>(L.boxes, regions, (bf16*)phi, (const bf16*)rhs, (const float*)c.wx,  \
                                            (const float*)c.wy, (const float*)c.wz, (const float*)c.invD,       \
                                            L.active); break;                                                  \
  }

size_t sweep_smem_bytes(int dt, int cap) {
  const size_t el = dt == DT_BF16 ? 2 : 4;
  return 128 + (size_t)NSLOT * (size_t)cap * (2 * el + 4 * sizeof(float));
}

bool launch_sweep(int dt, const LevelDev& L, void* phi, const void* rhs, const Coefs& c, int* err, cudaStream_t s) {
  const int n = L.n_sweep_regions;
  if (!n || dt == DT_F64 || L.sweep_cap <= 0) return false;
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 1;
  }
  const size_t smem = sweep_smem_bytes(dt, L.sweep_cap);
  const int grid = n < nsm ? n : nsm;
  count_launches(1);
  if (dt == DT_F32) {
    cudaFuncSetAttribute(k_sweep_tma<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_sweep_tma<float><<<grid, SWT, smem, s>>>(L.boxes, L.sweep_regions, n, (float*)phi, (const float*)rhs,
                                               (const float*)c.wx, (const float*)c.wy, (const float*)c.wz,
                                               (const float*)c.invD, L.active, L.sweep_cap, err);
  } else {
    cudaFuncSetAttribute(k_sweep_tma<bf16>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_sweep_tma<bf16><<<grid, SWT, smem, s>>>(L.boxes, L.sweep_regions, n, (bf16*)phi, (const bf16*)rhs,
                                              (const float*)c.wx, (const float*)c.wy, (const float*)c.wz,
                                              (const float*)c.invD, L.active, L.sweep_cap, err);
  }
  return true;
}

void launch_sweep_fixup(int dt, const LevelDev& L, void* phi, const void* rhs, const Coefs& c, cudaStream_t s) {
  const int n = L.n_sweep_regions;
  if (!n) return;
  const SweepRegion* regions = L.sweep_regions;
  count_launches(1);
  GMG_SWEEP_DISPATCH(dt, k_sweep_fixup)
}

}  // namespace gmg
