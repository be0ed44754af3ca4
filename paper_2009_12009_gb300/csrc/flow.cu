// flow.cu -- red-black Gauss-Seidel sweeps of one MG level as ONE dataflow launch.
//
// The smoother of Sec. "Linear Solvers" (red-black Gauss-Seidel, colour = parity of
// i + j + k in the level's global index) run as a sequence of colour phases (red, black,
// red, black, ...; or starting black), in place, in one persistent kernel:
//
//   * The level is cut, per problem, into z-slabs of whole planes, every box into work items
//     of about 128 cells (one warp, two pairs of cells per lane).  They are handed out to
//     warps in a host-built order, by FLOW_QUEUES atomic counters that share it out.
//   * A phase-c item on planes Q reads the other colour on planes Q-1..Q+1 as phase c-1
//     left it, and overwrites values phase c-1 read there.  So its warp waits (one lane, on
//     per-(phase, slab) completion counters, each on its own 128-byte line) until phase c-1
//     has finished in its slab and the two next to it; phase-0 items wait for nothing.
//     Every chunk comes after the chunks it waits for in the hand-out order, so a waiting
//     warp only ever waits for chunks held by running warps: no deadlock, whatever the
//     number of resident warps.
//   * Each value is therefore computed from exactly the operands of the two-pass sweep
//     (one launch per colour): results are bitwise those of k_smooth / k_smooth_update.
//   * Items of phase c+1 on a slab run shortly after phase c's on the slabs around it, so
//     the coefficient lines the second colour reads are still in L2: the sweep moves its
//     56 B/cell (FP64) from HBM about once instead of once per colour.
//
// Values written by another warp during the launch (the previous phase's colour, and the
// ghosts it pushed) are read from L2 (ld.global.cg): an SM's L1 is not coherent and may hold
// an older copy of the line.  Phase-0 items read only values no item of the launch writes
// before they finish, so they use ordinary loads.  A wait that gives up raises the device
// error flag (GMG_ERR_DEVICE_TIMEOUT for the caller) and the kernel runs to its end.
#include <algorithm>
#include <utility>

#include "dev_util.cuh"

namespace gmg {
namespace {

// smoothed-field loads: ordinary, or from L2 for values another block may have written
template <bool L2> __device__ __forceinline__ double lde(const double* p) { return L2 ? __ldcg(p) : *p; }
template <bool L2> __device__ __forceinline__ float lde(const float* p) { return L2 ? __ldcg(p) : *p; }
template <bool L2> __device__ __forceinline__ float lde(const bf16* p) {
  const unsigned short* u = reinterpret_cast<const unsigned short*>(p);
  return __bfloat162float(__ushort_as_bfloat16(L2 ? __ldcg(u) : *u));
}

// the value a store of v into T leaves, as the arithmetic type
__device__ __forceinline__ double stored(double v, const double*) { return v; }
__device__ __forceinline__ float stored(float v, const float*) { return v; }
__device__ __forceinline__ float stored(float v, const bf16*) { return __bfloat162float(__float2bfloat16_rn(v)); }

// spin budget of one wait (each round one L2 round trip plus a 100 ns sleep: ~2 s in all)
constexpr int FLOW_SPIN_LIMIT = 1 << 21;

// One item: every cell of `colour` in rows [y0, y1) x planes [z0, z1) of box B, one lane
// per x-pair as in k_smooth (same operands, same order of operations), one warp per item.
// ein and eout are the same array: a colour pass reads only the other colour (cells and the
// ghosts that copy them) and writes only its own colour and the ghosts that copy it, so no
// load reads a location a store of the pass writes -- the restrict-qualified views let the
// compiler issue a later pair's loads before an earlier pair's stores.  update: also
// phi += e on both cells of each pair (the other colour's e is final) as k_smooth_update.
template <class T, bool L2>
__device__ __forceinline__ void flow_item(const DevBox& B, int b, const FlowItem& I, int colour, bool update,
                                          int lane, const DevBox* __restrict__ boxes, const T* __restrict__ ein,
                                          T* __restrict__ eout, const T* __restrict__ rhs,
                                          const typename CoefOf<T>::type* __restrict__ wx,
                                          const typename CoefOf<T>::type* __restrict__ wy,
                                          const typename CoefOf<T>::type* __restrict__ wz,
                                          const typename CoefOf<T>::type* __restrict__ invD,
                                          const PushFace* __restrict__ push, double* __restrict__ phi,
                                          const PushFace* __restrict__ push_phi, int sp) {
  using A = typename Arith<T>::type;
  const int npx = (B.nx + 1) >> 1;
  const int ny = I.y1 - I.y0;
  const int total = npx * ny * (I.z1 - I.z0);
  const int64_t sx = B.sx, sy = B.sy;
  const int par = B.lo[0] + B.lo[1] + B.lo[2] + colour;
#pragma unroll 2
  for (int t = lane; t < total; t += 32) {
    const int p = t % npx;
    const int r = t / npx;
    const int j = I.y0 + r % ny;
    const int k = I.z0 + r / ny;
    const int i0 = 2 * p;
    const int off = (par + j + k) & 1;
    const int i = i0 + off;
    const int64_t q0 = elem_index(B, i0, j, k);
    A s = 0;
    if (i < B.nx) {
      const int64_t q = q0 + off;
      const int64_t qs = sp ? split_index(B, i, j, k) : q;
      s = ldg(rhs + ((sp & SPLIT_RHS) ? qs : q));
      s = fma((A)ldg(wx + q), (A)lde<L2>(ein + q - 1), s);
      s = fma((A)ldg(wx + q + 1), (A)lde<L2>(ein + q + 1), s);
      s = fma((A)ldg(wy + q), (A)lde<L2>(ein + q - sx), s);
      s = fma((A)ldg(wy + q + sx), (A)lde<L2>(ein + q + sx), s);
      s = fma((A)ldg(wz + q), (A)lde<L2>(ein + q - sy), s);
      s = fma((A)ldg(wz + q + sy), (A)lde<L2>(ein + q + sy), s);
      s = s * (A)ldg(invD + ((sp & SPLIT_INVD) ? qs : q));
      st(eout + q, s);
      if (push) push_ghosts(B, b, boxes, push, eout, i, j, k, s);
    }
    if (update) {
      // e of the pair: the value just stored, and the other colour's (final, maybe another
      // warp's) from L2
      if (i0 + 1 < B.nx) {
        const double e0 = off == 0 ? (double)stored(s, eout) : (double)lde<true>(ein + q0);
        const double e1 = off == 1 ? (double)stored(s, eout) : (double)lde<true>(ein + q0 + 1);
        double2 v = *reinterpret_cast<const double2*>(phi + q0);
        v.x += e0;
        v.y += e1;
        *reinterpret_cast<double2*>(phi + q0) = v;
        if (push_phi) {
          push_ghosts(B, b, boxes, push_phi, phi, i0, j, k, v.x);
          push_ghosts(B, b, boxes, push_phi, phi, i0 + 1, j, k, v.y);
        }
      } else {
        const double e0 = off == 0 ? (double)stored(s, eout) : (double)lde<true>(ein + q0);
        const double v = phi[q0] + e0;
        phi[q0] = v;
        if (push_phi) push_ghosts(B, b, boxes, push_phi, phi, i0, j, k, v);
      }
    }
  }
}

__device__ __forceinline__ int ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void red_release_add(int* p, int v) {
  asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Wait (one lane) until phase c - 1 has finished in every slab slab S depends on: the three
// counters are read together with acquire loads; a wait that runs out of its budget (or finds
// that another wait already did) raises err and returns.
__device__ __forceinline__ void wait_deps(const FlowSlab& S, const FlowSlab* __restrict__ slabs, const int* done,
                                          int nslab, int c, int* err) {
  int need[3];
  const int* pc[3];
#pragma unroll
  for (int u = 0; u < 3; ++u) {
    const int d = S.dep[u];
    need[u] = d >= 0 ? slabs[d].count : 0;
    pc[u] = done + (size_t)((c - 1) * nslab + (d >= 0 ? d : 0)) * FLOW_CNT_STRIDE;
  }
  for (int spins = 0;; ++spins) {
    int v[3];
#pragma unroll
    for (int u = 0; u < 3; ++u) v[u] = need[u] ? ld_acquire(pc[u]) : 0;
    bool ok = true;
#pragma unroll
    for (int u = 0; u < 3; ++u) ok &= v[u] >= need[u];
    if (ok) return;
    if (spins >= FLOW_SPIN_LIMIT || ((spins & 255) == 255 && ld_relaxed(err))) {
      atomicExch(err, 1);
      return;
    }
    __nanosleep(100);
  }
}

// cnt (one counter per FLOW_CNT_STRIDE ints): [0, FLOW_QUEUES) hand-out counters, then the
// warps finished, then [c * nslab + s] the items of phase c finished in slab s.  All zero
// at launch; the last warp to finish clears them.  Every warp works on its own: it takes the
// next chunk of its queue (queue q hands out chunks q, q + FLOW_QUEUES, ... of the order: a
// subsequence of it, so a chunk still comes after every chunk it waits for), waits for the
// slab's dependencies (once per (phase, slab): they stay satisfied), runs the chunk's items
// and counts them done with one release-add.
template <class T>
__global__ void __launch_bounds__(FLOW_BLOCK)
    k_flow(const DevBox* __restrict__ boxes, const FlowItem* __restrict__ items, const FlowSlab* __restrict__ slabs,
           int nslab, const FlowChunk* __restrict__ order, int norder, int* cnt, int colour0, int nphase,
           int update_last, T* e, const T* __restrict__ rhs, const typename CoefOf<T>::type* __restrict__ wx,
           const typename CoefOf<T>::type* __restrict__ wy, const typename CoefOf<T>::type* __restrict__ wz,
           const typename CoefOf<T>::type* __restrict__ invD, const int* __restrict__ active,
           const int* __restrict__ skip, const PushFace* __restrict__ push, double* phi,
           const PushFace* __restrict__ push_phi, int* err, int sp) {
  pdl_enter();
  const int lane = threadIdx.x & 31;
  const int warp = (int)(blockIdx.x * (FLOW_BLOCK / 32) + (threadIdx.x >> 5));
  const int q = warp % FLOW_QUEUES;
  int* disp = cnt + q * FLOW_CNT_STRIDE;
  int* fin = cnt + FLOW_QUEUES * FLOW_CNT_STRIDE;
  int* done = fin + FLOW_CNT_STRIDE;
  // two-stage pipeline: the entry of the chunk after the current one is loaded, and the
  // index of the one after that requested, while the current chunk runs
  int nxt = 0;
  if (lane == 0) nxt = atomicAdd(disp, 1) * FLOW_QUEUES + q;
  int cur = __shfl_sync(0xffffffffu, nxt, 0);
  FlowChunk ch = cur < norder ? order[cur] : FlowChunk{};
  if (lane == 0) nxt = atomicAdd(disp, 1) * FLOW_QUEUES + q;
  int ok_key = -1;  // (phase, slab) whose dependencies this warp has seen complete
  while (cur < norder) {
    const int cn = __shfl_sync(0xffffffffu, nxt, 0);
    const FlowChunk chn = cn < norder ? order[cn] : FlowChunk{};
    if (lane == 0 && cn < norder) nxt = atomicAdd(disp, 1) * FLOW_QUEUES + q;
    const int c = ch.phase_slab >> 24;
    const int sl = ch.phase_slab & 0xffffff;
    if (c > 0 && ch.phase_slab != ok_key) {
      if (lane == 0) wait_deps(slabs[sl], slabs, done, nslab, c, err);
      __syncwarp();
      ok_key = ch.phase_slab;
    }
    const DevBox B = boxes[ch.box];
    if (!(active && !active[B.solve]) && !(skip && skip[B.solve])) {
      const FlowItem I{ch.box, sl, ch.z0, ch.z1, ch.y0, ch.y1};
      const int colour = (colour0 + c) & 1;
      const bool upd = update_last && c == nphase - 1;
      if (c == 0)
        flow_item<T, false>(B, I.box, I, colour, upd, lane, boxes, e, e, rhs, wx, wy, wz, invD, push, phi, push_phi,
                            sp);
      else
        flow_item<T, true>(B, I.box, I, colour, upd, lane, boxes, e, e, rhs, wx, wy, wz, invD, push, phi, push_phi,
                           sp);
    }
    if (c + 1 < nphase) {
      __syncwarp();  // the lanes' stores of the item come before its count
      if (lane == 0) red_release_add(done + (size_t)(c * nslab + sl) * FLOW_CNT_STRIDE, 1);
    }
    cur = cn;
    ch = chn;
  }
  int last = 0;
  if (lane == 0) {
    __threadfence();
    last = atomicAdd(fin, 1) == (int)(gridDim.x * (FLOW_BLOCK / 32)) - 1;
  }
  if (__shfl_sync(0xffffffffu, last, 0)) {  // every other warp has finished: clear the counters
    for (int u = lane; u < FLOW_QUEUES + 1 + nphase * nslab; u += 32) cnt[(size_t)u * FLOW_CNT_STRIDE] = 0;
    __threadfence();
  }
}

// blocks of a launch: `warps` resident warps per SM (0: FLOW_WARPS_PER_SM), at most what
// the kernel's occupancy allows
template <class T>
int flow_grid(int warps) {
  static int nsm = 0, per = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_flow<T>, FLOW_BLOCK, 0);
    nsm = std::max(1, nsm);
    per = std::max(1, per);
  }
  const int want = (warps > 0 ? warps : FLOW_WARPS_PER_SM) / (FLOW_BLOCK / 32);
  return nsm * std::max(1, std::min(per, want));
}

template <class... P, class... Args>
void launch_flow_kernel(void (*k)(P...), unsigned grid, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(FLOW_BLOCK);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

}  // namespace

bool flow_ok(const LevelDev& L) { return L.n_flow_slabs > 0 && L.flow_cnt && L.push_ok; }

bool launch_flow(int dt, const LevelDev& L, void* e, const void* rhs, const Coefs& c, int colour0, int nphase,
                 double* phi, bool push_phi, int* err, cudaStream_t s, int warps) {
  if (!flow_ok(L) || nphase < 1 || nphase > FLOW_MAX_PHASES) return false;
  const int n = L.n_flow_order[nphase - 1];
  if (n <= 0) return false;
  const FlowChunk* order = L.flow_order[nphase - 1];
  const PushFace* pp = phi && push_phi ? L.push_faces : nullptr;
  const int upd = phi ? 1 : 0;
  count_launches(1);
  switch (dt) {
    case DT_F64: {
      const unsigned g = (unsigned)std::max(FLOW_QUEUES / 4, std::min((n + 3) / 4, flow_grid<double>(warps)));
      launch_flow_kernel(k_flow<double>, g, s, L.boxes, L.flow_items, L.flow_slabs, L.n_flow_slabs, order, n,
                         L.flow_cnt, colour0, nphase, upd, (double*)e, (const double*)rhs, (const double*)c.wx,
                         (const double*)c.wy, (const double*)c.wz, (const double*)c.invD, L.active, L.flow_skip,
                         L.push_faces, phi, pp, err, L.split);
    } break;
    case DT_F32: {
      const unsigned g = (unsigned)std::max(FLOW_QUEUES / 4, std::min((n + 3) / 4, flow_grid<float>(warps)));
      launch_flow_kernel(k_flow<float>, g, s, L.boxes, L.flow_items, L.flow_slabs, L.n_flow_slabs, order, n,
                         L.flow_cnt, colour0, nphase, upd, (float*)e, (const float*)rhs, (const float*)c.wx,
                         (const float*)c.wy, (const float*)c.wz, (const float*)c.invD, L.active, L.flow_skip,
                         L.push_faces, phi, pp, err, L.split);
    } break;
    default: {
      const unsigned g = (unsigned)std::max(FLOW_QUEUES / 4, std::min((n + 3) / 4, flow_grid<bf16>(warps)));
      launch_flow_kernel(k_flow<bf16>, g, s, L.boxes, L.flow_items, L.flow_slabs, L.n_flow_slabs, order, n,
                         L.flow_cnt, colour0, nphase, upd, (bf16*)e, (const bf16*)rhs, (const float*)c.wx,
                         (const float*)c.wy, (const float*)c.wz, (const float*)c.invD, L.active, L.flow_skip,
                         L.push_faces, phi, pp, err, L.split);
    } break;
  }
  return true;
}

}  // namespace gmg
