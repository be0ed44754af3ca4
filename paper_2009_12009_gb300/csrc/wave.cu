// wave.cu -- one red-black Gauss-Seidel sweep of a multigrid level per launch.
//
// The smoother of Sec. "Linear Solvers" (red-black Gauss-Seidel, colour = parity of i + j + k
// in the level's global index) as a wavefront: every thread block takes one tile (a band of
// rows of one box, all of its x and all of its planes) and marches through the tile's planes
// a slab at a time: the red cells of the slab's planes, a report, then the black cells of
// every plane whose red cells on both sides are done.  The black cells of a plane read the red
// cells the block has just written, so the coefficient lines they need were fetched for the
// red cells beside them a moment earlier (L1/L2), and every array of the level is read from
// HBM about once per sweep instead of once per colour.  The next slab's rows are prefetched
// into L2 with bulk prefetches while a slab is worked on.
//
// Tiles meet tiles of the same box (other row bands) and tiles of neighbouring boxes.  The
// red cells of a plane read black cells of the tiles next to them, and their black cells read
// those tiles' red cells.  So each tile counts its red planes in a progress counter (a
// release store after every step), and before the black cells of a plane it waits (acquire
// loads, bounded) until every neighbouring tile has reported that plane's reds: then the
// values it reads are those of the two-pass sweep, and the black cells it reads are still the
// old ones (the neighbour updates them only after this tile's report).  Values another block
// wrote during the launch are read from L2 (ld.global.cg): an SM's L1 is not coherent.
// Boxes stacked along z march in opposite directions and boxes side by side along x or y
// march alike (host tables), so every wait is for a step the other tile reaches no later:
// no wait can deadlock as long as every tile of a problem can be resident at once (checked
// before the launch).  Tiles are handed out in problem order by a ticket counter.  A wait
// that gives up raises the device error flag and the kernel runs to its end.
//
// Every value is computed from exactly the operands of one launch per colour (k_smooth) in
// the same order of operations: results are bitwise those of the two-pass sweep.
#include <algorithm>
#include <utility>

#include "dev_util.cuh"

namespace gmg {
namespace {

// spin budget of one wait (each round one L2 round trip plus a short sleep: a few seconds)
constexpr int WAVE_SPIN_LIMIT = 1 << 21;
// counter words: [0] ticket, [WAVE_CTL_STRIDE] tiles finished, [2 * WAVE_CTL_STRIDE + t] the
// red planes tile t has reported (one line each for the two hand-out words)
constexpr int WAVE_CTL_STRIDE = 32;

__device__ __forceinline__ unsigned wv_ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void wv_st_release(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int wv_ld_relaxed(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
// dependent launch: wait for the predecessor at entry; let the successor be scheduled only
// once this block has finished (an early start of the successor could take the slots that
// tiles this launch still waits for need)
__device__ __forceinline__ void wv_pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void wv_pdl_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// loads of values another block may have written during the launch (L2)
__device__ __forceinline__ double ldl2(const double* p) { return __ldcg(p); }
__device__ __forceinline__ float ldl2(const float* p) { return __ldcg(p); }
__device__ __forceinline__ float ldl2(const bf16* p) {
  return __bfloat162float(__ushort_as_bfloat16(__ldcg(reinterpret_cast<const unsigned short*>(p))));
}

// the value a store of v into T leaves, as the arithmetic type
__device__ __forceinline__ double kept(double v, const double*) { return v; }
__device__ __forceinline__ float kept(float v, const float*) { return v; }
__device__ __forceinline__ float kept(float v, const bf16*) { return __bfloat162float(__float2bfloat16_rn(v)); }

// Wait (one thread) until tile t has reported `need` red planes; *seen caches the last count
// observed (counts only grow).  A wait that runs out of budget, or finds the error flag
// raised by another wait, raises err and returns.
__device__ __forceinline__ void wave_wait(const unsigned* prog, int t, unsigned need, unsigned* seen, int* err) {
  if (*seen >= need) return;
  for (int spins = 0;; ++spins) {
    const unsigned v = wv_ld_acquire(prog + t);
    if (v >= need) {
      *seen = v;
      return;
    }
    if (spins >= WAVE_SPIN_LIMIT || ((spins & 255) == 255 && wv_ld_relaxed(err))) {
      atomicExch(err, 1);
      *seen = 0xffffffffu;  // give up on this neighbour for the rest of the launch
      return;
    }
    __nanosleep(64);
  }
}

// Ask L2 to fetch rows [j0, j1] of plane k of a field of box B (valid x extent, whole
// 16-byte units): one bulk prefetch per row, no registers, no completion to wait for.
template <class V>
__device__ __forceinline__ void prefetch_rows(const V* f, const DevBox& B, int j0, int j1, int k, int lane, int nl) {
  const unsigned bytes = ((unsigned)B.nx * (unsigned)sizeof(V)) & ~15u;
  if (!bytes) return;
  for (int j = j0 + lane; j <= j1; j += nl) {
    const V* p = f + elem_index(B, 0, j, k);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
  }
}

// The 14 operands of one Gauss-Seidel update in k_smooth's order: rhs, the x-, x+, y-, y+, z-,
// z+ face weights with their neighbours, 1/D.
template <class A>
struct Upd {
  A r, d, w[6], n[6];
};

template <class A>
__device__ __forceinline__ A gs_value(const Upd<A>& o) {
  A s = o.r;
#pragma unroll
  for (int f = 0; f < 6; ++f) s = fma(o.w[f], o.n[f], s);
  return s * o.d;
}

// MODE 0: a sweep of e in place.  MODE 1: the first sweep from e = 0 (valid cells and ghosts):
// the red cells are rhs / D without reading e (the two-pass sweep's products with zeros leave
// rhs + 0).  MODE 2: a sweep of e, then phi += e on both cells of every pair (the last pass of
// the finest level's post-smoothing, as k_smooth_update), phi's new values pushed into its
// ghosts when push_phi is given.
//
// A tile advances in steps of `slab` planes (in its marching order): the red cells of the
// step's planes, a report, then the black cells of every plane whose reds on both sides are
// done (all but the step's last plane, all of them in the last step); the next step's rows are
// prefetched into L2 meanwhile.  A thread's updates within a pass follow one another (the
// compiler keeps a load behind an earlier store that might alias it), so a block has one
// update per thread in flight.
template <class T, int PPT, int MODE, int MINB>
__global__ void __launch_bounds__(WAVE_BLOCK, MINB)
    k_wave(const DevBox* __restrict__ boxes, const WaveTile* __restrict__ tiles, int ntiles, unsigned* cnt, T* e,
           const T* __restrict__ rhs, const typename CoefOf<T>::type* __restrict__ wx,
           const typename CoefOf<T>::type* __restrict__ wy, const typename CoefOf<T>::type* __restrict__ wz,
           const typename CoefOf<T>::type* __restrict__ invD, const int* __restrict__ active,
           const int* __restrict__ skip, const PushFace* __restrict__ push, double* phi,
           const PushFace* __restrict__ push_phi, int* err, int slab, int sp) {
  using A = typename Arith<T>::type;
  wv_pdl_wait();
  __shared__ int s_tile;
  __shared__ int s_last;
  __shared__ unsigned s_seen[6];
  unsigned* prog = cnt + 2 * WAVE_CTL_STRIDE;
  const int tid = threadIdx.x;
  if (tid == 0) s_tile = (int)atomicAdd(cnt, 1u);
  if (tid < 6) s_seen[tid] = 0;
  __syncthreads();
  const int ti = s_tile;
  const WaveTile W = tiles[ti];
  const DevBox B = boxes[W.box];
  const bool run = !(active && !active[B.solve]) && !(skip && skip[B.solve]);
  if (run) {
    const int nz = B.nz;
    const int npx = B.nx >> 1;
    const int rows = W.y1 - W.y0;
    const int npairs = npx * rows;
    const int64_t sx = B.sx, sy = B.sy;
    const int par = B.lo[0] + B.lo[1] + B.lo[2];
    const int dir = W.dir;
    int64_t q0[PPT];  // element of cell (i0, j, 0) of the pair
    int pj[PPT], pr[PPT], ppx[PPT];
    bool ok[PPT];
#pragma unroll
    for (int u = 0; u < PPT; ++u) {
      const int p = tid + u * WAVE_BLOCK;
      ok[u] = p < npairs;
      const int r = ok[u] ? p / npx : 0;
      ppx[u] = ok[u] ? p - r * npx : 0;
      pr[u] = r;
      pj[u] = W.y0 + r;
      q0[u] = elem_index(B, 2 * ppx[u], pj[u], 0);
    }
    const int warp = tid >> 5, lane = tid & 31;
    int bdone = 0;  // black planes done (marching order)
    for (int r0 = 0; r0 < nz; r0 += slab) {
      const int r1 = min(nz, r0 + slab);  // red planes [r0, r1) of this step
      // L2 prefetch of the next step's planes (warps 0..3, rows by lane)
      if (r1 < nz && warp < 4) {
        const int n1 = min(nz, r1 + slab);
        for (int mq = r1; mq < n1; ++mq) {
          const int kk = dir ? nz - 1 - mq : mq;
          if (warp == 0) {
            prefetch_rows(e, B, W.y0 - 1, W.y1, kk, lane, 32);
          } else if (warp == 1) {
            prefetch_rows(rhs, B, W.y0, W.y1 - 1, kk, lane, 32);
            prefetch_rows(invD, B, W.y0, W.y1 - 1, kk, lane, 32);
          } else if (warp == 2) {
            prefetch_rows(wx, B, W.y0, W.y1 - 1, kk, lane, 32);
            prefetch_rows(wy, B, W.y0, W.y1, kk, lane, 32);
          } else {
            prefetch_rows(wz, B, W.y0, W.y1 - 1, kk + (dir ? 0 : 1), lane, 32);
          }
        }
      }
      // red pass: planes [r0, r1); every neighbour read is a black cell not yet updated
      for (int mq = r0; mq < r1; ++mq) {
        const int k = dir ? nz - 1 - mq : mq;
#pragma unroll
        for (int u = 0; u < PPT; ++u) {
          if (!ok[u]) continue;
          const int off = (par + pj[u] + k) & 1;  // the red cell of the pair is i0 + off
          const int64_t q = q0[u] + (int64_t)k * sy + off;
          const int64_t qs = sp ? split_index(B, 2 * ppx[u] + off, pj[u], k) : q;
          Upd<A> o;
          o.r = ldg(rhs + ((sp & SPLIT_RHS) ? qs : q));
          o.d = ldg(invD + ((sp & SPLIT_INVD) ? qs : q));
          A s;
          if (MODE == 1) {
            s = (o.r + (A)0) * o.d;
          } else {
            o.w[0] = ldg(wx + q);
            o.w[1] = ldg(wx + q + 1);
            o.w[2] = ldg(wy + q);
            o.w[3] = ldg(wy + q + sx);
            o.w[4] = ldg(wz + q);
            o.w[5] = ldg(wz + q + sy);
            o.n[0] = ld(e + q - 1);
            o.n[1] = ld(e + q + 1);
            o.n[2] = ld(e + q - sx);
            o.n[3] = ld(e + q + sx);
            o.n[4] = ld(e + q - sy);
            o.n[5] = ld(e + q + sy);
            s = gs_value(o);
          }
          st(e + q, s);
          if (push) push_ghosts(B, W.box, boxes, push, e, 2 * ppx[u] + off, pj[u], k, s);
        }
      }
      __syncthreads();  // this step's reds stored by every thread
      if (tid == 0) {
        __threadfence();
        wv_st_release(prog + ti, (unsigned)r1);
      }
      const int b1 = r1 == nz ? nz : r1 - 1;  // black planes [bdone, b1): reds on both sides done
      if (b1 > bdone) {
        if (tid < 6) {
          int t = -1;
          unsigned need = (unsigned)b1;
          const int kb_first = dir ? nz - 1 - bdone : bdone;
          const int kb_last = dir ? nz - b1 : b1 - 1;
          const int klo = min(kb_first, kb_last), khi = max(kb_first, kb_last);
          if (tid < 4) {
            t = tiles[ti].nb[tid];
          } else if (tid == 4 && klo == 0) {
            t = W.zb[0];
            need = (unsigned)W.zneed[0];
          } else if (tid == 5 && khi == nz - 1) {
            t = W.zb[1];
            need = (unsigned)W.zneed[1];
          }
          if (t >= 0 && t != ti) wave_wait(prog, t, need, &s_seen[tid], err);
        }
        __syncthreads();  // the neighbours' reds of those planes are visible
        // black pass: every neighbour read is a red cell already updated -- this block's
        // (ordinary loads after the barrier) or another block's (from L2)
        for (int mq = bdone; mq < b1; ++mq) {
          const int kb = dir ? nz - 1 - mq : mq;
#pragma unroll
          for (int u = 0; u < PPT; ++u) {
            if (!ok[u]) continue;
            const int ob = 1 - ((par + pj[u] + kb) & 1);  // the black cell of the pair is i0 + ob
            const int64_t qp = q0[u] + (int64_t)kb * sy;
            const int64_t q = qp + ob;
            const int64_t qs = sp ? split_index(B, 2 * ppx[u] + ob, pj[u], kb) : q;
            Upd<A> o;
            o.r = ldg(rhs + ((sp & SPLIT_RHS) ? qs : q));
            o.d = ldg(invD + ((sp & SPLIT_INVD) ? qs : q));
            o.w[0] = ldg(wx + q);
            o.w[1] = ldg(wx + q + 1);
            o.w[2] = ldg(wy + q);
            o.w[3] = ldg(wy + q + sx);
            o.w[4] = ldg(wz + q);
            o.w[5] = ldg(wz + q + sy);
            const A partner = (A)ld(e + qp + (1 - ob));
            const A outer = ob ? (ppx[u] < npx - 1 ? (A)ld(e + q + 1) : (A)ldl2(e + q + 1))
                               : (ppx[u] > 0 ? (A)ld(e + q - 1) : (A)ldl2(e + q - 1));
            o.n[0] = ob ? partner : outer;
            o.n[1] = ob ? outer : partner;
            o.n[2] = pr[u] > 0 ? (A)ld(e + q - sx) : (A)ldl2(e + q - sx);
            o.n[3] = pr[u] < rows - 1 ? (A)ld(e + q + sx) : (A)ldl2(e + q + sx);
            o.n[4] = kb > 0 ? (A)ld(e + q - sy) : (A)ldl2(e + q - sy);
            o.n[5] = kb < nz - 1 ? (A)ld(e + q + sy) : (A)ldl2(e + q + sy);
            const A s = gs_value(o);
            st(e + q, s);
            if (push) push_ghosts(B, W.box, boxes, push, e, 2 * ppx[u] + ob, pj[u], kb, s);
            if (MODE == 2) {
              const double eb = (double)kept(s, e);
              const double er = (double)partner;
              double2 v = *reinterpret_cast<const double2*>(phi + qp);
              v.x += ob == 0 ? eb : er;
              v.y += ob == 0 ? er : eb;
              *reinterpret_cast<double2*>(phi + qp) = v;
              if (push_phi) {
                push_ghosts(B, W.box, boxes, push_phi, phi, 2 * ppx[u], pj[u], kb, v.x);
                push_ghosts(B, W.box, boxes, push_phi, phi, 2 * ppx[u] + 1, pj[u], kb, v.y);
              }
            }
          }
        }
        bdone = b1;
      }
    }
  }
  // the last block to finish clears the counters for the next launch
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    s_last = atomicAdd(cnt + WAVE_CTL_STRIDE, 1u) == (unsigned)(ntiles - 1);
  }
  __syncthreads();
  if (s_last) {
    for (int t = tid; t < ntiles; t += WAVE_BLOCK) prog[t] = 0;
    if (tid == 0) {
      cnt[0] = 0;
      cnt[WAVE_CTL_STRIDE] = 0;
    }
    __threadfence();
  }
  wv_pdl_release();
}

template <class... P, class... Args>
void launch_wave_kernel(void (*k)(P...), unsigned grid, cudaStream_t s, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(WAVE_BLOCK);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = pdl_enabled() ? 1 : 0;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  cudaLaunchKernelEx(&cfg, k, std::forward<Args>(args)...);
}

// Planes per step: the data a step of every tile touches (its planes of the seven arrays,
// read by the red pass and again by the black pass) should stay within a share of L2.
constexpr double WAVE_L2_BYTES = 48.0 * (1 << 20);
int wave_slab(const LevelDev& L, int bytes_per_cell) {
  const double layer = (double)std::max<int64_t>(1, L.wave_layer_cells) * bytes_per_cell;
  return std::max(2, std::min(16, (int)(WAVE_L2_BYTES / layer)));
}

// blocks of kernel k that fit on the device at once (0 if the query fails)
template <class K>
int resident_blocks(K k) {
  int dev = 0, nsm = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, WAVE_BLOCK, 0) != cudaSuccess) return 0;
  return nsm * per;
}

// blocks per SM the register budget is held to (capacity = SMs x MINB tiles resident at once)
constexpr int WAVE_MINB = 8;

template <class T, int PPT, int MODE>
bool wave_go(const LevelDev& L, void* e, const void* rhs, const Coefs& c, double* phi, const PushFace* pp, int* err,
             cudaStream_t s) {
  using C = typename CoefOf<T>::type;
  static int cap = -1;
  if (cap < 0) cap = resident_blocks(k_wave<T, PPT, MODE, WAVE_MINB>);
  if (L.wave_max_solve_tiles > cap) return false;  // a problem's tiles must be resident together
  launch_wave_kernel(k_wave<T, PPT, MODE, WAVE_MINB>, (unsigned)L.n_wave_tiles, s, L.boxes, L.wave_tiles,
                     L.n_wave_tiles, L.wave_cnt, (T*)e, (const T*)rhs, (const C*)c.wx, (const C*)c.wy, (const C*)c.wz,
                     (const C*)c.invD, L.active, L.flow_skip, L.push_ok ? L.push_faces : nullptr, phi, pp, err,
                     wave_slab(L, (int)(2 * sizeof(T) + 5 * sizeof(C))), L.split);
  return true;
}

template <class T, int MODE>
bool wave_ppt(const LevelDev& L, void* e, const void* rhs, const Coefs& c, double* phi, const PushFace* pp, int* err,
              cudaStream_t s) {
  switch (L.wave_ppt) {
    case 1: return wave_go<T, 1, MODE>(L, e, rhs, c, phi, pp, err, s);
    case 2: return wave_go<T, 2, MODE>(L, e, rhs, c, phi, pp, err, s);
    case 4: return wave_go<T, 4, MODE>(L, e, rhs, c, phi, pp, err, s);
    default: return false;
  }
}

template <class T>
bool wave_mode(int mode, const LevelDev& L, void* e, const void* rhs, const Coefs& c, double* phi,
               const PushFace* pp, int* err, cudaStream_t s) {
  switch (mode) {
    case 0: return wave_ppt<T, 0>(L, e, rhs, c, phi, pp, err, s);
    case 1: return wave_ppt<T, 1>(L, e, rhs, c, phi, pp, err, s);
    default: return wave_ppt<T, 2>(L, e, rhs, c, phi, pp, err, s);
  }
}

}  // namespace

bool wave_ok(const LevelDev& L) { return L.n_wave_tiles > 0 && L.wave_cnt && L.push_ok && L.wave_ppt > 0; }

bool launch_wave(int dt, const LevelDev& L, void* e, const void* rhs, const Coefs& c, bool zero_start, double* phi,
                 bool push_phi, int* err, cudaStream_t s) {
  if (!wave_ok(L) || (zero_start && phi)) return false;
  const int mode = phi ? 2 : (zero_start ? 1 : 0);
  const PushFace* pp = phi && push_phi ? L.push_faces : nullptr;
  bool done = false;
  switch (dt) {
    case DT_F64: done = wave_mode<double>(mode, L, e, rhs, c, phi, pp, err, s); break;
    case DT_F32: done = wave_mode<float>(mode, L, e, rhs, c, phi, pp, err, s); break;
    default: done = wave_mode<bf16>(mode, L, e, rhs, c, phi, pp, err, s); break;
  }
  if (done) count_launches(1);
  return done;
}

}  // namespace gmg
