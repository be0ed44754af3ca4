// dev_util.cuh -- device helpers shared by the smoother kernels (kernels.cu, flow.cu):
// element-typed loads and stores, the dependent-launch entry and the ghost push.
#pragma once

#include <cuda_bf16.h>

#include "kernels.h"

namespace gmg {
namespace {

using bf16 = __nv_bfloat16;

template <class T> struct Arith { using type = float; };
template <> struct Arith<double> { using type = double; };
template <class T> struct CoefOf { using type = float; };
template <> struct CoefOf<double> { using type = double; };

__device__ __forceinline__ double ld(const double* p) { return *p; }
__device__ __forceinline__ float ld(const float* p) { return *p; }
__device__ __forceinline__ float ld(const bf16* p) { return __bfloat162float(*p); }
__device__ __forceinline__ double ldg(const double* p) { return __ldg(p); }
__device__ __forceinline__ float ldg(const float* p) { return __ldg(p); }
__device__ __forceinline__ float ldg(const bf16* p) { return __bfloat162float(*p); }

__device__ __forceinline__ void st(double* p, double v) { *p = v; }
__device__ __forceinline__ void st(float* p, double v) { *p = (float)v; }
__device__ __forceinline__ void st(float* p, float v) { *p = v; }
__device__ __forceinline__ void st(bf16* p, float v) { *p = __float2bfloat16_rn(v); }
__device__ __forceinline__ void st(bf16* p, double v) { *p = __float2bfloat16_rn((float)v); }

__device__ __forceinline__ int64_t axis_stride(const DevBox& B, int d) {
  return d == 0 ? 1 : (d == 1 ? (int64_t)B.sx : B.sy);
}

// Programmatic dependent launch: a kernel launched with the programmatic-serialization
// attribute may start while its predecessor in the stream finishes; it waits here for the
// predecessor's completion (and memory) before touching global memory, then lets its own
// successor launch early.  Without the attribute both instructions return at once.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Colour-split storage of a row (the finest level's right-hand side and 1/D, where the
// level allows it): the row's red cells (even global parity) at x-slots [0, nx/2), its black
// cells at [nx/2, nx), each half in x order; nx even.  A colour pass then reads half of every
// such row instead of every sector of it.  Ghost slots are not used (these arrays have none).
__device__ __forceinline__ int64_t split_index(const DevBox& B, int i, int j, int k) {
  return B.off + GX + (i >> 1) + (((B.lo[0] + B.lo[1] + B.lo[2] + i + j + k) & 1) ? (B.nx >> 1) : 0) +
         (int64_t)B.sx * (j + 1) + B.sy * (k + 1);
}
// the same slot from the ordinary element q0 of an even cell i0 of the row: the cell of colour
// c (0 red) of the pair (i0, i0 + 1) sits at q0 - i0 / 2 (+ nx / 2 if black)
__device__ __forceinline__ int64_t split_pair_slot(int64_t q0, int i0, int c, int nx) {
  return q0 - (i0 >> 1) + (c ? (nx >> 1) : 0);
}
// the element of cell (i, j, k), whose element in the ordinary layout is q, in an array that
// is colour-split (split) or not
__device__ __forceinline__ int64_t cell_slot(bool split, const DevBox& B, int i, int j, int k, int64_t q) {
  return split ? split_index(B, i, j, k) : q;
}

// decode a pair item of box B into (i0, j, k); i0 even
__device__ __forceinline__ void pair_decode(const DevBox& B, int t, int& i0, int& j, int& k) {
  const int npx = (B.nx + 1) >> 1;
  const int p = t % npx;
  const int r = t / npx;
  j = r % B.ny;
  k = r / B.ny;
  i0 = 2 * p;
}

// Ghost push: the new value v of cell (i, j, k) of box B (index b) is also written into
// the ghost cells that copy it -- one per face of B the cell lies on, the whole face being
// copied to a translate in one box (walls: into B's own ghost, negated) -- so the next step
// needs no ghost exchange.  The values a pull exchange would copy land in the same places;
// the caller uses it only where a ghost has its source's colour (even periodic lengths),
// so a colour pass never reads a ghost it writes.
template <class T, class A>
__device__ __forceinline__ void push_ghosts(const DevBox& B, int b, const DevBox* __restrict__ boxes,
                                            const PushFace* __restrict__ faces, T* f, int i, int j, int k, A v) {
  if (i != 0 && i != B.nx - 1 && j != 0 && j != B.ny - 1 && k != 0 && k != B.nz - 1) return;
#pragma unroll
  for (int fc = 0; fc < 6; ++fc) {
    const int d = fc >> 1;
    const int c = d == 0 ? i : (d == 1 ? j : k);
    const int nd = d == 0 ? B.nx : (d == 1 ? B.ny : B.nz);
    if (c != ((fc & 1) ? nd - 1 : 0)) continue;
    const PushFace P = faces[6 * b + fc];
    if (P.box < 0) continue;
    const A w = P.sign < 0 ? -v : v;
    if (P.direct) {
      st(f + elem_index(B, i, j, k) + P.delta, w);
    } else {
      const DevBox Bd = boxes[P.box];
      st(f + elem_index(Bd, i + P.dx, j + P.dy, k + P.dz), w);
    }
  }
}

// push_ghosts restricted to the wall faces: only the cell's own images
template <class T, class A>
__device__ __forceinline__ void push_walls(const DevBox& B, int b, const DevBox* __restrict__ boxes,
                                            const PushFace* __restrict__ faces, T* f, int i, int j, int k, A v) {
  if (i != 0 && i != B.nx - 1 && j != 0 && j != B.ny - 1 && k != 0 && k != B.nz - 1) return;
#pragma unroll
  for (int fc = 0; fc < 6; ++fc) {
    const int d = fc >> 1;
    const int c = d == 0 ? i : (d == 1 ? j : k);
    const int nd = d == 0 ? B.nx : (d == 1 ? B.ny : B.nz);
    if (c != ((fc & 1) ? nd - 1 : 0)) continue;
    const PushFace P = faces[6 * b + fc];
    if (P.box < 0 || !P.wall) continue;
    const A w = P.sign < 0 ? -v : v;
    if (P.direct) {
      st(f + elem_index(B, i, j, k) + P.delta, w);
    } else {
      const DevBox Bd = boxes[P.box];
      st(f + elem_index(Bd, i + P.dx, j + P.dy, k + P.dz), w);
    }
  }
}

}  // namespace
}  // namespace gmg
