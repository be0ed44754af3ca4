// diag.cu -- measurement helper with no counterpart in the paper: a kernel of independent
// FP64 fused multiply-add chains, timed by the benchmark to state the FP64 ceiling of the
// GPU it runs on (the roofline of the FP64-pipe-bound kernels).
#include <algorithm>

#include "kernels.h"
#include "gmg.h"

namespace gmg {
namespace {

__device__ double g_dfma_sink;  // written only if the chains reach a value they cannot, keeps them live

constexpr int DFMA_CHAINS = 16;
constexpr int DFMA_BLOCK = 256;

// every thread runs DFMA_CHAINS independent chains of `iters` FMAs: 2 * DFMA_CHAINS * iters
// flops per thread
__global__ void __launch_bounds__(DFMA_BLOCK) k_dfma(int iters, double seed) {
  double a[DFMA_CHAINS];
#pragma unroll
  for (int c = 0; c < DFMA_CHAINS; ++c) a[c] = seed + 1e-3 * (threadIdx.x + c);
  const double m = 1.0 + 1e-12, add = 1e-15;
#pragma unroll 4
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < DFMA_CHAINS; ++c) a[c] = fma(a[c], m, add);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < DFMA_CHAINS; ++c) s += a[c];
  if (s == -1.0) g_dfma_sink = s;
}

}  // namespace
}  // namespace gmg

extern "C" gmg_status gmg_dfma_probe(void* stream, int blocks_per_sm, int iters, double* flops) {
  if (blocks_per_sm < 1 || blocks_per_sm > 64 || iters < 1 || !flops) return GMG_ERR_BAD_INPUT;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) !=
                                                cudaSuccess)
    return GMG_ERR_CUDA;
  const int blocks = std::max(1, nsm) * blocks_per_sm;
  gmg::k_dfma<<<blocks, gmg::DFMA_BLOCK, 0, (cudaStream_t)stream>>>(iters, 1.0);
  if (cudaGetLastError() != cudaSuccess) return GMG_ERR_CUDA;
  *flops = 2.0 * gmg::DFMA_CHAINS * (double)iters * (double)blocks * gmg::DFMA_BLOCK;
  return GMG_OK;
}
