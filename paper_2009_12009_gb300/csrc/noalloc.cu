// noalloc.cu -- a BiCGStab solve of a single box that allocates nothing.
//
// Who needs it: callers that cannot allocate device memory at the time they solve --
// for example an operator inside another framework that is handed only its input and
// output tensors, code that runs while its own stream is being captured into a CUDA
// graph (cudaMalloc is not allowed during capture), or a host that forbids allocations
// after start-up.  Such a caller cannot provide the workspace that gmg_set_workspace
// needs, so this entry point takes its inputs and output as plain device arrays and
// keeps its scratch (the seven BiCGStab vectors) in one file-scope device array.
//
// The array is a static __device__ allocation: every GPU that loads this library holds
// it (NOALLOC_MAX_ELEMS * 7 doubles = 3.5 MiB) until the process exits.  All calls share
// it and it keeps the previous call's contents; the kernel initialises every entry it
// reads before reading it.  Calls whose kernels overlap on the GPU (different streams,
// or different host threads) race on the array and must be serialised by the caller.
#include <cuda_bf16.h>

#include <atomic>
#include <string>

#include "../../include/gmg.h"
#include "internal.h"

namespace gmg {
namespace {

constexpr int NT = 512;                      // threads of the single solving block
constexpr int NOALLOC_MAX_ELEMS = 65536;     // ghosted elements per vector, (nx+2)(ny+2)(nz+2)

// the scratch: seven ghosted vectors r, rhat, p, v, s, t, x
static __device__ __align__(256) double g_noalloc_scratch[7 * NOALLOC_MAX_ELEMS];

struct NBox {
  int nx, ny, nz;
  int per[3];      // 1: periodic along d (wrap inside the box); 0: walls
  double wsign[3][2];  // wall ghost = wsign * adjacent cell: -1 homogeneous Dirichlet, +1 homogeneous Neumann
  int ncell;
  int64_t sx, sy;  // ghosted strides
};

__device__ __forceinline__ int64_t gq(const NBox& b, int i, int j, int k) {
  return (int64_t)(i + 1) + b.sx * (j + 1) + b.sy * (k + 1);
}

__device__ double nsum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s += sh[w];
    sh[NT / 32] = s;
  }
  __syncthreads();
  return sh[NT / 32];
}

__device__ double nmax(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < NT / 32; ++w) s = fmax(s, sh[w]);
    sh[NT / 32] = s;
  }
  __syncthreads();
  return sh[NT / 32];
}

__device__ __forceinline__ void cell_ijk(const NBox& b, int c, int& i, int& j, int& k) {
  i = c % b.nx;
  j = (c / b.nx) % b.ny;
  k = c / (b.nx * b.ny);
}

// face ghosts of `in`: periodic wrap inside the box, or the wall rule on the adjacent cell
__device__ void nfill(const NBox& b, double* in) {
  const int n[3] = {b.nx, b.ny, b.nz};
  for (int d = 0; d < 3; ++d) {
    const int d1 = d == 0 ? 1 : 0, d2 = d == 2 ? 1 : 2;
    const int nf = n[d1] * n[d2];
    for (int e = threadIdx.x; e < 2 * nf; e += NT) {
      const int side = e / nf, u = (e % nf) % n[d1], v = (e % nf) / n[d1];
      int g[3], s[3];
      g[d1] = s[d1] = u;
      g[d2] = s[d2] = v;
      g[d] = side ? n[d] : -1;
      double sign;
      if (b.per[d]) { s[d] = side ? 0 : n[d] - 1; sign = 1.0; }
      else { s[d] = side ? n[d] - 1 : 0; sign = b.wsign[d][side]; }
      in[gq(b, g[0], g[1], g[2])] = sign * in[gq(b, s[0], s[1], s[2])];
    }
  }
  __syncthreads();
}

// out = A in: D*in minus the weighted neighbours, the weights read from dense face arrays
__device__ void napply(const NBox& b, const double* wx, const double* wy, const double* wz, const double* D,
                       double* in, double* out) {
  nfill(b, in);
  for (int c = threadIdx.x; c < b.ncell; c += NT) {
    int i, j, k;
    cell_ijk(b, c, i, j, k);
    const int64_t q = gq(b, i, j, k);
    const int64_t fx = i + (int64_t)(b.nx + 1) * (j + (int64_t)b.ny * k);
    const int64_t fy = i + (int64_t)b.nx * (j + (int64_t)(b.ny + 1) * k);
    const int64_t fz = c;
    double v = D[c] * in[q];
    v = fma(-wx[fx], in[q - 1], v);
    v = fma(-wx[fx + 1], in[q + 1], v);
    v = fma(-wy[fy], in[q - b.sx], v);
    v = fma(-wy[fy + b.nx], in[q + b.sx], v);
    v = fma(-wz[fz], in[q - b.sy], v);
    v = fma(-wz[fz + (int64_t)b.nx * b.ny], in[q + b.sy], v);
    out[q] = v;
  }
  __syncthreads();
}

__device__ double ndot(const NBox& b, const double* x, const double* y, double* sh) {
  double s = 0.0;
  for (int c = threadIdx.x; c < b.ncell; c += NT) {
    int i, j, k;
    cell_ijk(b, c, i, j, k);
    const int64_t q = gq(b, i, j, k);
    s += x[q] * y[q];
  }
  return nsum(s, sh);
}

__device__ double nnorm(const NBox& b, const double* x, double* sh) {
  double s = 0.0;
  for (int c = threadIdx.x; c < b.ncell; c += NT) {
    int i, j, k;
    cell_ijk(b, c, i, j, k);
    s = fmax(s, fabs(x[gq(b, i, j, k)]));
  }
  return nmax(s, sh);
}

__device__ double nvsum(const NBox& b, const double* x, double* sh) {
  double s = 0.0;
  for (int c = threadIdx.x; c < b.ncell; c += NT) {
    int i, j, k;
    cell_ijk(b, c, i, j, k);
    s += x[gq(b, i, j, k)];
  }
  return nsum(s, sh);
}

// The BiCGStab iteration of the bottom kernel (bottom.cu) on one box whose inputs are
// dense arrays and whose vectors live in the static scratch `work` (7 x stride).
__global__ void __launch_bounds__(NT) k_box_bicgstab_noalloc(NBox b, const double* __restrict__ wx,
                                                            const double* __restrict__ wy,
                                                            const double* __restrict__ wz,
                                                            const double* __restrict__ D,
                                                            const double* __restrict__ rhs, double* xout,
                                                            double* work, int64_t stride, int singular, int maxit,
                                                            double tol, int* iters) {
  __shared__ double sh[NT / 32 + 1];
  double* r = work;
  double* rh = work + stride;
  double* p = work + 2 * stride;
  double* v = work + 3 * stride;
  double* s = work + 4 * stride;
  double* t = work + 5 * stride;
  double* x = work + 6 * stride;
  // the scratch keeps the previous call's values: initialise everything read below
  for (int c = threadIdx.x; c < b.ncell; c += NT) {
    int i, j, k;
    cell_ijk(b, c, i, j, k);
    const int64_t q = gq(b, i, j, k);
    r[q] = rhs[c];
    p[q] = 0.0;
    v[q] = 0.0;
    x[q] = 0.0;
  }
  __syncthreads();
  if (singular) {
    const double mean = nvsum(b, r, sh) / (double)b.ncell;
    for (int c = threadIdx.x; c < b.ncell; c += NT) {
      int i, j, k;
      cell_ijk(b, c, i, j, k);
      r[gq(b, i, j, k)] -= mean;
    }
    __syncthreads();
  }
  for (int c = threadIdx.x; c < b.ncell; c += NT) {
    int i, j, k;
    cell_ijk(b, c, i, j, k);
    rh[gq(b, i, j, k)] = r[gq(b, i, j, k)];
  }
  __syncthreads();
  const double r0 = nnorm(b, r, sh);
  double rho_old = 1.0, alpha = 1.0, omega = 1.0;
  int it = 0;
  if (r0 > 0.0) {
    for (it = 1; it <= maxit; ++it) {
      const double rho = ndot(b, rh, r, sh);
      if (fabs(rho) < 1e-300) { --it; break; }
      const double beta = (rho / rho_old) * (alpha / omega);
      for (int c = threadIdx.x; c < b.ncell; c += NT) {
        int i, j, k;
        cell_ijk(b, c, i, j, k);
        const int64_t q = gq(b, i, j, k);
        p[q] = r[q] + beta * (p[q] - omega * v[q]);
      }
      __syncthreads();
      napply(b, wx, wy, wz, D, p, v);
      const double rv = ndot(b, rh, v, sh);
      if (fabs(rv) < 1e-300) { --it; break; }
      alpha = rho / rv;
      for (int c = threadIdx.x; c < b.ncell; c += NT) {
        int i, j, k;
        cell_ijk(b, c, i, j, k);
        const int64_t q = gq(b, i, j, k);
        s[q] = r[q] - alpha * v[q];
      }
      __syncthreads();
      if (nnorm(b, s, sh) <= tol * r0) {
        for (int c = threadIdx.x; c < b.ncell; c += NT) {
          int i, j, k;
          cell_ijk(b, c, i, j, k);
          const int64_t q = gq(b, i, j, k);
          x[q] += alpha * p[q];
        }
        __syncthreads();
        break;
      }
      napply(b, wx, wy, wz, D, s, t);
      const double tt = ndot(b, t, t, sh);
      if (tt == 0.0) {
        for (int c = threadIdx.x; c < b.ncell; c += NT) {
          int i, j, k;
          cell_ijk(b, c, i, j, k);
          const int64_t q = gq(b, i, j, k);
          x[q] += alpha * p[q];
        }
        __syncthreads();
        break;
      }
      omega = ndot(b, t, s, sh) / tt;
      for (int c = threadIdx.x; c < b.ncell; c += NT) {
        int i, j, k;
        cell_ijk(b, c, i, j, k);
        const int64_t q = gq(b, i, j, k);
        x[q] += alpha * p[q] + omega * s[q];
        r[q] = s[q] - omega * t[q];
      }
      __syncthreads();
      if (nnorm(b, r, sh) <= tol * r0) break;
      rho_old = rho;
    }
    if (it > maxit) it = maxit;
  }
  double shift = 0.0;
  if (singular) shift = nvsum(b, x, sh) / (double)b.ncell;
  for (int c = threadIdx.x; c < b.ncell; c += NT) {
    int i, j, k;
    cell_ijk(b, c, i, j, k);
    xout[c] = x[gq(b, i, j, k)] - shift;
  }
  if (threadIdx.x == 0 && iters) *iters = it;
}

// device address of the scratch, looked up once per device (with that device current);
// atomic so that host threads making their first call on a device at the same time are
// safe (each stores the same address)
constexpr int MAX_DEVICES = 64;
std::atomic<double*> g_scratch_ptr[MAX_DEVICES];

}  // namespace
}  // namespace gmg

namespace gmg {
void set_thread_error(const std::string& msg);
}

extern "C" gmg_status gmg_box_bicgstab_noalloc(void* stream, int nx, int ny, int nz, const int bc_lo[3],
                                               const int bc_hi[3], int singular, const double* wx, const double* wy,
                                               const double* wz, const double* diag, const double* rhs, double* x,
                                               int maxit, double tol, int* iters) {
  using namespace gmg;
  if (nx < 1 || ny < 1 || nz < 1 || !bc_lo || !bc_hi || !wx || !wy || !wz || !diag || !rhs || !x || maxit < 1 ||
      !(tol > 0.0)) {
    set_thread_error("gmg_box_bicgstab_noalloc: invalid arguments");
    return GMG_ERR_BAD_INPUT;
  }
  // edges beyond the limit are refused one by one first, so the product below is formed in
  // 64 bits from small factors (no overflow whatever the edges)
  const int64_t ghosted = (nx > NOALLOC_MAX_ELEMS || ny > NOALLOC_MAX_ELEMS || nz > NOALLOC_MAX_ELEMS)
                              ? (int64_t)NOALLOC_MAX_ELEMS + 1
                              : ((int64_t)nx + 2) * ((int64_t)ny + 2) * ((int64_t)nz + 2);
  if (ghosted > NOALLOC_MAX_ELEMS) {
    set_thread_error("gmg_box_bicgstab_noalloc: (nx+2)(ny+2)(nz+2) = " + std::to_string(ghosted) +
                     " exceeds the static scratch limit of " + std::to_string(NOALLOC_MAX_ELEMS) + " elements");
    return GMG_ERR_BAD_INPUT;
  }
  NBox b{};
  b.nx = nx; b.ny = ny; b.nz = nz;
  for (int d = 0; d < 3; ++d) {
    const bool pl = bc_lo[d] == GMG_BC_PERIODIC, ph = bc_hi[d] == GMG_BC_PERIODIC;
    if (pl != ph || bc_lo[d] < GMG_BC_PERIODIC || bc_lo[d] > GMG_BC_NEUMANN || bc_hi[d] < GMG_BC_PERIODIC ||
        bc_hi[d] > GMG_BC_NEUMANN) {
      set_thread_error("gmg_box_bicgstab_noalloc: bad boundary conditions");
      return GMG_ERR_BAD_INPUT;
    }
    b.per[d] = pl ? 1 : 0;
    b.wsign[d][0] = bc_lo[d] == GMG_BC_NEUMANN ? 1.0 : -1.0;
    b.wsign[d][1] = bc_hi[d] == GMG_BC_NEUMANN ? 1.0 : -1.0;
  }
  b.ncell = nx * ny * nz;
  b.sx = nx + 2;
  b.sy = (int64_t)(nx + 2) * (ny + 2);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
    set_thread_error(std::string("gmg_box_bicgstab_noalloc: cudaGetDevice: ") + cudaGetErrorString(e));
    return GMG_ERR_CUDA;
  }
  double* scratch = g_scratch_ptr[dev].load(std::memory_order_acquire);
  if (!scratch) {
    // first call on this device: resolve the scratch array's device address
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess || !ptr) {
      set_thread_error(std::string("gmg_box_bicgstab_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      return GMG_ERR_CUDA;
    }
    scratch = (double*)ptr;
    g_scratch_ptr[dev].store(scratch, std::memory_order_release);
  }
  k_box_bicgstab_noalloc<<<1, NT, 0, (cudaStream_t)stream>>>(b, wx, wy, wz, diag, rhs, x, scratch,
                                                              NOALLOC_MAX_ELEMS, singular ? 1 : 0, maxit, tol, iters);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_thread_error(std::string("gmg_box_bicgstab_noalloc: launch: ") + cudaGetErrorString(e));
    return GMG_ERR_CUDA;
  }
  return GMG_OK;
}
