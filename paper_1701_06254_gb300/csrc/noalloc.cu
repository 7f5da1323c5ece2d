// ||b - A x||_2 without any allocation: the per-block partial sums live in a
// file-scope device array instead of memory obtained from cudaMalloc.
//
// The array is one per device: every GPU that loads the library holds
// NOALLOC_MAX_BLOCKS doubles (32 KB) until the process exits.  Host code
// cannot take the array's address directly (in host code the symbol names a
// host-side stand-in); the first call on each device looks the device
// address up with cudaGetSymbolAddress and keeps it.
#include "common.cuh"
#include <mutex>

#define NOALLOC_ROWS_PER_BLOCK 4096        // block rows handled by one thread block
#define NOALLOC_MAX_BLOCKS 4096            // scratch capacity: one partial per thread block
#define NOALLOC_MAX_DEVICES 64

static __device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_BLOCKS];

static std::mutex g_noalloc_lock;
static double *g_noalloc_addr[NOALLOC_MAX_DEVICES];   // device address of the array, per device

// device address of the scratch array on the current device, looked up on
// the first call on that device (nullptr and an error text on failure)
static double *noalloc_scratch(int dev) {
  std::lock_guard<std::mutex> guard(g_noalloc_lock);
  if (!g_noalloc_addr[dev]) {
    double *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&p, g_noalloc_partials);
    if (e != cudaSuccess || !p) {
      rs_set_error("sim_ls_residual_norm_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return nullptr;
    }
    g_noalloc_addr[dev] = p;
  }
  return g_noalloc_addr[dev];
}

// partials[blk] = sum over the block's rows of |b_i - (A x)_i|^2; rows are
// taken in a fixed order by each thread, then a fixed tree over the block
__global__ void k_resid_sq_partials(int nb, const int *__restrict__ rp, const int *__restrict__ ci,
                                    const double *__restrict__ val, const double *__restrict__ b,
                                    const double *__restrict__ x, double *partials) {
  __shared__ double sh[256];
  int r0 = blockIdx.x * NOALLOC_ROWS_PER_BLOCK, r1 = min(nb, r0 + NOALLOC_ROWS_PER_BLOCK);
  double acc = 0.0;
  for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
    double a0 = b[2 * (size_t)r], a1 = b[2 * (size_t)r + 1];
    for (int q = rp[r]; q < rp[r + 1]; q++) {
      const double *B = val + 4 * (size_t)q;
      double x0 = x[2 * (size_t)ci[q]], x1 = x[2 * (size_t)ci[q] + 1];
      a0 -= B[0] * x0 + B[1] * x1;
      a1 -= B[2] * x0 + B[3] * x1;
    }
    acc += a0 * a0 + a1 * a1;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

// *out = sqrt(sum of the m partials), one warp, fixed order
__global__ void k_partials_sqrt(int m, const double *partials, double *out) {
  double t = 0.0;
  for (int k = threadIdx.x; k < m; k += 32) t += partials[k];
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
  if (threadIdx.x == 0) *out = sqrt(t);
}

static bool device_pointer(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Error paths return directly (no exception objects): nothing on this
// path allocates, on the device or on the host.
extern "C" sim_status sim_ls_residual_norm_noalloc(sim_ls_t ls, const double *x_dev, double *norm_dev) {
  if (!ls || !x_dev || !norm_dev) {
    rs_set_error("sim_ls_residual_norm_noalloc: NULL argument");
    return SIM_ERR_ARG;
  }
  if (!device_pointer(x_dev) || !device_pointer(norm_dev)) {
    rs_set_error("sim_ls_residual_norm_noalloc: x and norm must be device memory");
    return SIM_ERR_ARG;
  }
  int nblocks = (ls->nb + NOALLOC_ROWS_PER_BLOCK - 1) / NOALLOC_ROWS_PER_BLOCK;
  if (nblocks > NOALLOC_MAX_BLOCKS) {
    rs_set_error("sim_ls_residual_norm_noalloc: %d block rows exceed the limit of %d", ls->nb,
                 NOALLOC_MAX_BLOCKS * NOALLOC_ROWS_PER_BLOCK);
    return SIM_ERR_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= NOALLOC_MAX_DEVICES) {
    rs_set_error("sim_ls_residual_norm_noalloc: no usable current device (%s)", cudaGetErrorString(e));
    return SIM_ERR_CUDA;
  }
  double *scratch = noalloc_scratch(dev);
  if (!scratch) return SIM_ERR_CUDA;
  // every partial the second kernel reads is written by the first one in the
  // same call, so nothing in the scratch array needs clearing between calls
  k_resid_sq_partials<<<nblocks, 256, 0, ls->st>>>(ls->nb, ls->rp.p, ls->ci.p, ls->val.p, ls->b.p, x_dev, scratch);
  k_partials_sqrt<<<1, 32, 0, ls->st>>>(nblocks, scratch, norm_dev);
  RS_LAUNCHED(2);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    rs_set_error("sim_ls_residual_norm_noalloc: launch failed: %s", cudaGetErrorString(e));
    return SIM_ERR_CUDA;
  }
  return SIM_OK;
}
