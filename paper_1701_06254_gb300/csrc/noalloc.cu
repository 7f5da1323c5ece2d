// ||b - A x||_2 without any allocation: the per-block partial sums live in a
// file-scope device array instead of memory obtained from cudaMalloc.
//
// The array is one per device: every GPU that loads the library holds
// NOALLOC_MAX_BLOCKS doubles (32 KB) until the process exits.  Host code
// cannot take the array's address directly (in host code the symbol names a
// host-side stand-in); the first call on a handle looks the device address
// up with cudaGetSymbolAddress, with the handle's device current, and keeps
// it in the handle.  A device reset (cudaDeviceReset) invalidates every
// handle on that device together with the address it kept; handles created
// afterwards look the address up again.
#include "common.cuh"
#include "noalloc_limit.h"

static __device__ __align__(256) double g_noalloc_partials[NOALLOC_MAX_BLOCKS];

// device address of the scratch array for this handle's device (the
// current one), looked up on the handle's first call; nullptr and an error
// text on failure
static double *noalloc_scratch(sim_ls_s *ls) {
  if (!ls->noalloc_scratch) {
    double *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress((void **)&p, g_noalloc_partials);
    if (e != cudaSuccess || !p) {
      rs_set_error("sim_ls_residual_norm_noalloc: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
      return nullptr;
    }
    ls->noalloc_scratch = p;
  }
  return ls->noalloc_scratch;
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

// the device that holds p (device or managed memory), or -1
static int device_of(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return -1; }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) ? a.device : -1;
}

// Error paths return directly (no exception objects): nothing on this
// path allocates, on the device or on the host.
extern "C" sim_status sim_ls_residual_norm_noalloc(sim_ls_t ls, const double *x_dev, double *norm_dev) {
  if (!ls || !x_dev || !norm_dev) {
    rs_set_error("sim_ls_residual_norm_noalloc: NULL argument");
    return SIM_ERR_ARG;
  }
  long long nblocks = rs_noalloc_blocks(ls->nb);
  if (nblocks < 0) {
    rs_set_error("sim_ls_residual_norm_noalloc: %d block rows exceed the limit of %d", ls->nb,
                 NOALLOC_MAX_BLOCKS * NOALLOC_ROWS_PER_BLOCK);
    return SIM_ERR_ARG;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0) {
    rs_set_error("sim_ls_residual_norm_noalloc: no usable current device (%s)", cudaGetErrorString(e));
    return SIM_ERR_CUDA;
  }
  // the handle's matrix, x and norm must all live on the current device:
  // a kernel launched here must not touch another GPU's memory
  int dh = device_of(ls->rp.p), dx = device_of(x_dev), dn = device_of(norm_dev);
  if (dx < 0 || dn < 0) {
    rs_set_error("sim_ls_residual_norm_noalloc: x and norm must be device memory");
    return SIM_ERR_ARG;
  }
  if (dh != dev || dx != dev || dn != dev) {
    rs_set_error("sim_ls_residual_norm_noalloc: the handle (device %d), x (device %d) and norm (device %d) "
                 "must be on the current device %d", dh, dx, dn, dev);
    return SIM_ERR_ARG;
  }
  double *scratch = noalloc_scratch(ls);
  if (!scratch) return SIM_ERR_CUDA;
  // every partial the second kernel reads is written by the first one in the
  // same call, so nothing in the scratch array needs clearing between calls
  k_resid_sq_partials<<<(unsigned)nblocks, 256, 0, ls->st>>>(ls->nb, ls->rp.p, ls->ci.p, ls->val.p, ls->b.p, x_dev, scratch);
  k_partials_sqrt<<<1, 32, 0, ls->st>>>((int)nblocks, scratch, norm_dev);
  RS_LAUNCHED(2);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    rs_set_error("sim_ls_residual_norm_noalloc: launch failed: %s", cudaGetErrorString(e));
    return SIM_ERR_CUDA;
  }
  return SIM_OK;
}
