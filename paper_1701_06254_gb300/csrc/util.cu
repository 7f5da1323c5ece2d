// Utilities: error text, launch counter, scans, deterministic reductions.
#include "common.cuh"
#include <cstdarg>
#include <cmath>
#include <cstdio>

static thread_local char g_err[1024] = "";
std::atomic<unsigned long long> rs_launches{0};

void rs_set_error(const char *fmt, ...) {
  va_list ap; va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}
extern "C" const char *sim_last_error(void) { return g_err; }
extern "C" long long sim_launch_count(void) { return (long long)rs_launches.load(); }

// ------------------------------------------------------------------ scan --
#define SCAN_BS 256
#define SCAN_IT 4
#define SCAN_CHUNK (SCAN_BS * SCAN_IT)

__device__ __forceinline__ int block_excl_scan(int v, int *sh, int *total) {
  // sh: SCAN_BS/32 ints
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) { int y = __shfl_up_sync(0xffffffffu, x, o); if (lane >= o) x += y; }
  if (lane == 31) sh[wid] = x;
  __syncthreads();
  if (wid == 0) {
    int w = lane < SCAN_BS / 32 ? sh[lane] : 0, z = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) { int y = __shfl_up_sync(0xffffffffu, z, o); if (lane >= o) z += y; }
    if (lane < SCAN_BS / 32) sh[lane] = z - w;
    if (lane == SCAN_BS / 32 - 1) *total = z;
  }
  __syncthreads();
  int r = x - v + sh[wid];
  __syncthreads();
  return r;
}

__global__ void k_scan_partials(const int *in, int n, int *part) {
  __shared__ int sh[SCAN_BS / 32]; __shared__ int tot;
  int base = blockIdx.x * SCAN_CHUNK + threadIdx.x * SCAN_IT, s = 0;
  for (int k = 0; k < SCAN_IT; k++) if (base + k < n) s += in[base + k];
  block_excl_scan(s, sh, &tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}
// tail: where the total goes besides part[nblk] (out + n for a row-pointer
// array, a device counter, or nullptr); tot2 a second copy (or nullptr).
// Each block adds up the partial sums of the blocks before it (at most a few
// thousand integers, read from L2) instead of waiting for a separate scan of
// the partials; the last block writes the total.
__global__ void k_scan_final(const int *in, int *out, int n, int *part, int nblk, int *tail, int *tot2) {
  __shared__ int sh[SCAN_BS / 32]; __shared__ int tot, off;
  int o = 0;
  for (int k = threadIdx.x; k < (int)blockIdx.x; k += SCAN_BS) o += part[k];
  block_excl_scan(o, sh, &off);                     // off = sum of part[0 .. blockIdx.x - 1]
  int base = blockIdx.x * SCAN_CHUNK + threadIdx.x * SCAN_IT;
  int v[SCAN_IT], s = 0;
  for (int k = 0; k < SCAN_IT; k++) { v[k] = (base + k < n) ? in[base + k] : 0; s += v[k]; }
  int e = block_excl_scan(s, sh, &tot) + off;
  for (int k = 0; k < SCAN_IT; k++) if (base + k < n) { out[base + k] = e; e += v[k]; }
  if (blockIdx.x == nblk - 1 && threadIdx.x == 0) {
    const int t = off + tot;
    part[nblk] = t;
    if (tail) *tail = t;
    if (tot2) *tot2 = t;
  }
}

int rs_scan(const int *in, int *out, int n, cudaStream_t s) {
  if (n <= 0) return 0;
  int nblk = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
  static thread_local dbuf<int> part;
  part.ensure(nblk + 1);
  k_scan_partials<<<nblk, SCAN_BS, 0, s>>>(in, n, part.p);
  k_scan_final<<<nblk, SCAN_BS, 0, s>>>(in, out, n, part.p, nblk, nullptr, nullptr);
  RS_LAUNCHED(2);
  RS_CHECK_LAUNCH();
  int tot = 0;
  RS_CUDA(cudaMemcpyAsync(&tot, part.p + nblk, sizeof(int), cudaMemcpyDeviceToHost, s));
  RS_CUDA(cudaStreamSynchronize(s));
  return tot;
}

__global__ void k_scan_empty(int *tail, int *tot2) {
  if (tail) *tail = 0;
  if (tot2) *tot2 = 0;
}
// one block over the whole array, chunk after chunk (short arrays: one
// launch instead of three)
__global__ void k_scan_one(const int *in, int *out, int n, int *tail, int *tot2) {
  __shared__ int sh[SCAN_BS / 32]; __shared__ int tot;
  int carry = 0;
  for (int c0 = 0; c0 < n; c0 += SCAN_CHUNK) {
    int base = c0 + threadIdx.x * SCAN_IT;
    int v[SCAN_IT], s = 0;
    for (int k = 0; k < SCAN_IT; k++) { v[k] = (base + k < n) ? in[base + k] : 0; s += v[k]; }
    int e = block_excl_scan(s, sh, &tot) + carry;
    for (int k = 0; k < SCAN_IT; k++) if (base + k < n) { out[base + k] = e; e += v[k]; }
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (tail) *tail = carry;
    if (tot2) *tot2 = carry;
  }
}
void rs_scan_dev(const int *in, int *out, int n, int *tail, int *tot2, cudaStream_t s) {
  if (n <= 0) {
    k_scan_empty<<<1, 1, 0, s>>>(tail, tot2);
    RS_LAUNCHED(1);
    return;
  }
  if (n <= 8 * SCAN_CHUNK) {
    k_scan_one<<<1, SCAN_BS, 0, s>>>(in, out, n, tail, tot2);
    RS_LAUNCHED(1);
    RS_CHECK_LAUNCH();
    return;
  }
  int nblk = (n + SCAN_CHUNK - 1) / SCAN_CHUNK;
  static thread_local dbuf<int> part;
  part.ensure(nblk + 1);
  k_scan_partials<<<nblk, SCAN_BS, 0, s>>>(in, n, part.p);
  k_scan_final<<<nblk, SCAN_BS, 0, s>>>(in, out, n, part.p, nblk, tail, tot2);
  RS_LAUNCHED(2);
  RS_CHECK_LAUNCH();
}

// ------------------------------------------------------------ reductions --
__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__global__ void k_dot_partials(const double *x, const double *y, int n, double *part) {
  __shared__ double sh[32];
  double s = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) s += x[i] * y[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < blockDim.x / 32 ? sh[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) part[blockIdx.x] = t;
  }
}
__global__ void k_sum_partials(const double *part, int m, double *out) {
  __shared__ double sh[32];
  double s = 0;
  for (int i = threadIdx.x; i < m; i += blockDim.x) s += part[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double t = threadIdx.x < blockDim.x / 32 ? sh[threadIdx.x] : 0.0;
    t = warp_sum(t);
    if (threadIdx.x == 0) *out = t;
  }
}
static int dot_blocks(int n) { int b = (n + 4095) / 4096; return b < 1 ? 1 : (b > 1024 ? 1024 : b); }

void rs_dot_partials(const double *x, const double *y, int n, double *partials, int nblk, cudaStream_t s) {
  k_dot_partials<<<nblk, 256, 0, s>>>(x, y, n, partials);
  RS_LAUNCHED(1);
}
double rs_norm2(const double *x, int n, cudaStream_t s) {
  static thread_local dbuf<double> part;
  int nb = dot_blocks(n);
  part.ensure(nb + 1);
  k_dot_partials<<<nb, 256, 0, s>>>(x, x, n, part.p);
  k_sum_partials<<<1, 256, 0, s>>>(part.p, nb, part.p + nb);
  RS_LAUNCHED(2);
  RS_CHECK_LAUNCH();
  double r;
  RS_CUDA(cudaMemcpyAsync(&r, part.p + nb, sizeof(double), cudaMemcpyDeviceToHost, s));
  RS_CUDA(cudaStreamSynchronize(s));
  return sqrt(r);
}

// out[k] = x[k] . y[k] for k < m (m <= 16), one synchronisation for all
void rs_dots(const double *const *x, const double *const *y, int m, int n, double *out, cudaStream_t s) {
  static thread_local dbuf<double> part;
  int nb = dot_blocks(n);
  part.ensure((size_t)(nb + 1) * m);
  for (int k = 0; k < m; k++) {
    double *pk = part.p + (size_t)k * (nb + 1);
    k_dot_partials<<<nb, 256, 0, s>>>(x[k], y[k], n, pk);
    k_sum_partials<<<1, 256, 0, s>>>(pk, nb, pk + nb);
  }
  RS_LAUNCHED(2 * m);
  RS_CHECK_LAUNCH();
  std::vector<double> h = d2h(part.p, (size_t)(nb + 1) * m, s);
  for (int k = 0; k < m; k++) out[k] = h[(size_t)k * (nb + 1) + nb];
}

template <class T> __global__ void k_fill(T *p, T v, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}
static unsigned gs(size_t n) { size_t g = (n + 255) / 256; return (unsigned)(g < 1 ? 1 : (g > 4096 ? 4096 : g)); }
void rs_fill_i(int *p, int v, size_t n, cudaStream_t s) { if (n) { k_fill<<<gs(n), 256, 0, s>>>(p, v, n); RS_LAUNCHED(1); } }
void rs_fill_d(double *p, double v, size_t n, cudaStream_t s) { if (n) { k_fill<<<gs(n), 256, 0, s>>>(p, v, n); RS_LAUNCHED(1); } }
void rs_fill_f(float *p, float v, size_t n, cudaStream_t s) { if (n) { k_fill<<<gs(n), 256, 0, s>>>(p, v, n); RS_LAUNCHED(1); } }
__global__ void k_d2f(const double *a, float *b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) b[i] = (float)a[i];
}
void rs_cast_d2f(const double *a, float *b, size_t n, cudaStream_t s) { if (n) { k_d2f<<<gs(n), 256, 0, s>>>(a, b, n); RS_LAUNCHED(1); } }

// The option values that select a method or bound a loop, checked on the
// host before any device work: nullptr when all are valid, else a message
// naming the first bad one.  restart, max_lin and the tile sizes select
// their defaults when <= 0 (see rs_opts_from) and are not checked here.
const char *rs_opts_invalid(const sim_options *o) {
  if (o->precision < SIM_PREC_FP64 || o->precision > SIM_PREC_MIXED_BF16) return "unknown precision";
  if (o->decoupling < SIM_DEC_NONE || o->decoupling > SIM_DEC_QI) return "unknown decoupling";
  if (o->reorder != 0 && o->reorder != 1) return "reorder must be 0 or 1";
  if (o->newton != SIM_NEWTON_STANDARD && o->newton != SIM_NEWTON_INEXACT) return "unknown Newton variant";
  if (!(o->newton_tol >= 0.0 && o->newton_tol < HUGE_VAL)) return "newton_tol must be finite and >= 0";
  if (!(o->lin_tol >= 0.0 && o->lin_tol < HUGE_VAL)) return "lin_tol must be finite and >= 0";
  if (!(o->amg_theta >= 0.0 && o->amg_theta <= 1.0)) return "amg_theta must lie in [0, 1]";
  if (o->max_newton < 0 || o->max_cuts < 0 || o->amg_coarse_max < 0) return "negative iteration or size limit";
  if (o->krylov != SIM_KRYLOV_FGMRES && o->krylov != SIM_KRYLOV_BICGSTAB) return "unknown Krylov method";
  if (o->overlap != 1 && o->overlap != 2) return "RAS overlap must be 1 or 2";
  if (o->interp != SIM_INTERP_DIRECT && o->interp != SIM_INTERP_EXTI) return "unknown AMG interpolation";
  return nullptr;
}

rs_opts rs_opts_from(const sim_options *o) {
  rs_opts r;
  r.precision = o->precision; r.decoupling = o->decoupling; r.reorder = o->reorder; r.newton = o->newton;
  r.newton_tol = o->newton_tol; r.lin_tol = o->lin_tol; r.max_newton = o->max_newton;
  r.restart = o->restart > 0 ? o->restart : 50; r.max_lin = o->max_lin > 0 ? o->max_lin : 100;
  r.tile_x = o->tile_x > 0 ? o->tile_x : 4; r.tile_y = o->tile_y > 0 ? o->tile_y : 4;
  r.theta = o->amg_theta; r.max_levels = o->amg_max_levels < 1 ? 1 : (o->amg_max_levels > 32 ? 32 : o->amg_max_levels);
  r.coarse_max = o->amg_coarse_max; r.seed = o->seed; r.max_cuts = o->max_cuts; r.dt = o->dt;
  r.sat_chop = o->sat_chop > 0.0 ? o->sat_chop : 0.0;
  r.krylov = o->krylov; r.overlap = o->overlap; r.interp = o->interp; r.fp64_basis = o->fp64_basis != 0;
  return r;
}

extern "C" void sim_default_options(sim_options *o) {
  o->precision = SIM_PREC_FP64; o->decoupling = SIM_DEC_ABF; o->reorder = 1; o->newton = SIM_NEWTON_STANDARD;
  o->newton_tol = 1e-8; o->lin_tol = 1e-8; o->max_newton = 20; o->restart = 50; o->max_lin = 100;
  o->tile_x = 4; o->tile_y = 4; o->amg_theta = 0.25; o->amg_max_levels = 25; o->amg_coarse_max = 128;
  o->seed = 0x5EED; o->max_cuts = 6; o->dt = 1.0; o->cuda_stream = nullptr; o->sat_chop = 0.0;
  o->krylov = SIM_KRYLOV_FGMRES; o->overlap = 1; o->interp = SIM_INTERP_DIRECT; o->fp64_basis = 0;
}
