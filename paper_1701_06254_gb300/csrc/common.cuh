// Internal declarations of the sm_103a CPR-FGMRES library (libresim.so).
// Not part of the public ABI (that is include/resim.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <string>
#include <vector>
#include <atomic>
#include "../../include/resim.h"

#define RS_CDARCY (9.869233e-16 * 1e5 / 1e-3 * 86400.0)   // k[mD] A/L dp[bar]/mu[cP] -> m3/day
#define RS_PA2BAR 1e-5

// ---------------------------------------------------------------- errors --
void rs_set_error(const char *fmt, ...);
struct rs_error {                       // thrown inside the library, caught at the ABI
  sim_status code;
  explicit rs_error(sim_status c) : code(c) {}
};
#define RS_CUDA(call)                                                                 \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      rs_set_error("%s:%d %s: %s", __FILE__, __LINE__, #call, cudaGetErrorString(e_)); \
      throw rs_error(e_ == cudaErrorMemoryAllocation ? SIM_ERR_OOM : SIM_ERR_CUDA);   \
    }                                                                                 \
  } while (0)
#define RS_CHECK_LAUNCH() RS_CUDA(cudaGetLastError())
#define RS_FAIL(code, ...) do { rs_set_error(__VA_ARGS__); throw rs_error(code); } while (0)

extern std::atomic<unsigned long long> rs_launches;     // kernel launches issued (all handles)
#define RS_LAUNCHED(k) (rs_launches += (k))

// ---------------------------------------------------------------- memory --
template <class T> struct dbuf {            // owning device buffer
  T *p = nullptr; size_t n = 0;
  void alloc(size_t m) {
    if (m == n && p) return;
    free();
    if (m) RS_CUDA(cudaMalloc((void **)&p, m * sizeof(T)));
    n = m;
  }
  // grow with a quarter of headroom: sizes that follow the data (AMG levels,
  // SpGEMM scratch) creep up between Newton iterations, and every regrowth is
  // a cudaFree (which waits for the device) and a cudaMalloc
  void ensure(size_t m) { if (m > n) alloc(m + m / 4); }
  void free() { if (p) cudaFree(p); p = nullptr; n = 0; }
  ~dbuf() { free(); }
  dbuf() = default;
  dbuf(const dbuf &) = delete;
  dbuf &operator=(const dbuf &) = delete;
};
template <class T> void h2d(dbuf<T> &d, const T *h, size_t m, cudaStream_t s) {
  d.alloc(m);
  if (m) RS_CUDA(cudaMemcpyAsync(d.p, h, m * sizeof(T), cudaMemcpyDefault, s));
}
template <class T> void h2d(dbuf<T> &d, const std::vector<T> &h, cudaStream_t s) { h2d(d, h.data(), h.size(), s); }
template <class T> std::vector<T> d2h(const T *d, size_t m, cudaStream_t s) {
  std::vector<T> h(m);
  if (m) RS_CUDA(cudaMemcpyAsync(h.data(), d, m * sizeof(T), cudaMemcpyDefault, s));
  RS_CUDA(cudaStreamSynchronize(s));
  return h;
}
inline unsigned grid_for(size_t n, int bs) { size_t g = (n + bs - 1) / bs; return (unsigned)(g ? g : 1); }

// Programmatic dependent launch: a kernel launched with launch_pdl may be
// scheduled while the kernel before it in the stream is still running, so
// its launch latency overlaps that kernel's last wave.  Such a kernel calls
// pdl_wait() before it touches memory: the wait returns once the previous
// kernel has completed and its writes are visible (at once when there is no
// such kernel).  pdl_trigger() lets the next kernel be scheduled early.
// rs_pdl_off (per host thread) makes launch_pdl an ordinary launch: used
// while recording a graph body that cannot hold programmatic edges.
inline thread_local bool rs_pdl_off = false;
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
template <typename... KArgs, typename... Args>
inline void launch_pdl(void (*kern)(KArgs...), unsigned grid, unsigned block, size_t smem, cudaStream_t s,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid); cfg.blockDim = dim3(block); cfg.dynamicSmemBytes = smem; cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at; cfg.numAttrs = rs_pdl_off ? 0 : 1;
  RS_CUDA(cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...));
}

// ------------------------------------------------------- device helpers --
// Arithmetic used where a floating-point value decides an integer (the
// decoupled matrix, the reordering key, AMG strength / PMIS / P / RAP):
// explicit round-to-nearest operations that the compiler may not contract
// into fused multiply-adds, so results match a plain IEEE evaluation in the
// order written.
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ double div_rn(double a, double b) { return __ddiv_rn(a, b); }
// Comparisons of doubles taken on integers: dkey orders finite doubles and
// the infinities as IEEE comparison does (both zeros map to 0; dkey(-x) =
// -dkey(x)), so a comparison decides the same as on the doubles while the
// FP64 pipe (a small fraction of the FP32 rate on this GPU) is kept for
// arithmetic.
__device__ __forceinline__ long long dkey(double x) {
  long long b = __double_as_longlong(x), m = b & 0x7fffffffffffffffLL;
  return b < 0 ? -m : m;
}

// ------------------------------------------------------------ utilities --
// exclusive scan of n int32 values (in may alias out); returns the total
int rs_scan(const int *in, int *out, int n, cudaStream_t s);
// the same without a host wait: the total goes to device memory, at tail
// (e.g. out + n) and tot2 (either may be nullptr); in may alias out when
// tail is not in[n] of a later use.  Stream-ordered, no synchronisation.
void rs_scan_dev(const int *in, int *out, int n, int *tail, int *tot2, cudaStream_t s);
// deterministic reductions (fixed association order for a given n)
void rs_dot_partials(const double *x, const double *y, int n, double *partials, int nblk, cudaStream_t s);
double rs_norm2(const double *x, int n, cudaStream_t s);   // syncs
void rs_dots(const double *const *x, const double *const *y, int m, int n, double *out, cudaStream_t s);  // syncs
void rs_fill_i(int *p, int v, size_t n, cudaStream_t s);
void rs_fill_d(double *p, double v, size_t n, cudaStream_t s);
void rs_fill_f(float *p, float v, size_t n, cudaStream_t s);
void rs_cast_d2f(const double *a, float *b, size_t n, cudaStream_t s);

// --------------------------------------------------------------- options --
struct rs_opts {
  int precision, decoupling, reorder, newton;
  double newton_tol, lin_tol;
  int max_newton, restart, max_lin, tile_x, tile_y;
  double theta;
  int max_levels, coarse_max;
  uint64_t seed;
  int max_cuts;
  double dt, sat_chop;
  int krylov, overlap, interp, fp64_basis;
};
const char *rs_opts_invalid(const sim_options *o);
rs_opts rs_opts_from(const sim_options *o);

// ---------------------------------------------------------------- AMG -----
template <class T> struct csr_dev { int n = 0, m = 0, nnz = 0; dbuf<int> rp, ci; dbuf<T> v; };

struct amg_level {
  csr_dev<double> A;            // FP64 operator (setup)
  csr_dev<double> P, R;         // interpolation / restriction (FP64)
  csr_dev<float> A32, P32, R32; // mixed-precision values (rp, ci unused: the pattern is A's, P's, R's)
  dbuf<double> dinv;            // 1 / l1 diagonal
  dbuf<float> dinv32;
  dbuf<int8_t> cf;
  dbuf<uint8_t> strong;
  dbuf<int> tpos;               // position of (j,i) in row j for each (i,j)
  int nc = 0, rounds = 0;
  int tail_r = -1;               // PMIS rounds on the full grid before the one-block tail (-1: not known yet)
  int nnz_prev = 0;             // nnz(A) of this level at the previous setup (a launch-shape hint)
  dbuf<double> f, x, r, t;      // cycle work vectors (FP64)
  dbuf<float> f32, x32, r32, t32;
};

struct amg_hier {
  int nlev = 0;
  amg_level lev[32];
  int coarse_dense = 1;
  dbuf<double> lu;              // dense LU of the coarsest level
  dbuf<int> piv;
  dbuf<int> flag;               // device counters / error words
  int *hflag = nullptr;         // pinned host copy of flag, read at the setup's few waits
  dbuf<double> dense_a;         // the coarsest operator as a dense matrix (setup scratch)
  dbuf<double> dense_lu;        // its LU factors (setup scratch)
  dbuf<double> dense_rd;        // and the reciprocals of U's diagonal
  dbuf<double> hashw;           // PMIS weights
  dbuf<int8_t> newc;
  dbuf<int> plist;              // PMIS undecided-point lists (two of n)
  // the V-cycle of the current hierarchy as a CUDA graph ([0] FP64, [1] FP32),
  // captured on first use after a setup; the capture stream only records
  cudaGraphExec_t vc_exec[2] = {nullptr, nullptr};
  int vc_launches[2] = {0, 0};
  cudaStream_t cap = nullptr;
  void drop_graphs() {
    for (auto &e : vc_exec) if (e) { cudaGraphExecDestroy(e); e = nullptr; }
  }
  ~amg_hier() { drop_graphs(); if (cap) cudaStreamDestroy(cap); if (hflag) cudaFreeHost(hflag); }
};

void amg_setup(amg_hier &h, const rs_opts &o, cudaStream_t s);   // level 0 A must be filled
template <class T> int amg_vcycle(amg_hier &h, int l, cudaStream_t s);   // f -> x of level l; returns launches
template <class T> void amg_vcycle_graph(amg_hier &h, cudaStream_t s);   // level 0, replayed as one graph

// ---------------------------------------------------------------- RAS -----
struct ras_data {
  int nsub = 0, max_ext = 0, max_nnz = 0;
  // static (host-built at creation): per subdomain, ext rows in natural
  // order (cells ascending then wells ascending)
  dbuf<int> sub_ptr;            // nsub+1 offsets into ext arrays
  dbuf<int> order;              // apply launch order: most L + U levels first
  dbuf<int> ext;                // global row of each ext entry
  dbuf<uint8_t> owned;          // 1 if the ext entry is owned
  dbuf<int> ncell;              // cells among ext entries, per subdomain
  dbuf<int> lrp_ptr;            // nsub+1 offsets into the local-pattern entries
  dbuf<int> lrlen;              // local row length per ext entry
  dbuf<int> lrp;                // local row start per ext entry (natural ext order)
  dbuf<int> lci;                // ext-index column per local entry
  dbuf<int> lsrc;               // BSR block position per local entry
  // per setup
  dbuf<int> perm;               // position -> ext index (per subdomain segment)
  dbuf<int> ipos;               // ext index -> position
  dbuf<int> frp;                // factor row start per position (segment-local offsets)
  dbuf<int> fci;                // factor column (position) per entry
  dbuf<int> fdiag;              // diagonal entry per position
  dbuf<double> fval;            // FP64 factors (4 per entry)
  dbuf<float> fval32;           // FP32 factors
  dbuf<double> dinv;            // inverse U diagonal blocks (4 per row)
  dbuf<float> dinv32;
  dbuf<int> lvl;                // per position: L level, U level
  dbuf<int> lvl_rows;           // rows grouped by L level, then by U level
  dbuf<int> nlev;               // per subdomain: #L levels, #U levels
  dbuf<int> lvl_ptr;            // per subdomain: offsets of the L and U level groups
  int max_lvl_ptr = 0;
  // shared-memory apply: one factor stream per subdomain (see ras.cu)
  bool smem_path = false;
  bool built = false;           // a setup has run (level sets exportable)
  size_t smem_bytes = 0;        // ring + largest local vector
  int m_max = 0;                // most extended rows in a subdomain
  dbuf<long long> blob_off;     // nsub + 1 byte offsets (stream bounds)
  dbuf<unsigned char> blob;     // the streams
  dbuf<int> gidx;               // per subdomain and position: 2 * global row + owned flag
  dbuf<int4> gdesc;             // group descriptors (packing scratch)
};

// ---------------------------------------------------------- linear system --
struct sim_ls_s {
  int nx, ny, nz, n, nw, nb, nnzb;
  rs_opts o;
  cudaStream_t st = nullptr;
  std::vector<int> h_rp, h_ci, h_wc0;
  dbuf<int> rp, ci, dpos;       // pattern, diagonal position per row
  dbuf<double> val, b, key, dmat;
  dbuf<float> val32;
  dbuf<int> app_src;            // BSR positions of the A_pp entries
  ras_data ras;
  amg_hier amg;
  // Krylov
  dbuf<double> V, Z, w, r, y, hbuf, partial;
  dbuf<float> Z32;
  dbuf<double> x64a, x64b;      // CPR work (FP64)
  dbuf<float> x32a, x32b, x32c; // CPR work (FP32)
  double *hpin = nullptr;       // pinned host scalars: 4 per Arnoldi step (estimate, h_{j+1,j}, second pass)
  // one Arnoldi step as a CUDA graph (recorded after each setup)
  int graph_mode = 1;           // 0 separate launches, 1 a graph per Arnoldi step, 2 a device-side loop
  cudaGraphExec_t it_exec = nullptr;
  cudaGraphExec_t loop_exec = nullptr;   // the Arnoldi steps of a cycle in a graph WHILE node
  dbuf<double> loopd;           // loop parameters and results: threshold, step cap, steps done, non-finite flag
  int loop_state = 0;           // device-side loop: 0 not built, 1 built with programmatic edges, 2 without, -1 unavailable
  int last_mode = -1;           // launch mode the last FGMRES solve used (0, 1, 2)
  long long it_launches = 0;
  const void *it_sig[10] = {};   // buffers, restart length and precision it was recorded with
  cudaStream_t cap = nullptr;
  bool capturing = false;
  // the RAS setup runs on a stream of its own beside the AMG setup (both
  // need only the decoupled matrix): fork after the decoupling, join after both
  cudaStream_t st2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  dbuf<int> jd;                 // the step index the graph's kernels read
  dbuf<double> vcur, zcur64;
  dbuf<float> zcur32, vcur32;
  dbuf<float> w2, isp;          // double-float w planes; split 1 / h_{j+1,j}
  dbuf<int> ticket;             // last-block ticket of the Gram-Schmidt sweeps (zero between launches)
  dbuf<float> vallo;            // lo plane of the decoupled matrix (hi: val32)
  dbuf<double> bcg;             // BiCGSTAB vectors: rh, p, v, s, t, ph, sh, x (2 nb each)
  dbuf<float> bcg32;            // mixed precision: the FP32 preconditioned vector
  dbuf<float> cprt32;           // CPR: the first RAS stage's output (FP32)
  // timer brackets recorded inside the graph (event nodes): pairs of events
  // and the family of each pair, read back after every replay
  std::vector<cudaEvent_t> gev;
  std::vector<int> gev_fam;
  void drop_graph() {
    if (it_exec) { cudaGraphExecDestroy(it_exec); it_exec = nullptr; }
    if (loop_exec) { cudaGraphExecDestroy(loop_exec); loop_exec = nullptr; }
    if (loop_state > 0) loop_state = 0;
    for (auto e : gev) cudaEventDestroy(e);
    gev.clear(); gev_fam.clear();
  }
  void graph_timers();          // after a replay has completed
  int *errw = nullptr, *errw_dev = nullptr;   // device error word (host-mapped)
  bool have_setup = false;
  double *noalloc_scratch = nullptr;   // device address of the allocation-free norm's array (noalloc.cu)
  // timing: events in pairs, the family of each pair in ev_fam
  unsigned timer_mask = 0;
  int ev_open = 0;               // timer brackets not yet closed
  long long timer_launches[SIM_T_NFAMILIES] = {0};
  double timer_ms[SIM_T_NFAMILIES] = {0};
  std::vector<cudaEvent_t> ev;
  std::vector<int> ev_fam;
  int ev_used = 0;
  void timer_flush();
  ~sim_ls_s();
};

struct rs_timed {                       // brackets launches of one kernel family
  sim_ls_s *ls; bool on; int fam; int slot = 0; bool in_graph = false;
  rs_timed(sim_ls_s *l, int which);
  ~rs_timed() { stop(); }
  void stop();                          // end the bracket early (idempotent)
};

void ls_init(sim_ls_s *ls, int nx, int ny, int nz, int nw, const int *rp, const int *ci,
             const int *well_cell0, const rs_opts &o, cudaStream_t st);
void ls_setup(sim_ls_s *ls);
// solution in ls->y; x0: ls->y holds the initial guess (else zero)
int ls_solve(sim_ls_s *ls, double tol, int *its, double *relres, bool x0 = false);
void ls_cpr(sim_ls_s *ls, const double *v, double *z64, float *z32);
void ls_cpr32(sim_ls_s *ls, const float *v, float *z);
void ls_spmv64(sim_ls_s *ls, const double *x, double *y);
void ls_spmv64_untimed(sim_ls_s *ls, const double *x, double *y);
double ls_residual_norm(sim_ls_s *ls, const double *x_dev);
template <class T, class Tin> void ls_ras_apply(sim_ls_s *ls, const Tin *f, T *x, bool accumulate);
void ras_build_static(sim_ls_s *ls);
void ras_setup(sim_ls_s *ls);

// SpMV kernels (block 2x2, values Tv, vectors Tx in / Ty out)
template <class Tv, class Tx, class Ty>
void bsr_spmv(const int *rp, const int *ci, const Tv *val, const Tx *x, Ty *y, const Ty *f, int nb, cudaStream_t s);
template <class T>
void csr_spmv(const int *rp, const int *ci, const T *v, const T *x, T *y, int n, cudaStream_t s);

// simulator internals used by the ensemble driver (batch.cu)
void sim_dims(sim_t h, int *n, int *n_wells);
void sim_put_stats(sim_t h, const sim_stats *st);
int sim_history(sim_t h, double *y, double *sc, int have, bool save);   // y: 2 vectors of 2 nb

// learned warm start (nn.cu)
struct sim_ws_s;
void ws_rms2(int n, const double *v, double *out, cudaStream_t s);
void ws_predict(sim_ws_s *w, int nx, int ny, int nz, int nb, const double *b, const double *kx, const double *sw,
                const double *yp, const double *sc, double *y, cudaStream_t s);
void ws_record(sim_ws_s *w, int nx, int ny, int nz, const double *b, const double *kx, const double *sw,
               const double *yp, const double *sc, const double *y, cudaStream_t s);
