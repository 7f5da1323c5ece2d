// The Newton linear system and its solver (arXiv 1701.06254):
//   decoupling D^{-1} A x = D^{-1} b, eq. (29), with the ABF or Quasi-IMPES
//   operator (Sec. "Matrix decoupling strategy");
//   CPR-FPF, Algorithm 2, with the restriction / prolongation of eqs. (34)-(35);
//   restarted flexible GMRES, right preconditioned, stopping per eq. (24).
// Storage: 2x2 blocks with cell-interleaved unknowns (p, s_w), which is the
// field-split system of eqs. (20)-(23) under a fixed permutation; each well
// row is padded to a 2x2 block with a dummy unknown whose equation is 1*x = 0.
#include "common.cuh"
#define ORTHO_MAXV 64            // FGMRES restart length limit (m + 1 basis vectors)
#include <algorithm>
#include <cmath>
#include <cstring>

// ------------------------------------------------------------ timers -----
rs_timed::rs_timed(sim_ls_s *l, int which) : ls(l), on(which > 0 && (l->timer_mask >> which) & 1u), fam(which) {
  if (!on) return;
  if (ls->capturing) {          // recorded into the Arnoldi-step graph as event nodes
    in_graph = true;
    cudaEvent_t a, b;
    RS_CUDA(cudaEventCreate(&a));
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); RS_CUDA(cudaGetLastError()); }
    slot = (int)ls->gev.size();
    ls->gev.push_back(a); ls->gev.push_back(b); ls->gev_fam.push_back(fam);
    RS_CUDA(cudaEventRecordWithFlags(a, ls->st, cudaEventRecordExternal));
    return;
  }
  // each bracket takes its own pair of events at once, so brackets may nest;
  // the pool only grows (it is read back when the solve's work is complete)
  if (ls->ev_used + 2 > (int)ls->ev.size()) {
    for (int k = 0; k < 64; k++) { cudaEvent_t e; RS_CUDA(cudaEventCreate(&e)); ls->ev.push_back(e); ls->ev_fam.push_back(0); }
  }
  slot = ls->ev_used;
  ls->ev_used += 2;
  ls->ev_open++;
  ls->ev_fam[slot] = fam;
  RS_CUDA(cudaEventRecord(ls->ev[slot], ls->st));
}
void rs_timed::stop() {
  if (!on) return;
  on = false;
  if (in_graph) { cudaEventRecordWithFlags(ls->gev[slot + 1], ls->st, cudaEventRecordExternal); return; }
  cudaEventRecord(ls->ev[slot + 1], ls->st);
  ls->ev_open--;
  ls->timer_launches[fam]++;
}
void sim_ls_s::timer_flush() {
  if (!ev_used || ev_open) return;          // only when every bracket is closed
  cudaStreamSynchronize(st);
  for (int k = 0; k < ev_used; k += 2) {
    float ms = 0; cudaEventElapsedTime(&ms, ev[k], ev[k + 1]);
    timer_ms[ev_fam[k]] += ms;
  }
  ev_used = 0;
}
void sim_ls_s::graph_timers() {
  for (size_t k = 0; k + 1 < gev.size(); k += 2) {
    float ms = 0;
    RS_CUDA(cudaEventElapsedTime(&ms, gev[k], gev[k + 1]));
    timer_ms[gev_fam[k / 2]] += ms;
    timer_launches[gev_fam[k / 2]]++;
  }
}
sim_ls_s::~sim_ls_s() {
  drop_graph();
  if (cap) cudaStreamDestroy(cap);
  if (st2) cudaStreamDestroy(st2);
  if (ev_fork) cudaEventDestroy(ev_fork);
  if (ev_join) cudaEventDestroy(ev_join);
  for (auto e : ev) cudaEventDestroy(e);
  if (hpin) cudaFreeHost(hpin);
  if (errw) cudaFreeHost(errw);
}

// ---------------------------------------------------------- decoupling ---
// ABF: every cell row is multiplied by the inverse of its 2x2 diagonal
// block, [[d, -b], [-c, a]] / (ad - bc); each entry is formed by separate
// round-to-nearest multiplications, additions and divisions in the order
// written (so the decoupled matrix is the IEEE evaluation of this formula).
__global__ void k_abf(int n, int nb, const int *rp, const int *dpos, double *val, double *b, double *dmat, float *val32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  double *D = dmat + 4 * (size_t)i;
  if (i >= n) {
    D[0] = 1; D[1] = 0; D[2] = 0; D[3] = 1;
    if (val32) for (int q = rp[i]; q < rp[i + 1]; q++) for (int e = 0; e < 4; e++) val32[4 * (size_t)q + e] = (float)val[4 * (size_t)q + e];
    return;
  }
  const double *M = val + 4 * (size_t)dpos[i];
  double a = M[0], bb = M[1], c = M[2], d = M[3];
  D[0] = a; D[1] = bb; D[2] = c; D[3] = d;
  double det = sub_rn(mul_rn(a, d), mul_rn(bb, c));
  double i00 = div_rn(d, det), i01 = div_rn(-bb, det), i10 = div_rn(-c, det), i11 = div_rn(a, det);
  for (int q = rp[i]; q < rp[i + 1]; q++) {
    double *B = val + 4 * (size_t)q;
    double b00 = B[0], b01 = B[1], b10 = B[2], b11 = B[3];
    double n0 = add_rn(mul_rn(i00, b00), mul_rn(i01, b10));
    double n1 = add_rn(mul_rn(i00, b01), mul_rn(i01, b11));
    double n2 = add_rn(mul_rn(i10, b00), mul_rn(i11, b10));
    double n3 = add_rn(mul_rn(i10, b01), mul_rn(i11, b11));
    B[0] = n0; B[1] = n1; B[2] = n2; B[3] = n3;
    if (val32) { float4 f4 = make_float4((float)n0, (float)n1, (float)n2, (float)n3); reinterpret_cast<float4 *>(val32)[q] = f4; }
  }
  double r0 = b[2 * (size_t)i], r1 = b[2 * (size_t)i + 1];
  b[2 * (size_t)i] = add_rn(mul_rn(i00, r0), mul_rn(i01, r1));
  b[2 * (size_t)i + 1] = add_rn(mul_rn(i10, r0), mul_rn(i11, r1));
}

// Quasi-IMPES: pressure row -= Diag(A_ps) Diag(A_ss)^{-1} * saturation row.
__global__ void k_qi(int n, int nb, const int *rp, const int *dpos, double *val, double *b, double *dmat, float *val32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  double *D = dmat + 4 * (size_t)i;
  D[0] = 1; D[1] = 0; D[2] = 0; D[3] = 1;
  if (i < n) {
    const double *M = val + 4 * (size_t)dpos[i];
    double ratio = div_rn(M[1], M[3]);
    D[1] = ratio;
    for (int q = rp[i]; q < rp[i + 1]; q++) {
      double *B = val + 4 * (size_t)q;
      B[0] = sub_rn(B[0], mul_rn(ratio, B[2]));
      B[1] = sub_rn(B[1], mul_rn(ratio, B[3]));
    }
    b[2 * (size_t)i] = sub_rn(b[2 * (size_t)i], mul_rn(ratio, b[2 * (size_t)i + 1]));
  }
  if (val32) for (int q = rp[i]; q < rp[i + 1]; q++) for (int e = 0; e < 4; e++) val32[4 * (size_t)q + e] = (float)val[4 * (size_t)q + e];
}

// The same Quasi-IMPES decoupling with the FP32 copy and the double-float
// lo plane written in the same pass: one warp per 32 block rows reads its
// contiguous range of blocks coalesced (lane t takes block q0 + t + 32k;
// its row by a binary search over the warp's row pointers held in lanes),
// updates the pressure row of each cell block with the row's ratio (the same
// round-to-nearest operations as k_qi) and writes val, val32 and lo.  Well
// rows keep their blocks; D and b per row as in k_qi.
__global__ void __launch_bounds__(256) k_qi_fused(int n, int nb, const int *__restrict__ rp,
                                                  const int *__restrict__ dpos, double *__restrict__ val,
                                                  double *__restrict__ b, double *__restrict__ dmat,
                                                  float *__restrict__ val32, float *__restrict__ lo) {
  int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int r0 = (blockIdx.x * (blockDim.x >> 5) + wid) * 32;
  if (r0 >= nb) return;
  int r = r0 + lane, rend = min(r0 + 32, nb);
  int myq0 = r < nb ? rp[r] : rp[rend];
  double ratio = 0.0;
  if (r < n) {
    const double *M = val + 4 * (size_t)dpos[r];
    ratio = div_rn(M[1], M[3]);
  }
  if (r < nb) {
    double *D = dmat + 4 * (size_t)r;
    D[0] = 1; D[1] = r < n ? ratio : 0.0; D[2] = 0; D[3] = 1;
    if (r < n) b[2 * (size_t)r] = sub_rn(b[2 * (size_t)r], mul_rn(ratio, b[2 * (size_t)r + 1]));
  }
  int nr = rend - r0;
  int q0 = __shfl_sync(0xffffffffu, myq0, 0), q1 = rp[rend];
  for (int qb = q0; qb < q1; qb += 32) {
    int q = qb + lane;
    // the row of block q: the last row of the warp whose first block is <= q
    int lo_ = 0, hi_ = nr - 1;
#pragma unroll
    for (int it = 0; it < 5; it++) {
      int mid = (lo_ + hi_ + 1) >> 1;
      int st = __shfl_sync(0xffffffffu, myq0, mid);
      if (st <= q) lo_ = mid; else hi_ = mid - 1;
    }
    double rt = __shfl_sync(0xffffffffu, ratio, lo_);
    if (q < q1) {
      double4 B = reinterpret_cast<double4 *>(val)[q];
      if (r0 + lo_ < n) {
        B.x = sub_rn(B.x, mul_rn(rt, B.z));
        B.y = sub_rn(B.y, mul_rn(rt, B.w));
        reinterpret_cast<double2 *>(val)[2 * (size_t)q] = make_double2(B.x, B.y);
      }
      float4 h = make_float4((float)B.x, (float)B.y, (float)B.z, (float)B.w);
      reinterpret_cast<float4 *>(val32)[q] = h;
      reinterpret_cast<float4 *>(lo)[q] =
          make_float4(__double2float_rn(B.x - (double)h.x), __double2float_rn(B.y - (double)h.y),
                      __double2float_rn(B.z - (double)h.z), __double2float_rn(B.w - (double)h.w));
    }
  }
}

__global__ void k_identity_d(int nb, double *dmat) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb) return;
  double *D = dmat + 4 * (size_t)i;
  D[0] = 1; D[1] = 0; D[2] = 0; D[3] = 1;
}

// A_pp: entry [0][0] of every cell-cell block (Pi_r of eq. 34 keeps cell pressures)
__global__ void k_extract_app(int nnz, const int *src, const double *val, double *v) {
  int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < nnz) v[k] = val[4 * (size_t)src[k]];
}

// ------------------------------------------------ double-float helpers ---
// Unevaluated sums hi + lo of two FP32 numbers (about 48 significant bits):
// Knuth's two-sum, and Dekker's product with the FMA giving a product's
// rounding error exactly.
__device__ __forceinline__ void df_two_sum(float a, float b, float &s, float &e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
__device__ __forceinline__ void df_fast(float a, float b, float &s, float &e) {   // |a| >= |b|
  s = __fadd_rn(a, b);
  e = __fsub_rn(b, __fsub_rn(s, a));
}
// (ah + al)(bh + bl) = p + e up to the dropped al bl
__device__ __forceinline__ void df_mul(float ah, float al, float bh, float bl, float &p, float &e) {
  p = __fmul_rn(ah, bh);
  e = __fmaf_rn(ah, bh, -p);
  e = __fmaf_rn(ah, bl, e);
  e = __fmaf_rn(al, bh, e);
}
__device__ __forceinline__ void df_add(float &h, float &l, float h2, float l2) {
  float s, e;
  df_two_sum(h, h2, s, e);
  e = __fadd_rn(e, __fadd_rn(l, l2));
  df_fast(s, e, h, l);
}
__device__ __forceinline__ void df_split(double x, float &h, float &l) {
  h = __double2float_rn(x);
  l = __double2float_rn(x - (double)h);
}
// running sum s + c of products p + e
__device__ __forceinline__ void df_acc(float &s, float &c, float p, float e) {
  float t, err;
  df_two_sum(s, p, t, err);
  s = t;
  c = __fadd_rn(c, __fadd_rn(err, e));
}

// ------------------------------------------------------------- SpMV ------
template <class T> struct vec2_t;
template <> struct vec2_t<double> { typedef double2 type; };
template <> struct vec2_t<float> { typedef float2 type; };

// y = A x  (f == nullptr) or y = f - A x.  Optional, for CPR: with e, x's
// pressure components of the first np rows read as x_p + e (the pressure
// correction added on the fly, the same FP32 sum as a separate pass), and
// the corrected x written to xout for the warp's own rows; with pout, the
// pressure components of y of the first np rows also written there.  One
// warp owns 32 consecutive block rows: the warp reads its contiguous range of blocks coalesced
// (lane t takes block q0 + t + 32k), stages the 2-vectors A_q x_{c(q)} in
// shared memory, and each lane then sums the products of its own row in
// ascending block order.
#define SPMV_WARPS 8
#define SPMV_CHUNK 256
template <class Tv, class Tx, class Tf, class Ty>
__global__ void __launch_bounds__(SPMV_WARPS * 32)
k_bsr_spmv(int nb, const int *__restrict__ rp, const int *__restrict__ ci, const Tv *__restrict__ val,
           const Tx *__restrict__ x, const Tf *__restrict__ f, Ty *__restrict__ y, int np = 0,
           const Tx *__restrict__ e = nullptr, Tx *__restrict__ xout = nullptr, Ty *__restrict__ pout = nullptr) {
  __shared__ Ty prod[SPMV_WARPS][SPMV_CHUNK][2];
  int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int r0 = (blockIdx.x * SPMV_WARPS + wid) * 32;
  if (r0 >= nb) return;
  int r = r0 + lane, rend = min(r0 + 32, nb);
  int q0 = rp[r0], q1 = rp[rend];
  int myq0 = r < nb ? rp[r] : q1, myq1 = r < nb ? rp[r + 1] : q1;
  Ty a0 = 0, a1 = 0;
  typedef typename vec2_t<Tx>::type X2;
  for (int c0 = q0; c0 < q1; c0 += SPMV_CHUNK) {
    int c1 = min(c0 + SPMV_CHUNK, q1);
#pragma unroll 4
    for (int q = c0 + lane; q < c1; q += 32) {
      int c = __ldg(ci + q);
      X2 xv = reinterpret_cast<const X2 *>(x)[c];
      Ty b0, b1, b2, b3;
      if (sizeof(Tv) == 8) {
        double2 u = __ldg(reinterpret_cast<const double2 *>(val) + 2 * (size_t)q);
        double2 w = __ldg(reinterpret_cast<const double2 *>(val) + 2 * (size_t)q + 1);
        b0 = (Ty)u.x; b1 = (Ty)u.y; b2 = (Ty)w.x; b3 = (Ty)w.y;
      } else {
        float4 u = __ldg(reinterpret_cast<const float4 *>(val) + q);
        b0 = (Ty)u.x; b1 = (Ty)u.y; b2 = (Ty)u.z; b3 = (Ty)u.w;
      }
      if (e && c < np) xv.x = xv.x + e[c];
      Ty x0 = (Ty)xv.x, x1 = (Ty)xv.y;
      prod[wid][q - c0][0] = b0 * x0 + b1 * x1;
      prod[wid][q - c0][1] = b2 * x0 + b3 * x1;
    }
    __syncwarp();
    int s0 = max(myq0, c0), s1 = min(myq1, c1);
    for (int q = s0; q < s1; q++) { a0 += prod[wid][q - c0][0]; a1 += prod[wid][q - c0][1]; }
    __syncwarp();
  }
  if (r < nb) {
    if (f) { a0 = (Ty)f[2 * (size_t)r] - a0; a1 = (Ty)f[2 * (size_t)r + 1] - a1; }
    typedef typename vec2_t<Ty>::type Y2;
    Y2 o; o.x = a0; o.y = a1;
    reinterpret_cast<Y2 *>(y)[r] = o;
    if (pout && r < np) pout[r] = a0;
    if (xout) {
      X2 xr = reinterpret_cast<const X2 *>(x)[r];
      if (e && r < np) xr.x = xr.x + e[r];
      reinterpret_cast<X2 *>(xout)[r] = xr;
    }
  }
}

template <class Tv, class Tx, class Tf, class Ty>
static void spmv(const sim_ls_s *ls, const Tv *val, const Tx *x, const Tf *f, Ty *y, cudaStream_t s,
                 const Tx *e = nullptr, Tx *xout = nullptr, Ty *pout = nullptr) {
  unsigned g = grid_for(ls->nb, SPMV_WARPS * 32);
  k_bsr_spmv<Tv, Tx, Tf, Ty><<<g, SPMV_WARPS * 32, 0, s>>>(ls->nb, ls->rp.p, ls->ci.p, val, x, f, y, ls->n, e, xout,
                                                           pout);
  RS_LAUNCHED(1);
}

// w = A z for the double-float basis: the decoupled matrix as hi (val32) +
// lo (vallo) FP32 planes, z FP32 (exact), each block's products and each
// row's sum carried as double-float on the FP32 pipes (the FP64 SpMV above is
// bound by the FP64 rate).  Same traversal as k_bsr_spmv; w goes straight into
// its hi / lo planes (w, w + 2 nb).
__global__ void __launch_bounds__(SPMV_WARPS * 32)
k_bsr_spmv_df(int nb, const int *__restrict__ rp, const int *__restrict__ ci, const float *__restrict__ vh,
              const float *__restrict__ vl, const float *__restrict__ x, float *__restrict__ w) {
  __shared__ float2 prod[SPMV_WARPS][SPMV_CHUNK][2];
  int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int r0 = (blockIdx.x * SPMV_WARPS + wid) * 32;
  if (r0 >= nb) return;
  int r = r0 + lane, rend = min(r0 + 32, nb);
  int q0 = rp[r0], q1 = rp[rend];
  int myq0 = r < nb ? rp[r] : q1, myq1 = r < nb ? rp[r + 1] : q1;
  float a0h = 0.0f, a0l = 0.0f, a1h = 0.0f, a1l = 0.0f;
  for (int c0 = q0; c0 < q1; c0 += SPMV_CHUNK) {
    int c1 = min(c0 + SPMV_CHUNK, q1);
#pragma unroll 4
    for (int q = c0 + lane; q < c1; q += 32) {
      int c = __ldg(ci + q);
      float2 xv = reinterpret_cast<const float2 *>(x)[c];
      float4 bh = __ldg(reinterpret_cast<const float4 *>(vh) + q);
      float4 bl = __ldg(reinterpret_cast<const float4 *>(vl) + q);
      float p0, e0, p1, e1, h, l;
      // row 0 of the block: b0 x0 + b1 x1
      p0 = __fmul_rn(bh.x, xv.x); e0 = __fmaf_rn(bh.x, xv.x, -p0); e0 = __fmaf_rn(bl.x, xv.x, e0);
      p1 = __fmul_rn(bh.y, xv.y); e1 = __fmaf_rn(bh.y, xv.y, -p1); e1 = __fmaf_rn(bl.y, xv.y, e1);
      df_fast(p0, e0, h, l); df_add(h, l, p1, e1);
      prod[wid][q - c0][0] = make_float2(h, l);
      // row 1: b2 x0 + b3 x1
      p0 = __fmul_rn(bh.z, xv.x); e0 = __fmaf_rn(bh.z, xv.x, -p0); e0 = __fmaf_rn(bl.z, xv.x, e0);
      p1 = __fmul_rn(bh.w, xv.y); e1 = __fmaf_rn(bh.w, xv.y, -p1); e1 = __fmaf_rn(bl.w, xv.y, e1);
      df_fast(p0, e0, h, l); df_add(h, l, p1, e1);
      prod[wid][q - c0][1] = make_float2(h, l);
    }
    __syncwarp();
    int s0 = max(myq0, c0), s1 = min(myq1, c1);
    for (int q = s0; q < s1; q++) {
      float2 u = prod[wid][q - c0][0], v = prod[wid][q - c0][1];
      df_add(a0h, a0l, u.x, u.y);
      df_add(a1h, a1l, v.x, v.y);
    }
    __syncwarp();
  }
  if (r < nb) {
    size_t nu = 2 * (size_t)nb;
    reinterpret_cast<float2 *>(w)[r] = make_float2(a0h, a1h);
    reinterpret_cast<float2 *>(w + nu)[r] = make_float2(a0l, a1l);
  }
}
static void spmv_df(const sim_ls_s *ls, const float *x, float *w, cudaStream_t s) {
  unsigned g = grid_for(ls->nb, SPMV_WARPS * 32);
  k_bsr_spmv_df<<<g, SPMV_WARPS * 32, 0, s>>>(ls->nb, ls->rp.p, ls->ci.p, ls->val32.p, ls->vallo.p, x, w);
  RS_LAUNCHED(1);
}
// lo plane of the decoupled matrix: val - (double)val32
__global__ void k_val_lo(size_t m, const double *val, const float *val32, float *lo) {
  size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (k < m) lo[k] = __double2float_rn(val[k] - (double)val32[k]);
}

void ls_spmv64(sim_ls_s *ls, const double *x, double *y) {
  rs_timed tm(ls, SIM_T_SPMV64);
  spmv<double, double, double, double>(ls, ls->val.p, x, (const double *)nullptr, y, ls->st);
}
void ls_spmv64_untimed(sim_ls_s *ls, const double *x, double *y) {
  spmv<double, double, double, double>(ls, ls->val.p, x, (const double *)nullptr, y, ls->st);
}

// ------------------------------------------------------- CPR pieces ------
template <class Ti, class To>
__global__ void k_gather_p(int n, const Ti *r, To *f) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) f[i] = (To)r[2 * (size_t)i];
}
template <class T>
__global__ void k_add_p(int n, const T *e, T *x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) x[2 * (size_t)i] += e[i];
}

// CPR-FPF (Algorithm 2): z = R^{-1} v; r = v - A z; z += Pi_p M(A_pp)^{-1} Pi_r r;
// r = v - A z; z += R^{-1} r.  FP64 preconditioner: A is the decoupled FP64
// matrix; mixed: FP32 matrix, factors, hierarchy and vectors (FP64 coarsest).
// FP32 scratch vector of the CPR application (the first RAS stage's output)
static float *cpr_scratch(sim_ls_s *ls) {
  ls->cprt32.ensure(2 * (size_t)ls->nb);
  return ls->cprt32.p;
}

void ls_cpr(sim_ls_s *ls, const double *v, double *z64, float *z32) {
  cudaStream_t s = ls->st;
  int n = ls->n;
  amg_level &L0 = ls->amg.lev[0];
  if (ls->o.precision != SIM_PREC_FP64) {
    // the first RAS stage into a scratch vector; the second SpMV reads it
    // with the pressure correction added on the fly and writes the
    // corrected iterate into z; the first SpMV also writes the pressure
    // residual the V-cycle starts from
    float *r = ls->x32b.p, *zt = cpr_scratch(ls);
    ls_ras_apply<float, double>(ls, v, zt, false);                                     // RAS
    { rs_timed tm(ls, SIM_T_SPMV_PREC); spmv<float, float, double, float>(ls, ls->val32.p, zt, v, r, s, nullptr, nullptr, L0.f32.p); }  // r = v - A z
    { rs_timed tm(ls, SIM_T_VCYCLE); if (ls->capturing) amg_vcycle<float>(ls->amg, 0, s); else amg_vcycle_graph<float>(ls->amg, s); }  // pressure V-cycle
    { rs_timed tm(ls, SIM_T_SPMV_PREC); spmv<float, float, double, float>(ls, ls->val32.p, zt, v, r, s, L0.x32.p, z32); }  // z = z + P e, r = v - A z
    ls_ras_apply<float, float>(ls, r, z32, true);                                      // RAS, added
  } else {
    double *z = z64, *r = ls->x64a.p;
    ls_ras_apply<double, double>(ls, v, z, false);
    { rs_timed tm(ls, SIM_T_SPMV_PREC); spmv<double, double, double, double>(ls, ls->val.p, z, v, r, s); }
    k_gather_p<double, double><<<grid_for(n, 256), 256, 0, s>>>(n, r, L0.f.p);
    RS_LAUNCHED(1);
    { rs_timed tm(ls, SIM_T_VCYCLE); if (ls->capturing) amg_vcycle<double>(ls->amg, 0, s); else amg_vcycle_graph<double>(ls->amg, s); }
    k_add_p<double><<<grid_for(n, 256), 256, 0, s>>>(n, L0.x.p, z);
    RS_LAUNCHED(1);
    { rs_timed tm(ls, SIM_T_SPMV_PREC); spmv<double, double, double, double>(ls, ls->val.p, z, v, r, s); }
    ls_ras_apply<double, double>(ls, r, z, true);
  }
}

// CPR-FPF with an FP32 input vector (mixed precision with the double-float
// basis, whose hi plane is the FP32 value of a basis vector): the same steps
// as ls_cpr's mixed branch.
void ls_cpr32(sim_ls_s *ls, const float *v, float *z) {
  cudaStream_t s = ls->st;
  int n = ls->n;
  amg_level &L0 = ls->amg.lev[0];
  float *r = ls->x32b.p, *zt = cpr_scratch(ls);
  ls_ras_apply<float, float>(ls, v, zt, false);                                        // RAS
  { rs_timed tm(ls, SIM_T_SPMV_PREC); spmv<float, float, float, float>(ls, ls->val32.p, zt, v, r, s, nullptr, nullptr, L0.f32.p); }   // r = v - A z
  { rs_timed tm(ls, SIM_T_VCYCLE); if (ls->capturing) amg_vcycle<float>(ls->amg, 0, s); else amg_vcycle_graph<float>(ls->amg, s); }  // pressure V-cycle
  { rs_timed tm(ls, SIM_T_SPMV_PREC); spmv<float, float, float, float>(ls, ls->val32.p, zt, v, r, s, L0.x32.p, z); }   // z = z + P e, r = v - A z
  ls_ras_apply<float, float>(ls, r, z, true);                                          // RAS, added
}

// ------------------------------------------------------------ init -------
void ls_init(sim_ls_s *ls, int nx, int ny, int nz, int nw, const int *rp, const int *ci, const int *well_cell0,
             const rs_opts &o, cudaStream_t st) {
  ls->nx = nx; ls->ny = ny; ls->nz = nz; ls->n = nx * ny * nz; ls->nw = nw; ls->nb = ls->n + nw;
  ls->o = o; ls->st = st;
  int nb = ls->nb;
  ls->h_rp.assign(rp, rp + nb + 1);
  ls->nnzb = rp[nb];
  ls->h_ci.assign(ci, ci + ls->nnzb);
  ls->h_wc0.assign(well_cell0, well_cell0 + nw);
  std::vector<int> dpos(nb, -1), app_src, app_rp(ls->n + 1, 0), app_ci;
  for (int i = 0; i < nb; i++) {
    for (int q = rp[i]; q < rp[i + 1]; q++) {
      if (q > rp[i] && ci[q] <= ci[q - 1]) RS_FAIL(SIM_ERR_ARG, "row %d: columns not strictly ascending", i);
      if (ci[q] < 0 || ci[q] >= nb) RS_FAIL(SIM_ERR_ARG, "row %d: column out of range", i);
      if (ci[q] == i) dpos[i] = q;
      if (i < ls->n && ci[q] < ls->n) { app_src.push_back(q); app_ci.push_back(ci[q]); }
    }
    if (dpos[i] < 0) RS_FAIL(SIM_ERR_ARG, "row %d has no diagonal block", i);
    if (i < ls->n) app_rp[i + 1] = (int)app_src.size();
  }
  for (int w = 0; w < nw; w++)
    if (well_cell0[w] < 0 || well_cell0[w] >= ls->n) RS_FAIL(SIM_ERR_ARG, "well %d: bad first perforation", w);
  h2d(ls->rp, ls->h_rp, st); h2d(ls->ci, ls->h_ci, st); h2d(ls->dpos, dpos, st);
  ls->val.alloc(4 * (size_t)ls->nnzb); ls->b.alloc(2 * (size_t)nb); ls->key.alloc(ls->n);
  ls->dmat.alloc(4 * (size_t)nb);
  if (o.precision != SIM_PREC_FP64) ls->val32.alloc(4 * (size_t)ls->nnzb);
  h2d(ls->app_src, app_src, st);
  csr_dev<double> &A0 = ls->amg.lev[0].A;
  A0.n = A0.m = ls->n; A0.nnz = (int)app_src.size();
  h2d(A0.rp, app_rp, st); h2d(A0.ci, app_ci, st); A0.v.alloc(A0.nnz);
  ras_build_static(ls);
  size_t nu = 2 * (size_t)nb;
  ls->y.alloc(nu); ls->w.alloc(nu); ls->r.alloc(nu);
  ls->x64a.alloc(nu); ls->x64b.alloc(nu);
  if (o.precision != SIM_PREC_FP64) { ls->x32b.alloc(nu); ls->x32c.alloc(nu); }
  RS_CUDA(cudaHostAlloc((void **)&ls->hpin, 4 * (ORTHO_MAXV + 2) * sizeof(double), cudaHostAllocMapped));
  for (int k = 0; k < 4 * (ORTHO_MAXV + 2); k++) ls->hpin[k] = 0.0;
  RS_CUDA(cudaHostAlloc((void **)&ls->errw, 16 * sizeof(int), cudaHostAllocMapped));
  for (int k = 0; k < 16; k++) ls->errw[k] = 0;
  RS_CUDA(cudaHostGetDevicePointer((void **)&ls->errw_dev, ls->errw, 0));
  RS_CUDA(cudaStreamSynchronize(st));
}

void ls_setup(sim_ls_s *ls) {
  cudaStream_t s = ls->st;
  ls->drop_graph();                         // buffers of the hierarchy may move
  float *v32 = ls->o.precision != SIM_PREC_FP64 ? ls->val32.p : nullptr;
  unsigned g = grid_for(ls->nb, 128);
  {
  rs_timed tm(ls, SIM_T_DECOUPLE);
  if (ls->o.decoupling == SIM_DEC_ABF)
    k_abf<<<g, 128, 0, s>>>(ls->n, ls->nb, ls->rp.p, ls->dpos.p, ls->val.p, ls->b.p, ls->dmat.p, v32);
  else if (ls->o.decoupling == SIM_DEC_QI && !v32)
    k_qi<<<g, 128, 0, s>>>(ls->n, ls->nb, ls->rp.p, ls->dpos.p, ls->val.p, ls->b.p, ls->dmat.p, v32);
  else if (ls->o.decoupling != SIM_DEC_QI) {
    k_identity_d<<<g, 128, 0, s>>>(ls->nb, ls->dmat.p);
    if (v32) rs_cast_d2f(ls->val.p, v32, 4 * (size_t)ls->nnzb, s);
  }
  if (v32) {                                 // the double-float SpMV's lo plane
    size_t m4 = 4 * (size_t)ls->nnzb;
    ls->vallo.ensure(m4);
    cpr_scratch(ls);                         // allocated before any graph records it
    if (ls->o.decoupling == SIM_DEC_QI)      // decoupling, FP32 copy and lo plane in one pass
      k_qi_fused<<<grid_for(ls->nb, 256), 256, 0, s>>>(ls->n, ls->nb, ls->rp.p, ls->dpos.p, ls->val.p, ls->b.p,
                                                       ls->dmat.p, v32, ls->vallo.p);
    else
      k_val_lo<<<grid_for(m4, 256), 256, 0, s>>>(m4, ls->val.p, v32, ls->vallo.p);
    RS_LAUNCHED(1);
  }
  if (!(ls->o.decoupling == SIM_DEC_QI && v32)) RS_LAUNCHED(1);
  csr_dev<double> &A0 = ls->amg.lev[0].A;
  k_extract_app<<<grid_for(A0.nnz, 256), 256, 0, s>>>(A0.nnz, ls->app_src.p, ls->val.p, A0.v.p);
  RS_LAUNCHED(1);
  }
  RS_CHECK_LAUNCH();
  // The AMG setup on a second stream of the highest priority, concurrently
  // with the RAS setup (reordering, level sets, factors, streams) on the
  // first: independent work on the same decoupled matrix.  The AMG setup is
  // the longer chain (FP64-bound, and it waits for sizes a few times), so
  // its blocks go first.  (Issuing the RAS setup only once the AMG setup's
  // finest level was under way measured slower: 9.8 against 9.1 ms per
  // setup on the 1M-cell case.)
  if (!ls->st2) {
    int least = 0, greatest = 0;
    RS_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
    RS_CUDA(cudaStreamCreateWithPriority(&ls->st2, cudaStreamNonBlocking, greatest));
    RS_CUDA(cudaEventCreateWithFlags(&ls->ev_fork, cudaEventDisableTiming));
    RS_CUDA(cudaEventCreateWithFlags(&ls->ev_join, cudaEventDisableTiming));
  }
  RS_CUDA(cudaEventRecord(ls->ev_fork, s));
  RS_CUDA(cudaStreamWaitEvent(ls->st2, ls->ev_fork, 0));
  struct swap_stream {                       // ls->st names another stream inside a scope
    sim_ls_s *l; cudaStream_t keep;
    swap_stream(sim_ls_s *l_, cudaStream_t to) : l(l_), keep(l_->st) { l->st = to; }
    ~swap_stream() { l->st = keep; }
  };
  { rs_timed tm(ls, SIM_T_RAS_SETUP); ras_setup(ls); }   // no host waits: issued at once
  {
    swap_stream sw(ls, ls->st2);
    rs_timed tm(ls, SIM_T_AMG_SETUP);
    amg_setup(ls->amg, ls->o, ls->st2);
  }
  RS_CUDA(cudaEventRecord(ls->ev_join, ls->st2));
  RS_CUDA(cudaStreamWaitEvent(s, ls->ev_join, 0));
  ls->have_setup = true;
}

// ------------------------------------------------------------ FGMRES -----
// Classical Gram-Schmidt with a conditional second pass (Daniel, Gragg,
// Kaufman and Stewart): the second projection runs only when the first one
// kept less than 1% of w (||w_1||^2 < 1e-4 ||w||^2).  The test is taken on the device; the
// kernels of the second pass read the flag and return at once when it is
// clear, so the host never waits on it.  Each pass is one sweep over the
// rows: a block owns a fixed row range, threads accumulate their part of
// each dot product, warps reduce with shuffles and the block writes one
// partial per vector; a second kernel adds the partials in block order, so
// results do not depend on scheduling.
#define ORTHO_BS 256
// Each block owns a fixed chunk of ORTHO_CH rows and keeps its slice of w in
// shared memory.  Basis vectors are streamed vector-outer, rows-inner, so
// loads are coalesced and independent.
#define ORTHO_CH 2048
#define ORTHO_CH_DF 8192
static int ortho_blocks(int nu) { return (nu + ORTHO_CH - 1) / ORTHO_CH; }

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double block_sum_d(double v, double *sred) {   // result valid in thread 0
  v = warp_sum_d(v);
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) for (int q = 0; q < ORTHO_BS / 32; q++) t += sred[q];
  __syncthreads();
  return t;
}

// Basis vectors are taken ORTHO_G at a time: a thread keeps one accumulator
// per vector of the group and issues the group's loads for a row together.
#define ORTHO_G 8

// Sum of a[0..7] over the warp for each of the 8 slots at once: at every
// halving step a lane keeps half of its slots and adds the partner's copy of
// them (9 shuffles and 9 adds for 8 sums, instead of 5 of each per sum).
// Afterwards lane l holds the total of slot ((l>>4)&1)*4 + ((l>>3)&1)*2 + ((l>>2)&1).
__device__ __forceinline__ double warp_sum8_d(const double *a, int lane) {
  double b4[4], b2[2];
  bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4;
#pragma unroll
  for (int q = 0; q < 4; q++) {
    double keep = u16 ? a[q + 4] : a[q], give = u16 ? a[q] : a[q + 4];
    b4[q] = keep + __shfl_xor_sync(0xffffffffu, give, 16);
  }
#pragma unroll
  for (int q = 0; q < 2; q++) {
    double keep = u8 ? b4[q + 2] : b4[q], give = u8 ? b4[q] : b4[q + 2];
    b2[q] = keep + __shfl_xor_sync(0xffffffffu, give, 8);
  }
  double keep = u4 ? b2[1] : b2[0], give = u4 ? b2[0] : b2[1];
  double t = keep + __shfl_xor_sync(0xffffffffu, give, 4);
  t += __shfl_xor_sync(0xffffffffu, t, 2);
  t += __shfl_xor_sync(0xffffffffu, t, 1);
  return t;
}

// part[k][b] = V_k . w over the block's rows (k < nv); with_norm: part[nv][b] = w . w
__global__ void __launch_bounds__(ORTHO_BS) k_ortho_dots(int nu, int nv, const double *__restrict__ V,
                                                         const double *__restrict__ w, double *part, int with_norm,
                                                         const int *cond, const int *jd) {
  if (cond && *cond == 0) return;
  if (jd) nv = *jd + 1;                        // graph replay: the step index lives on the device
  extern __shared__ double ws[];             // ORTHO_CH doubles (dynamic)
  __shared__ double red[2][ORTHO_BS / 32][ORTHO_G];
  int nblk = gridDim.x, i0 = blockIdx.x * ORTHO_CH, len = min(ORTHO_CH, nu - i0);
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < len; t += ORTHO_BS) ws[t] = w[i0 + t];
  __syncthreads();
  int nt = nv + (with_norm ? 1 : 0);
  for (int k0 = 0, grp = 0; k0 < nt; k0 += ORTHO_G, grp ^= 1) {
    const double *vp[ORTHO_G];
    double acc[ORTHO_G];
#pragma unroll
    for (int g = 0; g < ORTHO_G; g++) {
      int k = k0 + g;                          // vector nv is w itself (its squared norm)
      vp[g] = k < nv ? V + (size_t)k * nu + i0 : (k == nv ? w + i0 : nullptr);
      acc[g] = 0.0;
    }
    for (int t = threadIdx.x; t < len; t += ORTHO_BS) {
      double wt = ws[t];
#pragma unroll
      for (int g = 0; g < ORTHO_G; g++)
        if (vp[g]) acc[g] += __ldg(vp[g] + t) * wt;
    }
    double tot = warp_sum8_d(acc, lane);
    if ((lane & 3) == 0) red[grp][warp][((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1)] = tot;
    __syncthreads();                           // red[grp] is rewritten two groups later, after another barrier
    if (threadIdx.x < ORTHO_G && k0 + threadIdx.x < nt) {
      double s = 0.0;
      for (int q = 0; q < ORTHO_BS / 32; q++) s += red[grp][q][threadIdx.x];
      part[(size_t)(k0 + threadIdx.x) * nblk + blockIdx.x] = s;
    }
  }
}

// w -= sum_k h_k V_k over the block's rows, then part[0][b] = ||w||^2
__global__ void __launch_bounds__(ORTHO_BS) k_ortho_update(int nu, int nv, const double *__restrict__ V, double *w,
                                                           const double *__restrict__ h, double *part,
                                                           const int *cond, const int *jd) {
  if (cond && *cond == 0) return;
  if (jd) nv = *jd + 1;
  extern __shared__ double ws[];
  __shared__ double sred[ORTHO_BS / 32];
  int i0 = blockIdx.x * ORTHO_CH, len = min(ORTHO_CH, nu - i0);
  for (int t = threadIdx.x; t < len; t += ORTHO_BS) ws[t] = w[i0 + t];
  for (int k0 = 0; k0 < nv; k0 += ORTHO_G) {   // each thread updates only its own rows: no barrier needed
    const double *vp[ORTHO_G];
    double hk[ORTHO_G];
#pragma unroll
    for (int g = 0; g < ORTHO_G; g++) {
      int k = k0 + g;
      vp[g] = k < nv ? V + (size_t)k * nu + i0 : nullptr;
      hk[g] = k < nv ? h[k] : 0.0;
    }
    // two rows per thread per iteration: their 16 loads are in flight together
    for (int t = threadIdx.x; t < len; t += 2 * ORTHO_BS) {
      int t2 = t + ORTHO_BS;
      bool two = t2 < len;
      double v0[ORTHO_G], v1[ORTHO_G];
#pragma unroll
      for (int g = 0; g < ORTHO_G; g++) {
        if (vp[g]) { v0[g] = __ldg(vp[g] + t); if (two) v1[g] = __ldg(vp[g] + t2); }
      }
      double s0 = ws[t], s1 = two ? ws[t2] : 0.0;
#pragma unroll
      for (int g = 0; g < ORTHO_G; g++)       // same order as one vector at a time: w - h_0 v_0 - h_1 v_1 ...
        if (vp[g]) { s0 -= hk[g] * v0[g]; if (two) s1 -= hk[g] * v1[g]; }
      ws[t] = s0;
      if (two) ws[t2] = s1;
    }
  }
  double n2 = 0.0;
  for (int t = threadIdx.x; t < len; t += ORTHO_BS) { double v = ws[t]; w[i0 + t] = v; n2 += v * v; }
  double tot = block_sum_d(n2, sred);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// ------------------------------------------------ double-float basis ----
// Mixed precision keeps the Arnoldi basis and the vector being
// orthogonalised as unevaluated sums hi + lo of two FP32 numbers (about 48
// significant bits), stored as two planes per vector (hi[nu], then lo[nu]).
// The Gram-Schmidt dot products and updates then run on the FP32 pipes:
// Dekker's product (an FMA yields the rounding error of a product) and
// Knuth's two-sum carry the low parts, instead of FP64 multiply-adds, whose
// rate bounds the FP64 kernels above.  Scalars (h, norms, Givens) stay
// FP64; the preconditioner reads a basis vector in FP32, which is its hi
// plane.
// warp_sum8_d for pairs: lane l ends with the total of the same slot
__device__ __forceinline__ void warp_sum8_df(const float *ah, const float *al, int lane, float &rh, float &rl) {
  float bh[4], bl[4], ch[2], cl[2];
  bool u16 = lane & 16, u8 = lane & 8, u4 = lane & 4;
#pragma unroll
  for (int q = 0; q < 4; q++) {
    float kh = u16 ? ah[q + 4] : ah[q], kl = u16 ? al[q + 4] : al[q];
    float gh = u16 ? ah[q] : ah[q + 4], gl = u16 ? al[q] : al[q + 4];
    gh = __shfl_xor_sync(0xffffffffu, gh, 16); gl = __shfl_xor_sync(0xffffffffu, gl, 16);
    df_add(kh, kl, gh, gl);
    bh[q] = kh; bl[q] = kl;
  }
#pragma unroll
  for (int q = 0; q < 2; q++) {
    float kh = u8 ? bh[q + 2] : bh[q], kl = u8 ? bl[q + 2] : bl[q];
    float gh = u8 ? bh[q] : bh[q + 2], gl = u8 ? bl[q] : bl[q + 2];
    gh = __shfl_xor_sync(0xffffffffu, gh, 8); gl = __shfl_xor_sync(0xffffffffu, gl, 8);
    df_add(kh, kl, gh, gl);
    ch[q] = kh; cl[q] = kl;
  }
  float kh = u4 ? ch[1] : ch[0], kl = u4 ? cl[1] : cl[0];
  float gh = u4 ? ch[0] : ch[1], gl = u4 ? cl[0] : cl[1];
  gh = __shfl_xor_sync(0xffffffffu, gh, 4); gl = __shfl_xor_sync(0xffffffffu, gl, 4);
  df_add(kh, kl, gh, gl);
#pragma unroll
  for (int o = 2; o > 0; o >>= 1) {
    float oh = __shfl_xor_sync(0xffffffffu, kh, o), ol = __shfl_xor_sync(0xffffffffu, kl, o);
    df_add(kh, kl, oh, ol);
  }
  rh = kh; rl = kl;
}
__device__ __forceinline__ double warp_sum_df(float h, float l) {        // result in every lane
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
    df_add(h, l, oh, ol);
  }
  return (double)h + (double)l;
}

// The block that finishes last (atomic ticket) sums the per-block partials
// part[k][b] into out[k] for k < nout, exactly as k_reduce_parts does (warp
// per k, lanes over a fixed stride of blocks, shuffle tree), and resets the
// ticket: the separate reduction launch between the sweeps disappears.
__device__ __forceinline__ bool last_block(int *ticket) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(ticket, 1) == (int)gridDim.x - 1;
  __syncthreads();
  return last;
}
__device__ __forceinline__ void reduce_tail(int nout, int nblk, const double *part, double *out, int *ticket) {
  __threadfence();
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int k = warp; k < nout; k += nw) {
    double t = 0;
    for (int b = lane; b < nblk; b += 32) t += __ldcg(part + (size_t)k * nblk + b);
    t = warp_sum_d(t);
    if (lane == 0) out[k] = t;
  }
  if (threadIdx.x == 0) *ticket = 0;
}

// k_ortho_dots on pair planes: V vector k at V + 2k nu (hi) and + (2k+1) nu
// (lo), w at w (hi) and w + nu (lo).  Vector offsets are 32-bit (the basis
// holds at most 2 (ORTHO_MAXV + 1) nu < 2^31 floats) and each thread takes
// two rows per iteration, so that 32 loads are in flight together.
__global__ void __launch_bounds__(ORTHO_BS, 4) k_ortho_dots_df(int nu, int ch, int nv, const float *__restrict__ V,
                                                               const float *__restrict__ w, double *part,
                                                               int with_norm, const int *cond, const int *jd,
                                                               int *ticket, double *out) {
  if (cond && *cond == 0) return;
  if (jd) nv = *jd + 1;
  extern __shared__ float2 wp[];               // ORTHO_CH pairs (dynamic)
  __shared__ double red[2][ORTHO_BS / 32][ORTHO_G];
  int nblk = gridDim.x, i0 = blockIdx.x * ch, len = min(ch, nu - i0);
  int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < len; t += ORTHO_BS) wp[t] = make_float2(w[i0 + t], w[(size_t)nu + i0 + t]);
  __syncthreads();
  const float *vb = V + i0;
  int nt = nv + (with_norm ? 1 : 0);
  for (int k0 = 0, grp = 0; k0 < nt; k0 += ORTHO_G, grp ^= 1) {
    float as[ORTHO_G], ac[ORTHO_G];
#pragma unroll
    for (int g = 0; g < ORTHO_G; g++) { as[g] = 0.0f; ac[g] = 0.0f; }
    int ng = min(ORTHO_G, nv - k0);            // basis vectors in this group; slot nv - k0 is w's norm
    for (int t = threadIdx.x; t < len; t += 2 * ORTHO_BS) {
      int t2 = t + ORTHO_BS;
      bool two = t2 < len;
      float ah[ORTHO_G], al[ORTHO_G], bh[ORTHO_G], bl[ORTHO_G];
#pragma unroll
      for (int g = 0; g < ORTHO_G; g++)
        if (g < ng) {
          int o = 2 * (k0 + g) * nu;
          ah[g] = __ldg(vb + o + t); al[g] = __ldg(vb + o + nu + t);
          if (two) { bh[g] = __ldg(vb + o + t2); bl[g] = __ldg(vb + o + nu + t2); }
        }
      float2 x = wp[t], y = two ? wp[t2] : make_float2(0.0f, 0.0f);
#pragma unroll
      for (int g = 0; g < ORTHO_G; g++) {
        float p, e;
        if (g < ng) {
          df_mul(ah[g], al[g], x.x, x.y, p, e); df_acc(as[g], ac[g], p, e);
          if (two) { df_mul(bh[g], bl[g], y.x, y.y, p, e); df_acc(as[g], ac[g], p, e); }
        } else if (k0 + g == nv && with_norm) {
          df_mul(x.x, x.y, x.x, x.y, p, e); df_acc(as[g], ac[g], p, e);
          if (two) { df_mul(y.x, y.y, y.x, y.y, p, e); df_acc(as[g], ac[g], p, e); }
        }
      }
    }
    float hh[ORTHO_G], ll[ORTHO_G];
#pragma unroll
    for (int g = 0; g < ORTHO_G; g++) df_fast(as[g], ac[g], hh[g], ll[g]);
    float rh, rl;
    warp_sum8_df(hh, ll, lane, rh, rl);
    if ((lane & 3) == 0)
      red[grp][warp][((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1)] = (double)rh + (double)rl;
    __syncthreads();                           // red[grp] is rewritten two groups later, after another barrier
    if (threadIdx.x < ORTHO_G && k0 + threadIdx.x < nt) {
      double sum = 0.0;
      for (int q = 0; q < ORTHO_BS / 32; q++) sum += red[grp][q][threadIdx.x];
      part[(size_t)(k0 + threadIdx.x) * nblk + blockIdx.x] = sum;
    }
  }
  if (last_block(ticket)) reduce_tail(nt, nblk, part, out, ticket);   // out[k] = V_k . w (and ||w||^2)
}

// k_ortho_update on pair planes: w -= sum_k h_k V_k (h FP64, split once per
// block), then part[0][b] = ||w||^2 over the block's rows; two rows per
// thread per iteration
__global__ void __launch_bounds__(ORTHO_BS, 4) k_ortho_update_df(int nu, int ch, int nv, const float *__restrict__ V,
                                                                 float *w, const double *__restrict__ h, double *part,
                                                                 const int *cond, const int *jd, int *ticket,
                                                                 double *nrm, int *flag, const double *h1) {
  if (cond && *cond == 0) return;
  if (jd) nv = *jd + 1;
  extern __shared__ float2 wp[];
  __shared__ float2 hs[ORTHO_MAXV + 1];
  __shared__ double sred[ORTHO_BS / 32];
  int i0 = blockIdx.x * ch, len = min(ch, nu - i0);
  for (int t = threadIdx.x; t < nv; t += ORTHO_BS) { float a, b; df_split(h[t], a, b); hs[t] = make_float2(a, b); }
  for (int t = threadIdx.x; t < len; t += ORTHO_BS) wp[t] = make_float2(w[i0 + t], w[(size_t)nu + i0 + t]);
  __syncthreads();
  const float *vb = V + i0;
  for (int k0 = 0; k0 < nv; k0 += ORTHO_G) {   // each thread updates only its own rows: no barrier needed
    int ng = min(ORTHO_G, nv - k0);
    for (int t = threadIdx.x; t < len; t += 2 * ORTHO_BS) {
      int t2 = t + ORTHO_BS;
      bool two = t2 < len;
      float ah[ORTHO_G], al[ORTHO_G], bh[ORTHO_G], bl[ORTHO_G];
#pragma unroll
      for (int g = 0; g < ORTHO_G; g++)
        if (g < ng) {
          int o = 2 * (k0 + g) * nu;
          ah[g] = __ldg(vb + o + t); al[g] = __ldg(vb + o + nu + t);
          if (two) { bh[g] = __ldg(vb + o + t2); bl[g] = __ldg(vb + o + nu + t2); }
        }
      float2 x = wp[t], y = two ? wp[t2] : make_float2(0.0f, 0.0f);
#pragma unroll
      for (int g = 0; g < ORTHO_G; g++)       // w - h_0 v_0 - h_1 v_1 ..., one vector at a time
        if (g < ng) {
          float2 hk = hs[k0 + g];
          float p, e, s2, err;
          df_mul(hk.x, hk.y, ah[g], al[g], p, e);
          df_two_sum(x.x, -p, s2, err);
          err = __fadd_rn(err, __fsub_rn(x.y, e));
          df_fast(s2, err, x.x, x.y);
          if (two) {
            df_mul(hk.x, hk.y, bh[g], bl[g], p, e);
            df_two_sum(y.x, -p, s2, err);
            err = __fadd_rn(err, __fsub_rn(y.y, e));
            df_fast(s2, err, y.x, y.y);
          }
        }
      wp[t] = x;
      if (two) wp[t2] = y;
    }
  }
  float ns = 0.0f, nc = 0.0f;
  for (int t = threadIdx.x; t < len; t += ORTHO_BS) {
    float2 x = wp[t];
    w[i0 + t] = x.x;
    w[(size_t)nu + i0 + t] = x.y;
    float p, e;
    df_mul(x.x, x.y, x.x, x.y, p, e);
    df_acc(ns, nc, p, e);
  }
  float nh, nl;
  df_fast(ns, nc, nh, nl);
  double wt = warp_sum_df(nh, nl);
  if ((threadIdx.x & 31) == 0) sred[threadIdx.x >> 5] = wt;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
    for (int q = 0; q < ORTHO_BS / 32; q++) tot += sred[q];
    part[blockIdx.x] = tot;
  }
  if (last_block(ticket)) {
    reduce_tail(1, gridDim.x, part, nrm, ticket);        // nrm = ||w||^2 after the pass
    // first pass: flag the second one when it kept less than 1% of w
    // (||w_1||^2 < 1e-4 ||w||^2, as k_dgks); ||w||^2 sits after the dot products
    if (flag && threadIdx.x == 0) { __threadfence(); *flag = (*(volatile double *)nrm < 1e-4 * h1[nv]) ? 1 : 0; }
  }
}
// V_{j+1} = w / h_{j+1,j}, the reciprocal split once by k_arnoldi_col (isp)
// v_{j+1} = w / h_{j+1,j} into the basis; with vcur, its hi plane also into
// the fixed buffer the next graph-replayed step's CPR reads
__global__ void k_scale_df(int nu, const float *w, const float *isp, float *V, int j1, const int *jd, float *vcur) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (jd) j1 = *jd + 1;
  if (i >= nu) return;
  float p, e, h, l;
  df_mul(w[i], w[(size_t)nu + i], isp[0], isp[1], p, e);
  df_fast(p, e, h, l);
  V[(size_t)(2 * j1) * nu + i] = h;
  V[(size_t)(2 * j1 + 1) * nu + i] = l;
  if (vcur) vcur[i] = h;
}
__global__ void k_start_df(int nu, const double *r, double beta, float *V, double *G, int m, float *vcur) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nu) {
    float h, l;
    df_split(r[i] * (1.0 / beta), h, l);
    V[i] = h; V[(size_t)nu + i] = l;
    if (vcur) vcur[i] = h;
  }
  if (i == 0) { double *g = G + (size_t)m * (m + 1) + 2 * m; for (int k = 0; k <= m; k++) g[k] = 0.0; g[0] = beta; }
}

static void ortho_attr() {
  static bool done = false;
  if (done) return;
  RS_CUDA(cudaFuncSetAttribute(k_ortho_dots, cudaFuncAttributeMaxDynamicSharedMemorySize, ORTHO_CH * 8));
  RS_CUDA(cudaFuncSetAttribute(k_ortho_update, cudaFuncAttributeMaxDynamicSharedMemorySize, ORTHO_CH * 8));
  RS_CUDA(cudaFuncSetAttribute(k_ortho_dots_df, cudaFuncAttributeMaxDynamicSharedMemorySize, ORTHO_CH_DF * 8));
  RS_CUDA(cudaFuncSetAttribute(k_ortho_update_df, cudaFuncAttributeMaxDynamicSharedMemorySize, ORTHO_CH_DF * 8));
  done = true;
}
static void ortho_dots(int nu, int nv, const double *V, const double *w, double *part, int with_norm, const int *cond,
                       int nblk, cudaStream_t s, const int *jd = nullptr) {
  ortho_attr();
  k_ortho_dots<<<nblk, ORTHO_BS, ORTHO_CH * 8, s>>>(nu, nv, V, w, part, with_norm, cond, jd);
}
static void ortho_update(int nu, int nv, const double *V, double *w, const double *h, double *part, const int *cond,
                         int nblk, cudaStream_t s, const int *jd = nullptr) {
  ortho_attr();
  k_ortho_update<<<nblk, ORTHO_BS, ORTHO_CH * 8, s>>>(nu, nv, V, w, h, part, cond, jd);
}

// double-float kernels: one wave of 4 blocks per SM, each owning an equal
// chunk of rows (a multiple of 64, at most ORTHO_CH_DF), its slice of w in
// shared memory
static int ortho_blocks_df(int nu, int *ch) {
  int nblk = 152 * 4;
  int c = ((nu + nblk - 1) / nblk + 63) & ~63;
  if (c > ORTHO_CH_DF) { c = ORTHO_CH_DF; nblk = (nu + c - 1) / c; }
  else nblk = (nu + c - 1) / c;
  *ch = c;
  return std::max(nblk, 1);
}
static void ortho_dots_df(int nu, int ch, int nv, const float *V, const float *w, double *part, int with_norm,
                          const int *cond, int nblk, cudaStream_t s, const int *jd, int *ticket, double *out) {
  ortho_attr();
  k_ortho_dots_df<<<nblk, ORTHO_BS, (size_t)ch * 8, s>>>(nu, ch, nv, V, w, part, with_norm, cond, jd, ticket, out);
}
static void ortho_update_df(int nu, int ch, int nv, const float *V, float *w, const double *h, double *part,
                            const int *cond, int nblk, cudaStream_t s, const int *jd, int *ticket, double *nrm,
                            int *flag, const double *h1) {
  ortho_attr();
  k_ortho_update_df<<<nblk, ORTHO_BS, (size_t)ch * 8, s>>>(nu, ch, nv, V, w, h, part, cond, jd, ticket, nrm, flag, h1);
}

// out[k] = sum over blocks of part[k][*]: one warp per k, lanes add a fixed
// stride of the partials, then a fixed shuffle tree (deterministic)
__global__ void k_reduce_parts(int nv, int nblk, const double *part, double *out, const int *cond, const int *jd,
                               int extra) {
  if (cond && *cond == 0) return;
  if (jd) nv = *jd + 1 + extra;
  int k = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (k >= nv) return;
  double t = 0;
  for (int b = lane; b < nblk; b += 32) t += part[(size_t)k * nblk + b];
  t = warp_sum_d(t);
  if (lane == 0) out[k] = t;
}
static void reduce_parts(int nv, int nblk, const double *part, double *out, const int *cond, cudaStream_t s,
                         const int *jd = nullptr, int extra = 0) {
  int cover = jd ? ORTHO_MAXV + 1 : nv;        // graph replay: enough warps for any step
  k_reduce_parts<<<(cover + 3) / 4, 128, 0, s>>>(nv, nblk, part, out, cond, jd, extra);
}
// flag = ||w_1||^2 < 1e-4 ||w||^2 (the first pass kept less than 1% of w)
__global__ void k_dgks(const double *w2_before, const double *w2_after, int *flag, const double *h1, const int *jd) {
  if (jd) w2_before = h1 + *jd + 1;            // ||w||^2 follows the step's dot products
  *flag = (*w2_after < 1e-4 * *w2_before) ? 1 : 0;
}

// Hessenberg column j: h = h1 + h2, h_{j+1,j} = ||w||; previous Givens
// rotations, a new one, and the residual estimate |g_{j+1}|.
// G layout: [0..m*(m+1)) H column-major (m+1 per column), cs[m], sn[m], g[m+1]
__global__ void k_arnoldi_col(int j, int m, const double *h1, const double *h2, const double *nrm_a,
                              const double *nrm_b, const int *flag, double *G, double *hnorm, volatile double *host,
                              const int *jd, float *isp) {
  // one warp: the column's inputs and the previous rotations are loaded
  // into shared memory in parallel, then lane 0 applies the rotations (a
  // serial recurrence) from there
  __shared__ double sc[ORTHO_MAXV + 1], scs[ORTHO_MAXV], ssn[ORTHO_MAXV];
  if (jd) { j = *jd; host += 4 * j; }          // graph replay: pinned slot j
  double *H = G, *cs = G + (size_t)m * (m + 1), *sn = cs + m, *g = sn + m;
  double *col = H + (size_t)j * (m + 1);
  const int lane = threadIdx.x;
  bool re = *flag != 0;
  for (int k = lane; k <= j; k += 32) sc[k] = re ? h1[k] + h2[k] : h1[k];
  for (int k = lane; k < j; k += 32) { scs[k] = cs[k]; ssn[k] = sn[k]; }
  __syncwarp();
  if (lane != 0) return;
  double hn = sqrt(re ? *nrm_b : *nrm_a);
  hnorm[0] = hn;
  hnorm[1] = hn > 0.0 ? 1.0 / hn : 0.0;
  if (isp) { float a, b; df_split(hnorm[1], a, b); isp[0] = a; isp[1] = b; }
  sc[j + 1] = 0.0;
  for (int k = 0; k < j; k++) {
    double t = scs[k] * sc[k] + ssn[k] * sc[k + 1];
    sc[k + 1] = -ssn[k] * sc[k] + scs[k] * sc[k + 1];
    sc[k] = t;
  }
  double rr = sqrt(sc[j] * sc[j] + hn * hn);
  double cj = sc[j] / rr, sj = hn / rr;
  cs[j] = cj; sn[j] = sj;
  for (int k = 0; k < j; k++) col[k] = sc[k];
  col[j] = rr; col[j + 1] = 0.0;
  double gj = g[j];
  g[j + 1] = -sj * gj;
  g[j] = cj * gj;
  host[0] = fabs(g[j + 1]);
  host[1] = hn;
  host[2] = re ? 1.0 : 0.0;
}
__global__ void k_scale(int nu, const double *w, const double *inv_hn, double *v, const int *jd) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (jd) v += (size_t)(*jd + 1) * nu;     // graph replay: v is the basis, the target is V_{j+1}
  if (i < nu) v[i] = w[i] * *inv_hn;       // 1 / h_{j+1,j} formed once by k_arnoldi_col
}
// graph replay helpers: the step's basis vector in and preconditioned vector out
// of fixed buffers, and the step counter
__global__ void k_basis_get(int nu, const double *V, const int *jd, double *vcur) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nu) vcur[i] = V[(size_t)*jd * nu + i];
}
template <class T>
__global__ void k_basis_put(int nu, const T *zcur, T *Z, const int *jd) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nu) Z[(size_t)*jd * nu + i] = zcur[i];
}
__global__ void k_step_inc(int *jd) { (*jd)++; }
__global__ void k_start(int nu, const double *r, double beta, double *v0, double *G, int m) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nu) v0[i] = r[i] * (1.0 / beta);
  if (i == 0) { double *g = G + (size_t)m * (m + 1) + 2 * m; for (int k = 0; k <= m; k++) g[k] = 0.0; g[0] = beta; }
}
__global__ void k_hsolve(int jend, int m, const double *G, double *yk) {
  const double *H = G, *g = G + (size_t)m * (m + 1) + 2 * m;
  for (int k = jend - 1; k >= 0; k--) {
    double s = g[k];
    for (int l = k + 1; l < jend; l++) s -= H[(size_t)l * (m + 1) + k] * yk[l];
    yk[k] = s / H[(size_t)k * (m + 1) + k];
  }
}
template <class Tz>
__global__ void k_xupdate(int nu, int jend, const double *yk, const Tz *Z, double *x) {
  __shared__ double sy[ORTHO_MAXV];
  for (int k = threadIdx.x; k < jend; k += blockDim.x) sy[k] = yk[k];
  __syncthreads();
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nu) return;
  double s = 0.0;
  for (int k = 0; k < jend; k++) s += sy[k] * (double)Z[(size_t)k * nu + i];
  x[i] += s;
}

// ------------------------------------------------------------ BiCGSTAB ---
// Right-preconditioned BiCGSTAB (van der Vorst), the paper's other Krylov
// method (its Examples 3, 6 and 7): two CPR applications per iteration.
// FP64 vectors throughout; in mixed precision the preconditioner returns an
// FP32 vector, widened to FP64 before its product with A.
__global__ void k_bcg_p(int nu, const double *r, const double *v, double beta, double omega, double *p) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nu) p[i] = r[i] + beta * (p[i] - omega * v[i]);
}
__global__ void k_bcg_s(int nu, const double *r, const double *v, double alpha, double *s) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nu) s[i] = r[i] - alpha * v[i];
}
__global__ void k_bcg_xr(int nu, double alpha, const double *ph, double omega, const double *sh, const double *s,
                         const double *t, double *x, double *r) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nu) { x[i] += alpha * ph[i] + omega * sh[i]; r[i] = s[i] - omega * t[i]; }
}
__global__ void k_bcg_xa(int nu, double alpha, const double *ph, double *x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nu) x[i] += alpha * ph[i];
}
__global__ void k_widen(int nu, const float *a, double *b) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nu) b[i] = (double)a[i];
}

// z = M^-1 v (CPR-FPF) in FP64
static void bcg_precond(sim_ls_s *ls, const double *v, double *z) {
  int nu = 2 * ls->nb;
  if (ls->o.precision != SIM_PREC_FP64) {
    ls_cpr(ls, v, nullptr, ls->bcg32.p);
    k_widen<<<grid_for(nu, 256), 256, 0, ls->st>>>(nu, ls->bcg32.p, z);
    RS_LAUNCHED(1);
  } else {
    ls_cpr(ls, v, z, nullptr);
  }
}

// Solves A M^-1 u = b, x = M^-1 u, from x = 0 or from the initial guess in
// ls->y (x0; the solution is left in ls->y).  Stops
// when the recursive residual meets tol ||b||, then checks the true residual
// b - A x; when that misses the tolerance, or on a breakdown (rho, (rh, v)
// or omega zero), it restarts from the true residual with rh = r.  At most
// max_lin iterations.  0 = converged, 1 = iteration cap, 2 = non-finite.
static int ls_solve_bicgstab(sim_ls_s *ls, double tol, int *its_out, double *relres, bool x0) {
  cudaStream_t st = ls->st;
  int nu = 2 * ls->nb, maxit = ls->o.max_lin, its = 0, rc = 1;
  ls->bcg.ensure(8 * (size_t)nu);
  if (ls->o.precision != SIM_PREC_FP64) ls->bcg32.ensure(nu);
  double *rh = ls->bcg.p, *p = rh + nu, *v = p + nu, *sv = v + nu, *t = sv + nu, *ph = t + nu, *sh = ph + nu;
  double *x = ls->y.p, *r = ls->r.p;
  unsigned g = grid_for(nu, 256);
  double bn = rs_norm2(ls->b.p, nu, st), rn = bn;
  if (bn == 0.0) { rs_fill_d(x, 0.0, nu, st); *its_out = 0; *relres = 0.0; return 0; }
  if (!std::isfinite(bn)) { rs_fill_d(x, 0.0, nu, st); *its_out = 0; *relres = NAN; return 2; }
  if (x0) {                                   // r = b - A x0
    spmv<double, double, double, double>(ls, ls->val.p, x, ls->b.p, r, st);
    rn = rs_norm2(r, nu, st);
  }
  if (!x0 || !std::isfinite(rn)) {
    rs_fill_d(x, 0.0, nu, st);
    RS_CUDA(cudaMemcpyAsync(r, ls->b.p, nu * sizeof(double), cudaMemcpyDeviceToDevice, st));
    rn = bn;
  }
  if (rn <= tol * bn) { *its_out = 0; *relres = rn / bn; return 0; }
  auto check = [&]() {
    if (ls->errw[0]) RS_FAIL(SIM_ERR_TIMEOUT, "RAS apply: bulk copy wait gave up (code %d)", ls->errw[0]);
  };
  for (;;) {
    RS_CUDA(cudaMemcpyAsync(rh, r, nu * sizeof(double), cudaMemcpyDeviceToDevice, st));
    rs_fill_d(p, 0.0, nu, st); rs_fill_d(v, 0.0, nu, st);
    double rho_prev = 1.0, alpha = 1.0, omega = 1.0;
    bool broke = false, done = false;
    while (its < maxit) {
      double rho;
      { const double *xs[1] = {rh}, *ys[1] = {r}; rs_dots(xs, ys, 1, nu, &rho, st); }
      if (!std::isfinite(rho)) { *its_out = its; *relres = NAN; return 2; }
      if (rho == 0.0) { broke = true; break; }
      double beta = (rho / rho_prev) * (alpha / omega);
      k_bcg_p<<<g, 256, 0, st>>>(nu, r, v, beta, omega, p);
      RS_LAUNCHED(1);
      bcg_precond(ls, p, ph);
      ls_spmv64(ls, ph, v);
      double rv;
      { const double *xs[1] = {rh}, *ys[1] = {v}; rs_dots(xs, ys, 1, nu, &rv, st); }
      check();
      if (!std::isfinite(rv)) { *its_out = its; *relres = NAN; return 2; }
      if (rv == 0.0) { broke = true; break; }
      alpha = rho / rv;
      k_bcg_s<<<g, 256, 0, st>>>(nu, r, v, alpha, sv);
      RS_LAUNCHED(1);
      its++;
      double sn = rs_norm2(sv, nu, st);
      if (!std::isfinite(sn)) { *its_out = its; *relres = NAN; return 2; }
      if (sn <= tol * bn) {
        k_bcg_xa<<<g, 256, 0, st>>>(nu, alpha, ph, x);
        RS_LAUNCHED(1);
        done = true;
        break;
      }
      bcg_precond(ls, sv, sh);
      ls_spmv64(ls, sh, t);
      double tt_ts[2];
      { const double *xs[2] = {t, t}, *ys[2] = {t, sv}; rs_dots(xs, ys, 2, nu, tt_ts, st); }
      check();
      omega = tt_ts[0] > 0.0 ? tt_ts[1] / tt_ts[0] : 0.0;
      k_bcg_xr<<<g, 256, 0, st>>>(nu, alpha, ph, omega, sh, sv, t, x, r);
      RS_LAUNCHED(1);
      rn = rs_norm2(r, nu, st);
      if (!std::isfinite(rn)) { *its_out = its; *relres = NAN; return 2; }
      if (rn <= tol * bn) { done = true; break; }
      if (omega == 0.0) { broke = true; break; }
      rho_prev = rho;
    }
    // true residual r = b - A x
    spmv<double, double, double, double>(ls, ls->val.p, x, ls->b.p, r, st);
    rn = rs_norm2(r, nu, st);
    ls->timer_flush();
    if (!std::isfinite(rn)) { rc = 2; break; }
    if (rn <= tol * bn) { rc = 0; break; }
    if (its >= maxit) { rc = 1; break; }
    if (!done && !broke) { rc = 1; break; }
  }
  *its_out = its;
  *relres = rc == 2 ? NAN : rn / bn;
  return rc;
}

// End of one Arnoldi step inside the device-side loop: continue the cycle
// while the step's residual estimate is finite and above the threshold, its
// h_{j+1,j} is not zero and the cycle has steps left (at most the restart
// length, so the loop always ends); record the steps done and whether a
// non-finite value appeared.  lp = {threshold, step cap, steps done, flag}.
__global__ void k_loop_cond(cudaGraphConditionalHandle h, const int *jd, const double *hp, double *lp) {
  int j = *jd - 1;                                   // the step just done (jd already advanced)
  double est = hp[4 * j], hn = hp[4 * j + 1];
  bool bad = !isfinite(est) || !isfinite(hn);
  bool more = !bad && est > lp[0] && (double)(j + 1) < lp[1] && hn != 0.0;
  lp[2] = (double)(j + 1);
  lp[3] = bad ? 1.0 : 0.0;
  cudaGraphSetConditional(h, more ? 1u : 0u);
}
__global__ void k_loop_params(double *lp, double thr, double cap) { lp[0] = thr; lp[1] = cap; lp[2] = 0.0; lp[3] = 0.0; }

int ls_solve(sim_ls_s *ls, double tol, int *its_out, double *relres, bool x0) {
  if (ls->o.krylov == SIM_KRYLOV_BICGSTAB) return ls_solve_bicgstab(ls, tol, its_out, relres, x0);
  cudaStream_t s = ls->st;
  int nu = 2 * ls->nb, m = std::min(ls->o.restart, ORTHO_MAXV - 1), maxit = ls->o.max_lin;
  // df: double-float Arnoldi basis (its kernels use 32-bit offsets into the
  // 2 (m + 1) nu floats of the basis; larger systems keep the FP64 basis)
  bool mixed = ls->o.precision != SIM_PREC_FP64;
  bool df = mixed && !ls->o.fp64_basis && 2.0 * (m + 1) * (double)nu < 2147483647.0;
  ls->V.ensure((size_t)(m + 1) * nu);
  if (mixed) ls->Z32.ensure((size_t)m * nu); else ls->Z.ensure((size_t)m * nu);
  int chd = 0, nblk = df ? ortho_blocks_df(nu, &chd) : ortho_blocks(nu);
  ls->partial.ensure((size_t)(ORTHO_MAXV + 1) * nblk + 8);
  ls->hbuf.ensure((size_t)(m + 1) * (m + 1) + 4 * (m + 1) + 4 * ORTHO_MAXV + 16);
  double *G = ls->hbuf.p, *h1 = G + (size_t)(m + 1) * (m + 1) + 3 * (m + 1), *h2 = h1 + ORTHO_MAXV + 1,
         *nrm = h2 + ORTHO_MAXV, *nrm_b = nrm + 1, *hn = nrm_b + 1, *yk = hn + 2;
  int *flag = reinterpret_cast<int *>(yk + ORTHO_MAXV);
  volatile double *hp = ls->hpin;
  double *hp_dev;
  RS_CUDA(cudaHostGetDevicePointer((void **)&hp_dev, ls->hpin, 0));
  double bn = rs_norm2(ls->b.p, nu, s);
  if (bn == 0.0) { rs_fill_d(ls->y.p, 0.0, nu, s); *its_out = 0; *relres = 0.0; return 0; }
  if (!std::isfinite(bn)) { rs_fill_d(ls->y.p, 0.0, nu, s); *its_out = 0; *relres = NAN; return 2; }
  double beta = bn;
  if (x0) {                      // initial guess in y: r = b - A y
    spmv<double, double, double, double>(ls, ls->val.p, ls->y.p, ls->b.p, ls->r.p, s);
    beta = rs_norm2(ls->r.p, nu, s);
  }
  if (!x0 || !std::isfinite(beta)) {
    rs_fill_d(ls->y.p, 0.0, nu, s);
    RS_CUDA(cudaMemcpyAsync(ls->r.p, ls->b.p, nu * sizeof(double), cudaMemcpyDeviceToDevice, s));
    beta = bn;
  }
  if (beta <= tol * bn) { *its_out = 0; *relres = beta / bn; return 0; }
  int its = 0, rc = 1;
  // Orthogonalisation of w against V_0..V_j (classical Gram-Schmidt with a
  // second pass under cancellation), the Hessenberg column with its Givens
  // rotations, and V_{j+1}.  jdp: the step index is read on the device (graph
  // replay) instead of j.  Mixed precision: double-float planes.
  float *V32 = reinterpret_cast<float *>(ls->V.p);
  if (df) {
    ls->w2.ensure(2 * (size_t)nu); ls->isp.ensure(2);
    if (!ls->ticket.p) { ls->ticket.ensure(1); RS_CUDA(cudaMemsetAsync(ls->ticket.p, 0, sizeof(int), s)); }
  }
  auto ortho_tail = [&](cudaStream_t c, int j, const int *jdp) {
    int nv = jdp ? 0 : j + 1;
    double *part = ls->partial.p;
    if (df) {
      float *w2 = ls->w2.p;                    // written by the double-float SpMV
      // the reductions, and the test for a second pass, run in the last
      // block of each sweep
      int *tk = ls->ticket.p;
      ortho_dots_df(nu, chd, nv, V32, w2, part, 1, nullptr, nblk, c, jdp, tk, h1);   // h1[nv] = ||w||^2
      ortho_update_df(nu, chd, nv, V32, w2, h1, part, nullptr, nblk, c, jdp, tk, nrm, flag, h1);
      ortho_dots_df(nu, chd, nv, V32, w2, part, 0, flag, nblk, c, jdp, tk, h2);
      ortho_update_df(nu, chd, nv, V32, w2, h2, part, flag, nblk, c, jdp, tk, nrm_b, nullptr, nullptr);
      k_arnoldi_col<<<1, 32, 0, c>>>(j, m, h1, h2, nrm, nrm_b, flag, G, hn, jdp ? hp_dev : hp_dev + 4 * j, jdp,
                                    ls->isp.p);
      k_scale_df<<<grid_for(nu, 256), 256, 0, c>>>(nu, w2, ls->isp.p, V32, j + 1, jdp, jdp ? ls->vcur32.p : nullptr);
      RS_LAUNCHED(6);
    } else {
      ortho_dots(nu, nv, ls->V.p, ls->w.p, part, 1, nullptr, nblk, c, jdp);
      reduce_parts(nv + 1, nblk, part, h1, nullptr, c, jdp, 1);
      ortho_update(nu, nv, ls->V.p, ls->w.p, h1, part, nullptr, nblk, c, jdp);
      reduce_parts(1, nblk, part, nrm, nullptr, c);
      k_dgks<<<1, 1, 0, c>>>(h1 + nv, nrm, flag, h1, jdp);
      ortho_dots(nu, nv, ls->V.p, ls->w.p, part, 0, flag, nblk, c, jdp);
      reduce_parts(nv, nblk, part, h2, flag, c, jdp, 0);
      ortho_update(nu, nv, ls->V.p, ls->w.p, h2, part, flag, nblk, c, jdp);
      reduce_parts(1, nblk, part, nrm_b, flag, c);
      k_arnoldi_col<<<1, 32, 0, c>>>(j, m, h1, h2, nrm, nrm_b, flag, G, hn, jdp ? hp_dev : hp_dev + 4 * j, jdp,
                                    nullptr);
      k_scale<<<grid_for(nu, 256), 256, 0, c>>>(nu, ls->w.p, hn + 1, jdp ? ls->V.p : ls->V.p + (size_t)(j + 1) * nu,
                                                jdp);
      RS_LAUNCHED(11);
    }
  };
  // One Arnoldi step j (CPR, SpMV, orthogonalisation, Givens); its residual
  // estimate and h_{j+1,j} land in pinned slot j
  auto enqueue = [&](int j) {
    if (df) {
      float *zj = ls->Z32.p + (size_t)j * nu;
      ls_cpr32(ls, V32 + (size_t)(2 * j) * nu, zj);
      rs_timed tm(ls, SIM_T_SPMV64);
      spmv_df(ls, zj, ls->w2.p, s);
    } else if (mixed) {          // FP64 basis with the FP32 preconditioner
      float *zj = ls->Z32.p + (size_t)j * nu;
      ls_cpr(ls, ls->V.p + (size_t)j * nu, nullptr, zj);
      rs_timed tm(ls, SIM_T_SPMV64);
      spmv<double, float, double, double>(ls, ls->val.p, zj, (const double *)nullptr, ls->w.p, s);
    } else {
      double *zj = ls->Z.p + (size_t)j * nu;
      ls_cpr(ls, ls->V.p + (size_t)j * nu, zj, nullptr);
      ls_spmv64(ls, zj, ls->w.p);
    }
    {
      rs_timed tm(ls, SIM_T_ORTHO);
      ortho_tail(s, j, nullptr);
    }
    RS_CHECK_LAUNCH();
  };
  // The same Arnoldi step as one CUDA graph, replayed for every j: the step
  // index lives on the device (jd), the basis vector is copied into a fixed
  // buffer and the preconditioned vector out of one, and the kernels that
  // depend on j read it from jd.  Recorded once per setup (the hierarchy's
  // buffers may move at a setup); kernel timers become event nodes of the
  // graph, read after each replay.
  // The recording holds raw pointers: record again whenever one of the
  // solver's own buffers, the restart length or the precision has changed.
  bool use_graph = ls->graph_mode > 0 && ls->ras.smem_path;
  // the device-side loop needs a body without timer event nodes
  bool use_loop = use_graph && ls->graph_mode == 2 && ls->timer_mask == 0;
  const void *sig[10] = {ls->V.p, ls->Z.p, ls->Z32.p, ls->w.p, ls->partial.p, ls->hbuf.p,
                         (const void *)(size_t)m, (const void *)(size_t)ls->o.precision,
                         (const void *)(size_t)ls->timer_mask, ls->w2.p};
  if (use_graph && ls->it_exec && memcmp(sig, ls->it_sig, sizeof(sig)) != 0) ls->drop_graph();
  // one Arnoldi step recorded on stream c (the capture stream)
  auto record_step = [&](cudaStream_t c) {
      const int *jd = ls->jd.p;
      if (df) {                              // vcur32 holds v_j (k_start_df, k_scale_df)
        ls_cpr32(ls, ls->vcur32.p, ls->zcur32.p);
        {
          rs_timed tm(ls, SIM_T_SPMV64);
          spmv_df(ls, ls->zcur32.p, ls->w2.p, c);
        }
        k_basis_put<float><<<grid_for(nu, 256), 256, 0, c>>>(nu, ls->zcur32.p, ls->Z32.p, jd);
      } else if (mixed) {
        k_basis_get<<<grid_for(nu, 256), 256, 0, c>>>(nu, ls->V.p, jd, ls->vcur.p);
        ls_cpr(ls, ls->vcur.p, nullptr, ls->zcur32.p);
        {
          rs_timed tm(ls, SIM_T_SPMV64);
          spmv<double, float, double, double>(ls, ls->val.p, ls->zcur32.p, (const double *)nullptr, ls->w.p, c);
        }
        k_basis_put<float><<<grid_for(nu, 256), 256, 0, c>>>(nu, ls->zcur32.p, ls->Z32.p, jd);
      } else {
        k_basis_get<<<grid_for(nu, 256), 256, 0, c>>>(nu, ls->V.p, jd, ls->vcur.p);
        ls_cpr(ls, ls->vcur.p, ls->zcur64.p, nullptr);
        ls_spmv64(ls, ls->zcur64.p, ls->w.p);
        k_basis_put<double><<<grid_for(nu, 256), 256, 0, c>>>(nu, ls->zcur64.p, ls->Z.p, jd);
      }
      rs_timed tm(ls, SIM_T_ORTHO);
      ortho_tail(c, 0, jd);
      tm.stop();
      k_step_inc<<<1, 1, 0, c>>>(ls->jd.p);
      RS_LAUNCHED(df ? 2 : 3);
      RS_CHECK_LAUNCH();
  };
  if (use_graph && !ls->it_exec) {
    ls->drop_graph();
    ortho_attr();
    ls->jd.ensure(1);
    if (df) ls->vcur32.ensure(nu); else ls->vcur.ensure(nu);
    if (mixed) ls->zcur32.ensure(nu); else ls->zcur64.ensure(nu);
    if (!ls->cap) RS_CUDA(cudaStreamCreateWithFlags(&ls->cap, cudaStreamNonBlocking));
    cudaStream_t keep = ls->st;
    cudaGraph_t g = nullptr;
    RS_CUDA(cudaStreamBeginCapture(ls->cap, cudaStreamCaptureModeRelaxed));
    ls->st = ls->cap;
    ls->capturing = true;
    try {
      record_step(ls->cap);
    } catch (...) {
      ls->st = keep; ls->capturing = false;
      cudaStreamEndCapture(ls->cap, &g);
      if (g) cudaGraphDestroy(g);
      ls->drop_graph();
      throw;
    }
    ls->st = keep;
    ls->capturing = false;
    RS_CUDA(cudaStreamEndCapture(ls->cap, &g));
    // kernels recorded (counted by the node list: other handles may launch
    // concurrently, so the global counter's difference is not this graph's)
    size_t nn = 0;
    cudaError_t e = cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    long long nk = 0;
    if (e == cudaSuccess && nn) e = cudaGraphGetNodes(g, nodes.data(), &nn);
    for (size_t q = 0; e == cudaSuccess && q < nn; q++) {
      cudaGraphNodeType t;
      e = cudaGraphNodeGetType(nodes[q], &t);
      if (t == cudaGraphNodeTypeKernel) nk++;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ls->it_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { ls->it_exec = nullptr; ls->drop_graph(); RS_CUDA(e); }
    memcpy(ls->it_sig, sig, sizeof(sig));
    ls->it_launches = nk;
    rs_launches -= (unsigned long long)nk;             // recorded, not launched
  }
  // The same step as the body of a graph WHILE node, ended by k_loop_cond:
  // a whole cycle of Arnoldi steps runs from one launch, and the host waits
  // once per cycle instead of once per step.
  if (use_loop && !ls->loop_exec && ls->loop_state == 0) {
    // first with the kernels' programmatic-launch edges, else with plain
    // edges; a driver that records neither leaves the per-step graph in use
    ls->loopd.ensure(4);
    cudaStream_t keep = ls->st;
    for (int attempt = 0; attempt < 2 && !ls->loop_exec; attempt++) {
      cudaGraph_t g = nullptr;
      bool ok = cudaGraphCreate(&g, 0) == cudaSuccess;
      rs_pdl_off = attempt == 1;
      try {
        cudaGraphConditionalHandle hc;
        cudaGraphNodeParams np = {};
        cudaGraphNode_t node;
        ok = ok && cudaGraphConditionalHandleCreate(&hc, g, 1, cudaGraphCondAssignDefault) == cudaSuccess;
        if (ok) {
          np.type = cudaGraphNodeTypeConditional;
          np.conditional.handle = hc;
          np.conditional.type = cudaGraphCondTypeWhile;
          np.conditional.size = 1;
          ok = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np) == cudaSuccess;
        }
        ok = ok && cudaStreamBeginCaptureToGraph(ls->cap, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                 cudaStreamCaptureModeRelaxed) == cudaSuccess;
        if (ok) {
          ls->st = ls->cap;
          ls->capturing = true;
          try {
            record_step(ls->cap);
            k_loop_cond<<<1, 1, 0, ls->cap>>>(hc, ls->jd.p, hp_dev, ls->loopd.p);
            ok = cudaGetLastError() == cudaSuccess;
          } catch (...) {
            ok = false;
          }
          ls->st = keep;
          ls->capturing = false;
          cudaGraph_t gb = nullptr;
          ok = cudaStreamEndCapture(ls->cap, &gb) == cudaSuccess && ok;
        }
        ok = ok && cudaGraphInstantiate(&ls->loop_exec, g, 0) == cudaSuccess;
      } catch (...) {
        ok = false;
      }
      rs_pdl_off = false;
      ls->st = keep; ls->capturing = false;
      if (g) cudaGraphDestroy(g);
      if (!ok) {
        if (ls->loop_exec) cudaGraphExecDestroy(ls->loop_exec);
        ls->loop_exec = nullptr;
        (void)cudaGetLastError();                     // the failed recording's error is not sticky
      }
      rs_launches -= (unsigned long long)ls->it_launches;   // recorded, not launched
      ls->loop_state = ok ? attempt + 1 : -1;
    }
  }
  if (use_loop && !ls->loop_exec) use_loop = false;
  ls->last_mode = use_loop ? 2 : use_graph ? 1 : 0;
  for (;;) {
    if (df) k_start_df<<<grid_for(nu, 256), 256, 0, s>>>(nu, ls->r.p, beta, V32, G, m, use_graph ? ls->vcur32.p : nullptr);
    else k_start<<<grid_for(nu, 256), 256, 0, s>>>(nu, ls->r.p, beta, ls->V.p, G, m);
    RS_LAUNCHED(1);
    int jend = 0;
    if (use_graph) RS_CUDA(cudaMemsetAsync(ls->jd.p, 0, sizeof(int), s));
    if (use_loop) {
      // the cycle on the device: at most min(m, max_lin - its) steps
      k_loop_params<<<1, 1, 0, s>>>(ls->loopd.p, tol * bn, (double)std::min(m, maxit - its));
      RS_CUDA(cudaGraphLaunch(ls->loop_exec, s));
      std::vector<double> lo = d2h(ls->loopd.p + 2, 2, s);
      if (ls->errw[0]) RS_FAIL(SIM_ERR_TIMEOUT, "RAS apply: bulk copy wait gave up (code %d)", ls->errw[0]);
      jend = (int)lo[0];
      its += jend;
      RS_LAUNCHED(1 + (long long)jend * (ls->it_launches + 1));
      if (lo[1] != 0.0) { *its_out = its; *relres = NAN; return 2; }
    }
    for (int j = 0; j < m && !use_loop; j++) {
      if (use_graph) {
        RS_CUDA(cudaGraphLaunch(ls->it_exec, s));
        RS_LAUNCHED(ls->it_launches);
      } else {
        enqueue(j);
      }
      RS_CUDA(cudaStreamSynchronize(s));
      if (use_graph) ls->graph_timers();
      if (ls->errw[0]) RS_FAIL(SIM_ERR_TIMEOUT, "RAS apply: bulk copy wait gave up (code %d)", ls->errw[0]);
      double est = hp[4 * j], hnv = hp[4 * j + 1];
      its++;
      jend = j + 1;
      if (!std::isfinite(est) || !std::isfinite(hnv)) { *its_out = its; *relres = NAN; return 2; }
      if (est <= tol * bn || its >= maxit || hnv == 0.0) break;
    }
    k_hsolve<<<1, 1, 0, s>>>(jend, m, G, yk);
    if (mixed) k_xupdate<float><<<grid_for(nu, 256), 256, 0, s>>>(nu, jend, yk, ls->Z32.p, ls->y.p);
    else k_xupdate<double><<<grid_for(nu, 256), 256, 0, s>>>(nu, jend, yk, ls->Z.p, ls->y.p);
    RS_LAUNCHED(2);
    spmv<double, double, double, double>(ls, ls->val.p, ls->y.p, ls->b.p, ls->r.p, s);   // true residual
    beta = rs_norm2(ls->r.p, nu, s);
    ls->timer_flush();
    if (!std::isfinite(beta)) { rc = 2; break; }
    if (beta <= tol * bn) { rc = 0; break; }
    if (its >= maxit) { rc = 1; break; }
  }
  *its_out = its;
  *relres = beta / bn;
  return rc;
}

// ------------------------------------------------ residual norm (API) ----
// ||b - A x||_2: residual vector in a library-owned buffer, then the
// deterministic two-stage sum of squares.
double ls_residual_norm(sim_ls_s *ls, const double *x_dev) {
  size_t nu = 2 * (size_t)ls->nb;
  ls->r.ensure(nu);
  spmv<double, double, double, double>(ls, ls->val.p, x_dev, ls->b.p, ls->r.p, ls->st);
  return rs_norm2(ls->r.p, (int)nu, ls->st);
}
