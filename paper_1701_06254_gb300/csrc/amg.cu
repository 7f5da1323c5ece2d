// Algebraic multigrid on the pressure block A_pp: the M(A_pp)^{-1} stage of
// CPR-FPF (the pressure stage of Algorithm 2) of arXiv 1701.06254.  The paper fixes no AMG
// component; this library uses
//   strength   S_i = { j != i : -a_ij >= theta * max_{k != i}(-a_ik) }
//   coarsening PMIS with weights |S^T_i| + h(i), h = splitmix64 hash in [0,1)
//   interpolation direct (positive off-diagonals lumped into the diagonal)
//                 or extended+i (distance two, option interp),
//              R = P^T, Galerkin A_c = R (A P)
//   cycle      V(1,1), l1-Jacobi smoothing, zero initial guess
//   coarsest   dense inverse (FP64): LU with partial pivoting in shared
//              memory, then the columns of the inverse in parallel (n <=
//              128), else an LU with partial pivoting in one block
// Setup runs in FP64 with explicit round-to-nearest operations in a fixed
// order, so the C/F split, P and every coarse operator are bit-identical to
// a plain sequential evaluation of the same formulas on the same input.
#include "common.cuh"
#include <algorithm>
#include <climits>

// ------------------------------------------------------------ pattern -----
__global__ void k_tpos(int n, const int *rp, const int *ci, int *tpos, int *err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int q = rp[i]; q < rp[i + 1]; q++) {
    int j = ci[q], lo = rp[j], hi = rp[j + 1] - 1, pos = -1;
    while (lo <= hi) {
      int mid = (lo + hi) >> 1, c = ci[mid];
      if (c == i) { pos = mid; break; }
      if (c < i) lo = mid + 1; else hi = mid - 1;
    }
    if (pos < 0) atomicExch(err, 1);       // pattern not structurally symmetric
    tpos[q] = pos < 0 ? q : pos;
  }
}

// the same with one warp per row (levels with long rows: a thread walking
// 40 binary searches one after another was latency-bound)
__global__ void k_tpos_warp(int n, const int *rp, const int *ci, int *tpos, int *err) {
  int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (i >= n) return;
  for (int q = rp[i] + lane; q < rp[i + 1]; q += 32) {
    int j = ci[q], lo = rp[j], hi = rp[j + 1] - 1, pos = -1;
    while (lo <= hi) {
      int mid = (lo + hi) >> 1, c = ci[mid];
      if (c == i) { pos = mid; break; }
      if (c < i) lo = mid + 1; else hi = mid - 1;
    }
    if (pos < 0) atomicExch(err, 1);
    tpos[q] = pos < 0 ? q : pos;
  }
}

// Strength of connection (S), and with dinv given the l1-Jacobi diagonal of
// the same row (d_i = a_ii + sum_{j != i} |a_ij|; 1 / d_i, FP64 and FP32),
// from one pass over the row.
__global__ void k_strength(int n, const int *rp, const int *ci, const double *v, double theta, uint8_t *S,
                           double *dinv, float *dinv32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  bool have = false; double mx = 0.0; long long mxk = 0;
  double s = 0.0, aii = 0.0;
  for (int q = rp[i]; q < rp[i + 1]; q++) {
    const double a = v[q];
    if (ci[q] == i) { aii = a; continue; }
    s = add_rn(s, fabs(a));
    long long tk = -dkey(a);                        // key of t = -a_iq
    if (!have || tk > mxk) { mx = -a; mxk = tk; have = true; }
  }
  long long thrk = dkey(mul_rn(theta, mx));
  bool any = have && mxk > 0;                       // max_k (-a_ik) > 0
  for (int q = rp[i]; q < rp[i + 1]; q++)
    S[q] = (uint8_t)(any && ci[q] != i && -dkey(v[q]) >= thrk);
  if (dinv) {
    double d = add_rn(aii, s);
    dinv[i] = 1.0 / d;
    if (dinv32) dinv32[i] = (float)(1.0 / d);
  }
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

// Append i to a list when `on` (one atomic per warp: the warp's entries get
// consecutive slots in lane order; the list's order is arbitrary and no
// result depends on it).  Every lane of the warp must call it.
__device__ __forceinline__ void warp_append(bool on, int i, int *count, int *list) {
  unsigned m = __ballot_sync(0xffffffffu, on);
  int lane = threadIdx.x & 31, base = 0;
  if (lane == 0 && m) base = atomicAdd(count, __popc(m));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (on) list[base + __popc(m & ((1u << lane) - 1u))] = i;
}

__global__ void k_pmis_init(int n, const int *rp, const int *ci, const uint8_t *S, const int *tpos,
                            uint64_t seed, int level, double *w, int8_t *cf, int8_t *newc, int *undecided,
                            int *list) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  int cnt = 0;
  if (i < n) {
    const int q1 = rp[i + 1];
    for (int q0 = rp[i]; q0 < q1; q0 += 4) {       // |S^T_i|, four entries' loads at a time
      int jj[4], tp[4];
#pragma unroll
      for (int u = 0; u < 4; u++) { const bool in = q0 + u < q1; jj[u] = in ? ci[q0 + u] : i; tp[u] = in ? tpos[q0 + u] : 0; }
#pragma unroll
      for (int u = 0; u < 4; u++) cnt += jj[u] != i && S[tp[u]];
    }
    uint64_t z = splitmix64(seed ^ ((uint64_t)level << 40) ^ (uint64_t)(uint32_t)i);
    double h = (double)(z >> 11) * (1.0 / 9007199254740992.0);
    w[i] = add_rn((double)cnt, h);
    cf[i] = cnt == 0 ? (int8_t)-1 : (int8_t)0;
    newc[i] = 0;                       // no candidate flag left over from another level or setup
  }
  warp_append(i < n && cnt != 0, i, undecided, list);
}

// One PMIS round over the undecided points only: list (cnt[r] entries) ->
// next (cnt[r + 1] entries).  A round whose list is empty does nothing, so
// rounds launched past the last one cost a launch each.  L lanes per point
// (1 for short rows; 4 or 16 split a row's entries, verdicts combined by
// ballots); the grid strides over the list.
//   select: an undecided point is a candidate unless an undecided strong
//           neighbour (in S or S^T) has a larger weight (ties: lower index);
//   update: candidates become C; an undecided point with a strong (S)
//           neighbour that is C or a candidate becomes F; the rest stay
//           undecided and go to the next list.
// Weights are >= +0, so their bit patterns order them.  newc of a point that
// left the lists keeps its last value: 1 only for C points, which the update
// test also finds through cf.
// the two steps of one round over list entries g0, g0 + stride, ... (L
// lanes per point; every lane of a warp runs the loop to its common end)
#define PMIS_B 4
template <int L>
__device__ __forceinline__ void pmis_select_pts(const int *rp, const int *ci, const uint8_t *S, const int *tpos,
                                                const double *w, const int8_t *cf, int8_t *newc, const int *list,
                                                int m, int g_first, int stride) {
  const int k = threadIdx.x % L;
  for (int g0 = g_first;; g0 += stride) {
    if (__all_sync(0xffffffffu, g0 >= m)) break;
    int g = g0 < m ? g0 : m - 1, i = list[g];
    bool beaten = false;
    const long long wi = __double_as_longlong(w[i]);
    const int q1 = rp[i + 1];
    // PMIS_B entries of the lane at a time, their loads issued together (two
    // dependent levels instead of a chain per entry)
    for (int q0 = rp[i] + k; q0 < q1 && !beaten; q0 += PMIS_B * L) {
      int jj[PMIS_B], tp[PMIS_B]; bool sq[PMIS_B];
#pragma unroll
      for (int u = 0; u < PMIS_B; u++) {
        const int q = q0 + u * L; const bool in = q < q1;
        jj[u] = in ? ci[q] : i; sq[u] = in && S[q]; tp[u] = in ? tpos[q] : 0;
      }
#pragma unroll
      for (int u = 0; u < PMIS_B; u++) {
        const int j = jj[u];
        if (j == i) continue;
        const bool st = sq[u] || S[tp[u]];
        const int8_t c = cf[j];
        const long long wj = __double_as_longlong(w[j]);
        beaten |= st && c == 0 && (wj > wi || (wj == wi && j < i));
      }
    }
    if (L > 1) {
      unsigned lanes = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << ((threadIdx.x & 31) / L * L));
      beaten = (__ballot_sync(0xffffffffu, beaten) & lanes) != 0;
    }
    if (k == 0 && g0 < m) newc[i] = beaten ? 0 : 1;
  }
}
template <int L>
__device__ __forceinline__ void pmis_update_pts(const int *rp, const int *ci, const uint8_t *S, int8_t *cf,
                                                const int8_t *newc, const int *list, int m, int g_first, int stride,
                                                int *next, int *cnt_next) {
  const int k = threadIdx.x % L;
  for (int g0 = g_first;; g0 += stride) {
    if (__all_sync(0xffffffffu, g0 >= m)) break;
    int g = g0 < m ? g0 : m - 1, i = list[g];
    bool sel = newc[i] != 0, hit = false;
    if (!sel) {
      const int q1 = rp[i + 1];
      for (int q0 = rp[i] + k; q0 < q1 && !hit; q0 += PMIS_B * L) {
        int jj[PMIS_B]; bool sq[PMIS_B];
#pragma unroll
        for (int u = 0; u < PMIS_B; u++) {
          const int q = q0 + u * L; const bool in = q < q1;
          jj[u] = in ? ci[q] : i; sq[u] = in && S[q];
        }
#pragma unroll
        for (int u = 0; u < PMIS_B; u++) {
          const int j = jj[u];
          hit |= sq[u] && (cf[j] == 1 || newc[j]);
        }
      }
    }
    if (L > 1) {
      unsigned lanes = (L == 32) ? 0xffffffffu : (((1u << L) - 1u) << ((threadIdx.x & 31) / L * L));
      hit = (__ballot_sync(0xffffffffu, hit) & lanes) != 0;
    }
    bool lead = k == 0 && g0 < m;
    if (lead && sel) cf[i] = 1;
    else if (lead && hit) cf[i] = -1;
    warp_append(lead && !sel && !hit, i, cnt_next, next);
  }
}

template <int L>
__global__ void k_pmis_select_w(const int *rp, const int *ci, const uint8_t *S, const int *tpos, const double *w,
                                const int8_t *cf, int8_t *newc, const int *list, const int *cnt) {
  int m = *cnt;
  if (m == 0) return;
  pmis_select_pts<L>(rp, ci, S, tpos, w, cf, newc, list, m, (blockIdx.x * blockDim.x + threadIdx.x) / L,
                     gridDim.x * blockDim.x / L);
}

template <int L>
__global__ void k_pmis_update_w(const int *rp, const int *ci, const uint8_t *S, int8_t *cf, const int8_t *newc,
                                const int *list, const int *cnt, int *next, int *cnt_next) {
  int m = *cnt;
  if (m == 0) return;
  pmis_update_pts<L>(rp, ci, S, cf, newc, list, m, (blockIdx.x * blockDim.x + threadIdx.x) / L,
                     gridDim.x * blockDim.x / L, next, cnt_next);
}

// Rounds r0, r0 + 1, ... until a list is empty, in one block: the same two
// steps per round with block barriers between them, for the short lists of
// the last rounds (a launch per step costs more than the step there).
// *z = the first round r whose list cnt[r] is empty (searched from 0), or
// -1 when rmax rounds were not enough.
template <int L>
__global__ void __launch_bounds__(1024) k_pmis_tail(const int *rp, const int *ci, const uint8_t *S, const int *tpos,
                                                    const double *w, int8_t *cf, int8_t *newc, int *plist, int n,
                                                    int *cnt, int r0, int rmax, int *z) {
  const volatile int *vcnt = cnt;
  __shared__ int zs;
  if (threadIdx.x == 0) {
    zs = -1;
    for (int r = 0; r <= r0; r++) if (vcnt[r] == 0) { zs = r; break; }
  }
  __syncthreads();
  if (zs >= 0) { if (threadIdx.x == 0) *z = zs; return; }
  const int first = threadIdx.x / L, stride = blockDim.x / L;
  for (int r = r0; r < rmax; r++) {
    const int m = vcnt[r];
    if (m == 0) { if (threadIdx.x == 0) *z = r; return; }
    const int *lst = plist + (size_t)(r & 1) * n;
    int *nxt = plist + (size_t)((r + 1) & 1) * n;
    pmis_select_pts<L>(rp, ci, S, tpos, w, cf, newc, lst, m, first, stride);
    __syncthreads();
    pmis_update_pts<L>(rp, ci, S, cf, newc, lst, m, first, stride, nxt, cnt + r + 1);
    __syncthreads();
  }
  if (threadIdx.x == 0) *z = vcnt[rmax] == 0 ? rmax : -1;
}

// lanes per row for the PMIS steps: one thread for short rows, then the
// V-cycle's counts (4 lanes for 9-24 entries, 16 beyond)
static int pmis_lanes(long long nnz, int n) {
  double avg = n ? (double)nnz / n : 0.0;
  return avg <= 8.0 ? 1 : avg <= 24.0 ? 4 : 16;
}

__global__ void k_cflag(int n, const int8_t *cf, int *flag) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) flag[i] = cf[i] == 1;
}

// ------------------------------------------------------- interpolation ----
__global__ void k_interp_count(int n, const int *rp, const int *ci, const uint8_t *S, const int8_t *cf, int *len) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = 0;
  if (cf[i] == 1) c = 1;
  else for (int q = rp[i]; q < rp[i + 1]; q++) if (S[q] && cf[ci[q]] == 1) c++;
  len[i] = c;
}

// pcap: capacity of pci / pv (a row that would pass it sets *err and is
// skipped; nnz(P) <= nnz(A) makes that impossible for direct interpolation)
__global__ void k_interp_fill(int n, const int *rp, const int *ci, const double *v, const uint8_t *S,
                              const int8_t *cf, const int *cidx, const int *prp, int *pci, double *pv, int pcap,
                              int *err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int o = prp[i];
  if (prp[i + 1] > pcap) { atomicExch(err, 1); return; }
  if (cf[i] == 1) { pci[o] = cidx[i]; pv[o] = 1.0; return; }
  if (prp[i + 1] == o) return;
  // sums in the row's column order: sneg / spos (one FP64 add per entry,
  // its target chosen by the sign) while the strong C entries are listed;
  // then snegc and the weights over that list only
  const int MAXC = 32;
  int m = prp[i + 1] - o, qs[MAXC], nq = 0;
  double sneg = 0.0, spos = 0.0, snegc = 0.0, aii = 0.0;
  for (int q = rp[i]; q < rp[i + 1]; q++) {
    double a = v[q];
    int j = ci[q];
    if (S[q] && cf[j] == 1 && nq < MAXC) qs[nq++] = q;
    if (j == i) { aii = a; continue; }
    bool neg = dkey(a) < 0;
    double acc = add_rn(neg ? sneg : spos, a);
    if (neg) sneg = acc; else spos = acc;
  }
  if (m <= MAXC) {
    for (int t = 0; t < m; t++) snegc = add_rn(snegc, v[qs[t]]);
  } else {
    for (int q = rp[i]; q < rp[i + 1]; q++) if (S[q] && cf[ci[q]] == 1) snegc = add_rn(snegc, v[q]);
  }
  double dg = add_rn(aii, spos), alpha = div_rn(sneg, snegc);
  if (m <= MAXC) {
    for (int t = 0; t < m; t++) {
      int q = qs[t];
      pci[o + t] = cidx[ci[q]]; pv[o + t] = div_rn(-mul_rn(alpha, v[q]), dg);
    }
  } else {
    for (int q = rp[i]; q < rp[i + 1]; q++)
      if (S[q] && cf[ci[q]] == 1) { pci[o] = cidx[ci[q]]; pv[o++] = div_rn(-mul_rn(alpha, v[q]), dg); }
  }
}

// --------------------------------------------- extended+i interpolation ---
// De Sterck, Falgout, Nolting and Yang (2008).  For an F point i the
// interpolatory set C^_i is its strong C neighbours plus the strong C
// neighbours of its strong F neighbours k; with a^_kl the couplings of row k
// of the sign opposite to a_kk and D_k = sum over l in C^_i + {i} of a^_kl,
//   at_ii = a_ii + sum_{weak n not in C^_i} a_in + sum_k a_ik a^_ki / D_k
//           (a_ik itself when D_k = 0),
//   w_ij  = -(a_ij + sum_{k: D_k != 0, j in row k} a_ik a^_kj / D_k) / at_ii,
// sums in row i's (and row k's) column order with round-to-nearest
// operations, so the result equals a plain IEEE evaluation in that order.
// One thread per row; rows of A have ascending columns.
__device__ __forceinline__ double exti_hat(double akk, double akl) {
  if (akk < 0.0) return akl > 0.0 ? akl : 0.0;
  return akl < 0.0 ? akl : 0.0;
}
__device__ __forceinline__ int row_find(const int *ci, int a, int b, int col) {
  while (a < b) {
    int m = (a + b) >> 1, c = ci[m];
    if (c == col) return m;
    if (c < col) a = m + 1; else b = m;
  }
  return -1;
}
__device__ __forceinline__ bool in_list(const int *s, int m, int x) {
  int lo = 0, hi = m;
  while (lo < hi) { int md = (lo + hi) >> 1, v = s[md]; if (v == x) return true; if (v < x) lo = md + 1; else hi = md; }
  return false;
}
// upper bound on |C^_i| (candidates before duplicates are removed)
__global__ void k_exti_bound(int n, const int *rp, const int *ci, const uint8_t *S, const int8_t *cf, int *ub) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = 0;
  if (cf[i] != 1)
    for (int q = rp[i]; q < rp[i + 1]; q++) {
      int j = ci[q];
      if (!S[q] || j == i) continue;
      if (cf[j] == 1) c++;
      else for (int r = rp[j]; r < rp[j + 1]; r++) if (S[r] && cf[ci[r]] == 1) c++;
    }
  ub[i] = c;
}
// C^_i of each F row, sorted and without duplicates, in its segment of
// cand (offsets uoff); len[i] = |C^_i| (1 for a C point)
__global__ void k_exti_cands(int n, const int *rp, const int *ci, const uint8_t *S, const int8_t *cf, const int *uoff,
                             int *cand, int *len) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (cf[i] == 1) { len[i] = 1; return; }
  int *c = cand + uoff[i], m = 0;
  for (int q = rp[i]; q < rp[i + 1]; q++) {
    int j = ci[q];
    if (!S[q] || j == i) continue;
    if (cf[j] == 1) c[m++] = j;
    else for (int r = rp[j]; r < rp[j + 1]; r++) if (S[r] && cf[ci[r]] == 1) c[m++] = ci[r];
  }
  for (int a = 1; a < m; a++) { int v = c[a], b = a - 1; while (b >= 0 && c[b] > v) { c[b + 1] = c[b]; b--; } c[b + 1] = v; }
  int u = 0;
  for (int a = 0; a < m; a++) if (u == 0 || c[a] != c[u - 1]) c[u++] = c[a];
  len[i] = u;
}
// D_k for each strong F neighbour k of an F row, stored at k's position q in row i
__global__ void k_exti_dk(int n, const int *rp, const int *ci, const double *v, const uint8_t *S, const int8_t *cf,
                          const int *uoff, const int *cand, const int *prp, double *D) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || cf[i] == 1) return;
  const int *cs = cand + uoff[i];
  int m = prp[i + 1] - prp[i];
  for (int q = rp[i]; q < rp[i + 1]; q++) {
    int k = ci[q];
    D[q] = 0.0;
    if (!S[q] || k == i || cf[k] != -1) continue;
    int dk = row_find(ci, rp[k], rp[k + 1], k);
    double akk = dk >= 0 ? v[dk] : 0.0, d = 0.0;
    for (int r = rp[k]; r < rp[k + 1]; r++) {
      int l = ci[r];
      if (l == i || in_list(cs, m, l)) d = add_rn(d, exti_hat(akk, v[r]));
    }
    D[q] = d;
  }
}
__global__ void k_exti_fill(int n, const int *rp, const int *ci, const double *v, const uint8_t *S, const int8_t *cf,
                            const int *cidx, const int *uoff, const int *cand, const double *D, const int *prp, int *pci,
                            double *pv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int o = prp[i], m = prp[i + 1] - o;
  if (cf[i] == 1) { pci[o] = cidx[i]; pv[o] = 1.0; return; }
  if (m == 0) return;
  const int *cs = cand + uoff[i];
  int di = row_find(ci, rp[i], rp[i + 1], i);
  double at = di >= 0 ? v[di] : 0.0;
  for (int q = rp[i]; q < rp[i + 1]; q++) {
    int j = ci[q];
    if (j == i) continue;
    if (S[q]) {
      if (cf[j] == 1) continue;
      if (D[q] == 0.0) at = add_rn(at, v[q]);
      else {
        int dk = row_find(ci, rp[j], rp[j + 1], j), ki = row_find(ci, rp[j], rp[j + 1], i);
        double akk = dk >= 0 ? v[dk] : 0.0, aki = ki >= 0 ? v[ki] : 0.0;
        at = add_rn(at, div_rn(mul_rn(v[q], exti_hat(akk, aki)), D[q]));
      }
    } else if (!in_list(cs, m, j)) at = add_rn(at, v[q]);
  }
  for (int a = 0; a < m; a++) {
    int j = cs[a];
    int qj = row_find(ci, rp[i], rp[i + 1], j);
    double num = qj >= 0 ? v[qj] : 0.0;
    for (int q = rp[i]; q < rp[i + 1]; q++) {
      int k = ci[q];
      if (!S[q] || k == i || cf[k] != -1 || D[q] == 0.0) continue;
      int kj = row_find(ci, rp[k], rp[k + 1], j);
      if (kj < 0) continue;
      int dk = row_find(ci, rp[k], rp[k + 1], k);
      double akk = dk >= 0 ? v[dk] : 0.0;
      num = add_rn(num, div_rn(mul_rn(v[q], exti_hat(akk, v[kj])), D[q]));
    }
    pci[o + a] = cidx[j];
    pv[o + a] = div_rn(-num, at);
  }
}

// ------------------------------------------------------------ transpose ---
__global__ void k_col_count(int nnz, const int *ci, int *cnt) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < nnz) atomicAdd(&cnt[ci[q]], 1);
}
__global__ void k_transpose_fill(int n, const int *rp, const int *ci, const double *v, const int *trp, int *fill,
                                 int *tci, double *tv) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int q = rp[i]; q < rp[i + 1]; q++) {
    int j = ci[q], o = trp[j] + atomicAdd(&fill[j], 1);
    tci[o] = i; tv[o] = v[q];
  }
}
// one warp per row: rows of at most 32 entries by a bitonic network across
// the lanes (columns within a row are distinct, so the order is unique),
// longer rows by an insertion sort in the first lane
__global__ void k_sort_rows_warp(int n, const int *rp, int *ci, double *v) {
  int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (i >= n) return;
  int a0 = rp[i], len = rp[i + 1] - a0;
  if (len <= 32) {
    int c = lane < len ? ci[a0 + lane] : INT_MAX;
    double x = lane < len ? v[a0 + lane] : 0.0;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1)
#pragma unroll
      for (int j = k >> 1; j > 0; j >>= 1) {
        int oc = __shfl_xor_sync(0xffffffffu, c, j);
        double ox = __shfl_xor_sync(0xffffffffu, x, j);
        bool up = (lane & k) == 0, lower = (lane & j) == 0;
        bool take = lower == up ? oc < c : oc > c;     // keep the smaller key on the ascending side
        if (take) { c = oc; x = ox; }
      }
    if (lane < len) { ci[a0 + lane] = c; v[a0 + lane] = x; }
  } else if (lane == 0) {
    int a1 = a0 + len;
    for (int a = a0 + 1; a < a1; a++) {
      int c = ci[a]; double x = v[a]; int b = a - 1;
      while (b >= a0 && ci[b] > c) { ci[b + 1] = ci[b]; v[b + 1] = v[b]; b--; }
      ci[b + 1] = c; v[b + 1] = x;
    }
  }
}

// the same with G lanes per row (G = 8 or 16) for levels whose rows are
// short: a bitonic network over the group's lanes (rows of at most G
// entries), longer rows by an insertion sort in the group's first lane
template <int G>
__global__ void k_sort_rows_g(int n, const int *rp, int *ci, double *v) {
  if (n <= 0) return;
  int gi = (blockIdx.x * blockDim.x + threadIdx.x) / G, k = threadIdx.x % G;
  bool valid = gi < n;
  int i = valid ? gi : n - 1;                       // whole groups stay in the shuffles
  int a0 = rp[i], len = rp[i + 1] - a0;
  bool small = len <= G;
  int c = (small && k < len) ? ci[a0 + k] : INT_MAX;
  double x = (small && k < len) ? v[a0 + k] : 0.0;
#pragma unroll
  for (int kk = 2; kk <= G; kk <<= 1)
#pragma unroll
    for (int j = kk >> 1; j > 0; j >>= 1) {
      int oc = __shfl_xor_sync(0xffffffffu, c, j, G);
      double ox = __shfl_xor_sync(0xffffffffu, x, j, G);
      bool up = (k & kk) == 0, lower = (k & j) == 0;
      bool take = lower == up ? oc < c : oc > c;     // keep the smaller key on the ascending side
      if (take) { c = oc; x = ox; }
    }
  if (!valid) return;
  if (small) {
    if (k < len) { ci[a0 + k] = c; v[a0 + k] = x; }
  } else if (k == 0) {
    int a1 = a0 + len;
    for (int a = a0 + 1; a < a1; a++) {
      int cc = ci[a]; double xx = v[a]; int b = a - 1;
      while (b >= a0 && ci[b] > cc) { ci[b + 1] = ci[b]; v[b + 1] = v[b]; b--; }
      ci[b + 1] = cc; v[b + 1] = xx;
    }
  }
}

// -------------------------------------------------------------- SpGEMM ----
// C = A B, each column of a row of C the sum of its products A_ik B_kj in
// the order of k (the row of A's column order), starting from 0.  Rows of A
// with at most SPG_KMAX entries and at most SPG_MERGE_P products, on products
// of many rows (spg_merge_p): k_spgemm_merge (one thread per row); the
// others: k_spgemm_hash (one warp per row).  One pass: each row is written at the offset of its product
// count (an upper bound of its length) into a scratch array, then the rows
// are packed.
// products per row of C; mx = 1 + the most products of a row that the
// hash kernel handles, 0 if there is none
#define SPG_KMAX 8
#define SPG_MERGE_P 96
__global__ void k_row_products(int n, const int *arp, const int *aci, const int *brp, int *prod, int *mx, int merge_p) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int s = 0;
  for (int q = arp[i]; q < arp[i + 1]; q++) { int k = aci[q]; s += brp[k + 1] - brp[k]; }
  prod[i] = s;
  if (arp[i + 1] - arp[i] > SPG_KMAX || s > merge_p) atomicMax(mx, s + 1);   // + 1: "a hash row exists" even with 0 products
}
// C row i = scratch[toff[i] .. toff[i] + clen[i]), eight lanes per row
__global__ void k_pack_rows(int n, const int *toff, const int *clen, const int *crp, const int *tci, const double *tv,
                            int *cci, double *cv) {
  int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 3, lane = threadIdx.x & 7;
  if (row >= n) return;
  int a = toff[row], b = crp[row], len = clen[row];
  for (int t = lane; t < len; t += 8) { cci[b + t] = tci[a + t]; cv[b + t] = tv[a + t]; }
}

// C = A B for the rows of A with at most K entries and at most merge_p
// products, one thread per row: a k-way merge of the k rows of B that the
// row of A selects (each sorted by column, its head kept in registers).  The
// smallest head column is the next column of C; its products are summed in
// the order of the row of A, starting from 0, as in the hash kernel below,
// so both kernels give the same bits.  Only short rows take this path (the
// finest level's stencil rows and most of its restriction): a thread walks
// its row of C serially, which loses to a warp per row once rows grow
// (measured on the coarser levels of the 1M-cell hierarchy).
template <int K>
__global__ void __launch_bounds__(128) k_spgemm_merge(int n, const int *arp, const int *aci, const double *av,
                                                      const int *brp, const int *bci, const double *bv,
                                                      const int *toff, int *clen, int *cci, double *cv, int merge_p) {
  int row = blockIdx.x * blockDim.x + threadIdx.x;
  if (row >= n) return;
  int a0 = arp[row], k = arp[row + 1] - a0;
  if (k > K || toff[row + 1] - toff[row] > merge_p) return;
  int pos[K], end[K], col[K];
  double a[K];
#pragma unroll
  for (int q = 0; q < K; q++) {
    col[q] = INT_MAX; pos[q] = 0; end[q] = 0; a[q] = 0.0;
    if (q < k) {
      int kk = aci[a0 + q];
      pos[q] = brp[kk]; end[q] = brp[kk + 1]; a[q] = av[a0 + q];
      if (pos[q] < end[q]) col[q] = bci[pos[q]];
    }
  }
  int out = toff[row], cnt = 0;
  for (;;) {
    int c = INT_MAX;
#pragma unroll
    for (int q = 0; q < K; q++) c = min(c, col[q]);
    if (c == INT_MAX) break;
    // the heads on column c, in q order.  Only they issue FP64 work: each is
    // picked out of the register arrays by a chain of selects (integer
    // pipes), so the FP64 pipe (a small fraction of the FP32 rate on this
    // GPU) sees one product and one sum per actual product instead of one
    // predicated pair per head
    unsigned hit = 0;
#pragma unroll
    for (int q = 0; q < K; q++) hit |= (col[q] == c ? 1u : 0u) << q;
    double s = 0.0;
    for (unsigned h = hit; h; h &= h - 1) {
      int qq = __ffs(h) - 1;
      double aq = a[0];
      int pq = pos[0];
#pragma unroll
      for (int q = 1; q < K; q++) { aq = qq == q ? a[q] : aq; pq = qq == q ? pos[q] : pq; }
      s = add_rn(s, mul_rn(aq, bv[pq]));
    }
#pragma unroll
    for (int q = 0; q < K; q++)
      if (hit >> q & 1u) {
        pos[q]++;
        col[q] = pos[q] < end[q] ? bci[pos[q]] : INT_MAX;
      }
    cci[out + cnt] = c; cv[out + cnt] = s;
    cnt++;
  }
  clen[row] = cnt;
}

// Rows that the merge kernel leaves (more than SPG_KMAX entries in A, or
// more than merge_p products), one warp per row of C.  The products are
// taken in sequence order (row of A ascending, then row of B ascending), 32
// at a time; each lane claims its column's slot in an open-addressing hash
// table (compare-and-swap on the key, linear probing; the table has at
// least as many slots as the row has products, so a probe always ends), and
// the lanes of one chunk that hit the same slot are summed by the lowest of
// them in lane order.  So each column's products are summed in sequence
// order starting from 0, as in the merge kernel.  The occupied slots are
// then compacted, sorted by column (bitonic; the columns are distinct) and
// written at the row's scratch offset.  The table sits in shared memory, or
// (gscratch, for the rare rows beyond what shared memory holds) in a global
// scratch area; tcap slots per warp.  Rows with at most lo_p products
// belong to the other launch.
__host__ __device__ constexpr size_t spg_warp_doubles(int tcap) {
  // vals[tcap], seg_a[32], prodbuf[32] (doubles), keys[tcap], seg_off[33], seg_k[32] (ints)
  return (size_t)tcap + 64 + ((size_t)tcap + 65 + 1) / 2;
}
__global__ void __launch_bounds__(256) k_spgemm_hash(int n, const int *arp, const int *aci, const double *av,
                                                     const int *brp, const int *bci, const double *bv,
                                                     const int *toff, int *clen, int *cci, double *cv, int tcap,
                                                     int lo_p, double *gscratch, int merge_p) {
  extern __shared__ double sm_hash[];
  const int warps = blockDim.x >> 5, wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned FULL = 0xffffffffu;
  const size_t wd = spg_warp_doubles(tcap);
  double *base = gscratch ? gscratch + ((size_t)blockIdx.x * warps + wid) * wd : sm_hash + (size_t)wid * wd;
  double *vals = base, *seg_a = base + tcap, *prodbuf = seg_a + 32;
  int *keys = reinterpret_cast<int *>(prodbuf + 32), *seg_off = keys + tcap, *seg_k = seg_off + 33;
  volatile int *vkeys = keys;
  for (int row = blockIdx.x * warps + wid; row < n; row += gridDim.x * warps) {
    int a0 = arp[row], a1 = arp[row + 1], out = toff[row], p = toff[row + 1] - out;
    if (a1 - a0 <= SPG_KMAX && p <= merge_p) continue;        // the merge kernel's row
    if (p > tcap || p <= lo_p) continue;                      // the other launch's row
    int T = 32;
    while (T < p) T <<= 1;
    for (int i = lane; i < T; i += 32) { keys[i] = -1; vals[i] = 0.0; }
    __syncwarp();
    for (int q0 = a0; q0 < a1; q0 += 32) {
      int q = q0 + lane, len = 0, k = 0;
      double a = 0.0;
      if (q < a1) { k = aci[q]; len = brp[k + 1] - brp[k]; a = av[q]; }
      int incl = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) { int y = __shfl_up_sync(FULL, incl, o); if (lane >= o) incl += y; }
      int tot = __shfl_sync(FULL, incl, 31);
      seg_off[lane] = incl - len; seg_k[lane] = k; seg_a[lane] = a;
      __syncwarp();
      int nseg = min(32, a1 - q0);
      for (int t0 = 0; t0 < tot; t0 += 32) {
        int t = t0 + lane, slot = -1 - lane;
        double prod = 0.0;
        if (t < tot) {
          int lo = 0, hi = nseg - 1;                          // last segment starting at or before t
          while (lo < hi) { int md = (lo + hi + 1) >> 1; if (seg_off[md] <= t) lo = md; else hi = md - 1; }
          int b = brp[seg_k[lo]] + (t - seg_off[lo]), c = bci[b];
          prod = mul_rn(seg_a[lo], bv[b]);
          int h = (int)(((unsigned)c * 0x9E3779B1u) & (unsigned)(T - 1));
          for (int it = 0; it < T; it++) {
            int key = vkeys[h];
            if (key == c) break;
            if (key == -1) {
              int old = atomicCAS(&keys[h], -1, c);
              if (old == -1 || old == c) break;
            }
            h = (h + 1) & (T - 1);
          }
          slot = h;
        }
        unsigned grp = __match_any_sync(FULL, slot);
        prodbuf[lane] = prod;
        __syncwarp();
        if (t < tot && lane == __ffs(grp) - 1) {
          double s = vals[slot];
          for (unsigned m = grp; m; m &= m - 1) s = add_rn(s, prodbuf[__ffs(m) - 1]);
          vals[slot] = s;
        }
        __syncwarp();
      }
    }
    // compact the occupied slots to the front of the table
    int u = 0;
    for (int i0 = 0; i0 < T; i0 += 32) {
      int key = keys[i0 + lane];
      double v = vals[i0 + lane];
      unsigned mask = __ballot_sync(FULL, key >= 0);
      int pre = __popc(mask & ((1u << lane) - 1u));
      __syncwarp();
      if (key >= 0) { keys[u + pre] = key; vals[u + pre] = v; }
      u += __popc(mask);
      __syncwarp();
    }
    if (u <= 64) {
      // up to 64 entries: two per lane in registers (indices lane and lane +
      // 32, padded with INT_MAX), sorted by the same bitonic network over
      // shuffles instead of shared-memory passes
      int k0 = lane < u ? keys[lane] : INT_MAX, k1 = lane + 32 < u ? keys[lane + 32] : INT_MAX;
      double v0 = lane < u ? vals[lane] : 0.0, v1 = lane + 32 < u ? vals[lane + 32] : 0.0;
      const int M = u <= 32 ? 32 : 64;
      for (int kk = 2; kk <= M; kk <<= 1)
        for (int j = kk >> 1; j > 0; j >>= 1) {
          if (j == 32) {                                // partners in the lane's two registers (kk = 64: ascending)
            if (k0 > k1) { int x = k0; k0 = k1; k1 = x; double w = v0; v0 = v1; v1 = w; }
            continue;
          }
#pragma unroll
          for (int r = 0; r < 2; r++) {
            if (r == 1 && M == 32) break;
            int x = r ? k1 : k0;
            double vx = r ? v1 : v0;
            int y = __shfl_xor_sync(FULL, x, j);
            double vy = __shfl_xor_sync(FULL, vx, j);
            int i = lane + 32 * r;
            bool keep_min = ((i & j) == 0) == ((i & kk) == 0);   // the lower index keeps the minimum when ascending
            bool take = keep_min ? y < x : y > x;
            if (take) { x = y; vx = vy; }
            if (r) { k1 = x; v1 = vx; } else { k0 = x; v0 = vx; }
          }
        }
      if (lane < u) { cci[out + lane] = k0; cv[out + lane] = v0; }
      if (lane + 32 < u) { cci[out + lane + 32] = k1; cv[out + lane + 32] = v1; }
    } else {
      int M = 1;
      while (M < u) M <<= 1;
      for (int i = u + lane; i < M; i += 32) keys[i] = INT_MAX;
      __syncwarp();
      for (int kk = 2; kk <= M; kk <<= 1)
        for (int j = kk >> 1; j > 0; j >>= 1) {
          for (int i = lane; i < M; i += 32) {
            int ixj = i ^ j;
            if (ixj > i) {
              int x = keys[i], y = keys[ixj];
              bool up = (i & kk) == 0;
              if ((x > y) == up) {
                keys[i] = y; keys[ixj] = x;
                double w = vals[i]; vals[i] = vals[ixj]; vals[ixj] = w;
              }
            }
          }
          __syncwarp();
        }
      for (int i = lane; i < u; i += 32) { cci[out + i] = keys[i]; cv[out + i] = vals[i]; }
    }
    if (lane == 0) clen[row] = u;
    __syncwarp();
  }
}

// SpGEMM C = A B in two phases with one host wait between them.
// spgemm_count: products per row of C (scratch offsets, toff) and their
// total in *tot, the long-row marker (1 + the most products of a row that
// the hash kernel handles, 0 if none) in *mx (which must be 0 before);
// no host wait.  spgemm_fill: given those two values on the host, the
// numeric product into scratch, the row pointers of C (C.rp[n] and *nnz =
// nnz(C) on the device) and the packed rows; C's arrays are sized by the
// product total, an upper bound of nnz(C), so no further wait is needed.
struct spg_scratch { dbuf<int> toff, clen, tci; dbuf<double> tv, gs; };
static spg_scratch &spg() { static thread_local spg_scratch z; return z; }
// Rows for the thread-per-row merge kernel (at most SPG_KMAX entries in A
// and at most this many products): only when the product has enough rows to
// fill the GPU with threads; on smaller products a thread's serial merge is
// the launch's critical path (60-90 µs on the 1M-cell hierarchy's coarse
// levels) and every row goes to the hash kernel.  Both kernels give the
// same bits, so the split changes no result.
static int spg_merge_p(int n) { return n >= 65536 ? SPG_MERGE_P : -1; }

static void spgemm_count(const csr_dev<double> &A, const csr_dev<double> &B, int *tot, int *mx, cudaStream_t s) {
  spg_scratch &z = spg();
  int n = A.n;
  z.toff.ensure(n + 1); z.clen.ensure(n + 1);
  k_row_products<<<grid_for(n, 256), 256, 0, s>>>(n, A.rp.p, A.ci.p, B.rp.p, z.toff.p, mx, spg_merge_p(n));
  RS_LAUNCHED(1);
  rs_scan_dev(z.toff.p, z.toff.p, n, z.toff.p + n, tot, s);      // row offsets into the scratch arrays
}

static void spgemm_fill(const csr_dev<double> &A, const csr_dev<double> &B, csr_dev<double> &C, int total, int mx1,
                        int *nnz, cudaStream_t s) {
  spg_scratch &z = spg();
  int n = A.n, mx = std::max(mx1 - 1, 0);
  // hash-table slots per warp: at least the products of the largest row in
  // the launch; rows beyond 1024 products (above the 99.9th percentile on
  // the channelised cases) go to a second launch with a global scratch area
  int tall = 64;
  while (tall < mx) tall <<= 1;
  int tcap = std::min(tall, 1024);
  size_t wbytes = spg_warp_doubles(tcap) * sizeof(double);
  int warps = (int)std::min<size_t>(8, std::max<size_t>(1, (100 * 1024) / wbytes));
  size_t smem = wbytes * warps;
  static bool attr = false;
  if (!attr) {
    RS_CUDA(cudaFuncSetAttribute(k_spgemm_hash, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr = true;
  }
  z.tci.ensure(std::max(total, 1)); z.tv.ensure(std::max(total, 1));
  C.n = n; C.m = B.m; C.nnz = -1;                      // known on the host at the next wait
  C.rp.ensure(n + 1);
  int mp = spg_merge_p(n);
  if (mp >= 0) {
    k_spgemm_merge<SPG_KMAX><<<grid_for(n, 128), 128, 0, s>>>(n, A.rp.p, A.ci.p, A.v.p, B.rp.p, B.ci.p, B.v.p,
                                                              z.toff.p, z.clen.p, z.tci.p, z.tv.p, mp);
    RS_LAUNCHED(1);
  }
  if (mx1 > 0) {                                       // rows for the hash kernel
    unsigned grid = (unsigned)std::min<size_t>((n + warps - 1) / warps, 152 * 32);
    k_spgemm_hash<<<grid, warps * 32, smem, s>>>(n, A.rp.p, A.ci.p, A.v.p, B.rp.p, B.ci.p, B.v.p, z.toff.p,
                                                 z.clen.p, z.tci.p, z.tv.p, tcap, -1, nullptr, mp);
    RS_LAUNCHED(1);
    if (tall > tcap) {                                 // rows beyond the shared-memory capacity
      const int gw = 4, gblocks = 64;
      z.gs.ensure((size_t)gblocks * gw * spg_warp_doubles(tall));
      k_spgemm_hash<<<gblocks, gw * 32, 0, s>>>(n, A.rp.p, A.ci.p, A.v.p, B.rp.p, B.ci.p, B.v.p, z.toff.p, z.clen.p,
                                                z.tci.p, z.tv.p, tall, tcap, z.gs.p, mp);
      RS_LAUNCHED(1);
    }
  }
  RS_CHECK_LAUNCH();
  rs_scan_dev(z.clen.p, C.rp.p, n, C.rp.p + n, nnz, s);
  C.ci.ensure(std::max(total, 1)); C.v.ensure(std::max(total, 1));
  k_pack_rows<<<grid_for((size_t)n * 8, 256), 256, 0, s>>>(n, z.toff.p, z.clen.p, C.rp.p, z.tci.p, z.tv.p, C.ci.p,
                                                          C.v.p);
  RS_LAUNCHED(1);
  RS_CHECK_LAUNCH();
}

// ------------------------------------------------------------ smoother ----
__global__ void k_l1(int n, const int *rp, const int *ci, const double *v, double *dinv, float *dinv32) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0, aii = 0.0;
  for (int q = rp[i]; q < rp[i + 1]; q++) { if (ci[q] == i) aii = v[q]; else s = add_rn(s, fabs(v[q])); }
  double d = add_rn(aii, s);
  dinv[i] = 1.0 / d;
  if (dinv32) dinv32[i] = (float)(1.0 / d);
}

// --------------------------------------------------------- dense coarsest -
__global__ void k_dense_build(int n, const int *rp, const int *ci, const double *v, double *a) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int j = 0; j < n; j++) a[(size_t)i * n + j] = 0.0;
  for (int q = rp[i]; q < rp[i + 1]; q++) a[(size_t)i * n + ci[q]] = v[q];
}
// LU with partial pivoting (first row of maximal |a_ik|), then the inverse
// column by column; one block.
__global__ void k_dense_lu_inv(int n, double *a, int *piv, double *inv) {
  __shared__ double smx[1024]; __shared__ int sid[1024];
  int t = threadIdx.x, nt = blockDim.x;
  for (int k = 0; k < n; k++) {
    double best = -1.0; int bi = n;
    for (int i = k + t; i < n; i += nt) { double x = fabs(a[(size_t)i * n + k]); if (x > best) { best = x; bi = i; } }
    smx[t] = best; sid[t] = bi;
    __syncthreads();
    for (int o = nt >> 1; o > 0; o >>= 1) {
      if (t < o) {
        double x = smx[t + o]; int xi = sid[t + o];
        if (x > smx[t] || (x == smx[t] && xi < sid[t])) { smx[t] = x; sid[t] = xi; }
      }
      __syncthreads();
    }
    int p = sid[0];
    if (t == 0) piv[k] = p;
    if (p != k)
      for (int j = t; j < n; j += nt) { double x = a[(size_t)k * n + j]; a[(size_t)k * n + j] = a[(size_t)p * n + j]; a[(size_t)p * n + j] = x; }
    __syncthreads();
    for (int i = k + 1 + t; i < n; i += nt) a[(size_t)i * n + k] = div_rn(a[(size_t)i * n + k], a[(size_t)k * n + k]);
    __syncthreads();
    for (int e = t; e < (n - k - 1) * (n - k - 1); e += nt) {
      int i = k + 1 + e / (n - k - 1), j = k + 1 + e % (n - k - 1);
      a[(size_t)i * n + j] = sub_rn(a[(size_t)i * n + j], mul_rn(a[(size_t)i * n + k], a[(size_t)k * n + j]));
    }
    __syncthreads();
  }
  // inverse: column c of A^{-1} solves A x = e_c
  for (int c = t; c < n; c += nt) {
    double *x = inv + (size_t)c * n;            // stored transposed: inv[c][i] = (A^{-1})_{ic}
    for (int i = 0; i < n; i++) x[i] = (i == c) ? 1.0 : 0.0;
    for (int k = 0; k < n; k++) if (piv[k] != k) { double y = x[k]; x[k] = x[piv[k]]; x[piv[k]] = y; }
    for (int i = 0; i < n; i++) { double s = x[i]; for (int j = 0; j < i; j++) s -= a[(size_t)i * n + j] * x[j]; x[i] = s; }
    for (int i = n - 1; i >= 0; i--) { double s = x[i]; for (int j = i + 1; j < n; j++) s -= a[(size_t)i * n + j] * x[j]; x[i] = s / a[(size_t)i * n + i]; }
  }
}

// The inverse of the coarsest operator (n <= 128) in two kernels.  FP64
// is the slow pipe here (a warp's FP64 instruction holds its SM
// sub-partition for tens of cycles), so both keep FP64 work off the serial
// chain: one reciprocal per pivot, stored for the second kernel.
// k_dense_lu_smem: LU with partial pivoting in shared memory (at most 128
// KB), one block.  Step k: warp 0 finds the pivot row (largest |a_ik|, i >=
// k, the lowest index on ties; |a_ik| compared on its bit pattern, which
// orders non-negative doubles), swaps the whole rows, forms r_k = 1/a_kk and
// the multipliers l_ik = a_ik r_k (i > k); then every warp takes rows i > k
// and every lane columns j > k: a_ij -= l_ik a_kj.  Two block barriers per
// step; n^3/3 multiply-adds in all.
__global__ void __launch_bounds__(512) k_dense_lu_smem(int n, const double *ag, int *piv, double *lu, double *rdiag) {
  extern __shared__ double sa[];
  const int t = threadIdx.x, lane = t & 31, w = t >> 5, nw = blockDim.x >> 5;
  for (int e = t; e < n * n; e += blockDim.x) sa[e] = ag[e];
  __syncthreads();
  for (int k = 0; k < n; k++) {
    if (w == 0) {
      long long best = -1; int bi = n;
      for (int i = k + lane; i < n; i += 32) {
        long long x = __double_as_longlong(sa[i * n + k]) & 0x7fffffffffffffffLL;
        if (x > best) { best = x; bi = i; }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        long long x = __shfl_xor_sync(0xffffffffu, best, o); int xi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (x > best || (x == best && xi < bi)) { best = x; bi = xi; }
      }
      const int p = bi < n ? bi : k;
      if (p != k)
        for (int j = lane; j < n; j += 32) { double x = sa[k * n + j]; sa[k * n + j] = sa[p * n + j]; sa[p * n + j] = x; }
      __syncwarp();
      const double r = 1.0 / sa[k * n + k];
      for (int i = k + 1 + lane; i < n; i += 32) sa[i * n + k] *= r;
      if (lane == 0) { piv[k] = p; rdiag[k] = r; }
    }
    __syncthreads();
    for (int i = k + 1 + w; i < n; i += nw) {
      const double l = sa[i * n + k];
      for (int j = k + 1 + lane; j < n; j += 32) sa[i * n + j] = fma(-l, sa[k * n + j], sa[i * n + j]);
    }
    __syncthreads();
  }
  for (int e = t; e < n * n; e += blockDim.x) lu[e] = sa[e];
}

// k_dense_inv_cols: column c of A^{-1} = U^{-1} L^{-1} P e_c, one warp per
// column (two per block), the factors staged in shared memory.  Lane r
// keeps rows r, r + 32, ... (NR of them) in registers; the forward sweep
// starts at the row where the swaps put the unit entry (L has a unit
// diagonal), and both sweeps go column by column (x_j broadcast from its
// lane, then every row below or above subtracts its term; registers that
// hold no such row are not touched).  Stored transposed:
// inv[c][i] = (A^{-1})_{ic}.  Equal to the row-by-row LU solve up to
// rounding.
template <int NR>
__global__ void __launch_bounds__(64) k_dense_inv_cols(int n, const double *lu, const int *piv, const double *rdiag,
                                                      double *inv) {
  extern __shared__ double sl[];
  double *sr = sl + (size_t)n * n;
  int *sp = reinterpret_cast<int *>(sr + n);
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) sl[e] = lu[e];
  for (int k = threadIdx.x; k < n; k += blockDim.x) { sp[k] = piv[k]; sr[k] = rdiag[k]; }
  __syncthreads();
  const int lane = threadIdx.x & 31, c = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (c >= n) return;
  int pos = c;                                      // the unit entry of P e_c after the swaps in order
  for (int k = 0; k < n; k++) { int p = sp[k]; pos = pos == k ? p : (pos == p ? k : pos); }
  double b[NR];
#pragma unroll
  for (int u = 0; u < NR; u++) b[u] = (lane + 32 * u) == pos ? 1.0 : 0.0;
  // column j = 32 jb + jj: its b sits in register jb of lane jj (jb a
  // compile-time index, so b stays in registers)
#pragma unroll
  for (int jb = 0; jb < NR; jb++) {                  // L y = P e_c (rows before pos stay 0)
    for (int jj = pos > 32 * jb ? pos - 32 * jb : 0; jj < 32 && 32 * jb + jj < n - 1; jj++) {
      const int j = 32 * jb + jj;
      const double yj = __shfl_sync(0xffffffffu, b[jb], jj);
#pragma unroll
      for (int u = jb; u < NR; u++) {               // rows below j live in registers jb and up
        const int i = lane + 32 * u;
        if (i > j && i < n) b[u] = fma(-sl[i * n + j], yj, b[u]);
      }
    }
  }
#pragma unroll
  for (int jb = NR - 1; jb >= 0; jb--) {             // U x = y
    for (int jj = 31; jj >= 0; jj--) {
      const int j = 32 * jb + jj;
      if (j >= n) continue;
      const double xj = __shfl_sync(0xffffffffu, b[jb], jj) * sr[j];
#pragma unroll
      for (int u = 0; u <= jb; u++) {               // rows at or above j live in registers up to jb
        const int i = lane + 32 * u;
        if (i == j) b[u] = xj;
        else if (i < j) b[u] = fma(-sl[i * n + j], xj, b[u]);
      }
    }
  }
#pragma unroll
  for (int u = 0; u < NR; u++) {
    const int i = lane + 32 * u;
    if (i < n) inv[(size_t)c * n + i] = b[u];
  }
}

// ----------------------------------------------------------- host setup ---
// FP32 values of an FP64 operator (the pattern stays the FP64 operator's)
static void csr_cast(const csr_dev<double> &a, csr_dev<float> &b, cudaStream_t s) {
  b.n = a.n; b.m = a.m; b.nnz = a.nnz;
  b.v.ensure(a.nnz);
  rs_cast_d2f(a.v.p, b.v.p, a.nnz, s);
}

// Words of h.flag, the setup's device counters, read back into the pinned
// h.hflag at the few points where the host needs a size: per level once
// after the split, P and the products of A P are known (wait 1), and once
// after the products of R (A P) are known (wait 2); nnz of the coarse
// operators at the next wait 1 or at the end.
enum {
  AF_SYM = 0,        // pattern of A not structurally symmetric
  AF_PCAP = 1,       // a row of P beyond its capacity
  AF_NC = 2,         // C points (coarse size)
  AF_PNNZ = 3,       // nnz(P)
  AF_APTOT = 4, AF_APMX = 5, AF_APNNZ = 6,     // products, long-row marker and nnz of A P
  AF_RAPTOT = 7, AF_RAPMX = 8,                 // the same for R (A P)
  AF_PRND = 9,       // PMIS rounds taken (-1: not finished within the cap)
  AF_SLOTS = 16,
  AF_LNNZ = 16,      // [16 + l]: nnz of level l's operator (l >= 1)
  AF_CNT = 48,       // [48 + r]: undecided points after PMIS round r - 1 (r = 0: after the initialisation)
  AF_ROUNDS_MAX = 1020,
  AF_WORDS = AF_CNT + AF_ROUNDS_MAX + 8
};
// PMIS: a list of at most this many points x lanes goes to the one-block
// tail (two passes of its 1024 threads per step); the counts of the first
// PMIS_HINT_ROUNDS rounds are read back to choose the next setup's switch
static const int PMIS_TAIL_PTS = 2048, PMIS_HINT_ROUNDS = 24;

static const int *amg_read(amg_hier &h, int lo, int count, cudaStream_t s) {
  RS_CUDA(cudaMemcpyAsync(h.hflag + lo, h.flag.p + lo, (size_t)count * sizeof(int), cudaMemcpyDeviceToHost, s));
  RS_CUDA(cudaStreamSynchronize(s));
  return h.hflag;
}

// PMIS rounds [r0, r1) over the undecided-point lists (round r reads list r
// % 2 with cnt[r] entries and fills list (r + 1) % 2, counting into cnt[r +
// 1]); a round after the last undecided point was decided does nothing.
// Grids stride over the lists: the first two rounds sized for every point,
// later ones for an eighth (their lists are short; a longer one is strided).
static void pmis_rounds(amg_level &L, amg_hier &h, int n, int lanes, int r0, int r1, cudaStream_t s) {
  int *cnt = h.flag.p + AF_CNT;
  for (int r = r0; r < r1; r++) {
    size_t pts = r < 2 ? (size_t)n : ((size_t)n + 7) / 8;
    unsigned g = (unsigned)std::min<size_t>(grid_for(pts * lanes, 128), 152 * 16);
    const int *lst = h.plist.p + (size_t)(r & 1) * n;
    int *nxt = h.plist.p + (size_t)((r + 1) & 1) * n;
#define PMIS_ROUND(LL)                                                                                        \
    if (lanes == LL) {                                                                                        \
      k_pmis_select_w<LL><<<g, 128, 0, s>>>(L.A.rp.p, L.A.ci.p, L.strong.p, L.tpos.p, h.hashw.p, L.cf.p,      \
                                            h.newc.p, lst, cnt + r);                                          \
      k_pmis_update_w<LL><<<g, 128, 0, s>>>(L.A.rp.p, L.A.ci.p, L.strong.p, L.cf.p, h.newc.p, lst, cnt + r,   \
                                            nxt, cnt + r + 1);                                                \
    }
    PMIS_ROUND(1) PMIS_ROUND(4) PMIS_ROUND(16)
#undef PMIS_ROUND
  }
  RS_LAUNCHED(2 * (r1 - r0));
  RS_CHECK_LAUNCH();
}

// the rounds from r0 on in one block of 1024 threads (k_pmis_tail); the
// number of rounds taken goes to the flag word AF_PRND
static void pmis_tail(amg_level &L, amg_hier &h, int n, int lanes, int r0, cudaStream_t s) {
  int *F = h.flag.p;
#define PMIS_TAIL(LL)                                                                                          \
  if (lanes == LL)                                                                                             \
    k_pmis_tail<LL><<<1, 1024, 0, s>>>(L.A.rp.p, L.A.ci.p, L.strong.p, L.tpos.p, h.hashw.p, L.cf.p, h.newc.p,  \
                                       h.plist.p, n, F + AF_CNT, r0, AF_ROUNDS_MAX, F + AF_PRND);
  PMIS_TAIL(1) PMIS_TAIL(4) PMIS_TAIL(16)
#undef PMIS_TAIL
  RS_LAUNCHED(1);
  RS_CHECK_LAUNCH();
}

// P (and the C-point numbering in cidx) of level L from its C/F split, and
// the products of A P; no host wait for direct interpolation (nnz(P) <=
// nnz(A) sizes P), two for extended+i.  Returns nnz(P) when it is known on
// the host, else -1.
static int build_p(amg_level &L, amg_hier &h, const rs_opts &o, int n, size_t acap, dbuf<int> &cidx,
                   cudaStream_t s) {
  int *F = h.flag.p;
  k_cflag<<<grid_for(n, 256), 256, 0, s>>>(n, L.cf.p, cidx.p);
  RS_LAUNCHED(1);
  rs_scan_dev(cidx.p, cidx.p, n, cidx.p + n, F + AF_NC, s);
  L.P.n = n;
  L.P.rp.ensure(n + 1);
  int pnnz = -1;
  if (o.interp == SIM_INTERP_EXTI) {
    static thread_local dbuf<int> uoff, cand;
    static thread_local dbuf<double> dk;
    uoff.ensure(n + 1);
    k_exti_bound<<<grid_for(n, 128), 128, 0, s>>>(n, L.A.rp.p, L.A.ci.p, L.strong.p, L.cf.p, uoff.p);
    RS_LAUNCHED(1);
    int ncand = rs_scan(uoff.p, uoff.p, n, s);
    cand.ensure(ncand > 0 ? ncand : 1);
    k_exti_cands<<<grid_for(n, 128), 128, 0, s>>>(n, L.A.rp.p, L.A.ci.p, L.strong.p, L.cf.p, uoff.p, cand.p,
                                                  L.P.rp.p);
    RS_LAUNCHED(1);
    pnnz = rs_scan(L.P.rp.p, L.P.rp.p, n, s);
    RS_CUDA(cudaMemcpyAsync(L.P.rp.p + n, &pnnz, sizeof(int), cudaMemcpyHostToDevice, s));
    RS_CUDA(cudaStreamSynchronize(s));                 // pnnz is a local
    L.P.ci.ensure(pnnz > 0 ? pnnz : 1); L.P.v.ensure(pnnz > 0 ? pnnz : 1);
    dk.ensure(acap > 0 ? acap : 1);
    k_exti_dk<<<grid_for(n, 128), 128, 0, s>>>(n, L.A.rp.p, L.A.ci.p, L.A.v.p, L.strong.p, L.cf.p, uoff.p, cand.p,
                                               L.P.rp.p, dk.p);
    k_exti_fill<<<grid_for(n, 128), 128, 0, s>>>(n, L.A.rp.p, L.A.ci.p, L.A.v.p, L.strong.p, L.cf.p, cidx.p,
                                                 uoff.p, cand.p, dk.p, L.P.rp.p, L.P.ci.p, L.P.v.p);
    RS_LAUNCHED(2);
  } else {
    k_interp_count<<<grid_for(n, 256), 256, 0, s>>>(n, L.A.rp.p, L.A.ci.p, L.strong.p, L.cf.p, L.P.rp.p);
    RS_LAUNCHED(1);
    rs_scan_dev(L.P.rp.p, L.P.rp.p, n, L.P.rp.p + n, F + AF_PNNZ, s);
    L.P.ci.ensure(acap > 0 ? acap : 1); L.P.v.ensure(acap > 0 ? acap : 1);
    k_interp_fill<<<grid_for(n, 128), 128, 0, s>>>(n, L.A.rp.p, L.A.ci.p, L.A.v.p, L.strong.p, L.cf.p, cidx.p,
                                                   L.P.rp.p, L.P.ci.p, L.P.v.p, (int)L.P.ci.n, F + AF_PCAP);
    RS_LAUNCHED(1);
  }
  RS_CHECK_LAUNCH();
  spgemm_count(L.A, L.P, F + AF_APTOT, F + AF_APMX, s);
  return pnnz;
}

void amg_setup(amg_hier &h, const rs_opts &o, cudaStream_t s) {
  h.drop_graphs();                                  // buffers below may move
  h.flag.ensure(AF_WORDS);
  if (!h.hflag) RS_CUDA(cudaMallocHost((void **)&h.hflag, AF_WORDS * sizeof(int)));
  int *F = h.flag.p;
  bool mixed = o.precision != SIM_PREC_FP64;
  int l = 0;
  for (;;) {
    amg_level &L = h.lev[l];
    int n = L.A.n;
    // nnz(A) of a coarse level is known on the host only at this level's
    // first wait: until then its capacity bounds it, and the previous
    // setup's count picks the launch shapes (which do not change results)
    size_t acap = l == 0 ? (size_t)L.A.nnz : L.A.ci.n;
    long long nnz_hint = L.A.nnz >= 0 ? L.A.nnz : (L.nnz_prev > 0 ? L.nnz_prev : (long long)acap);
    L.dinv.ensure(n);
    if (mixed) L.dinv32.ensure(n);
    L.f.ensure(n); L.x.ensure(n); L.r.ensure(n); L.t.ensure(n);
    if (mixed) { L.f32.ensure(n); L.x32.ensure(n); L.r32.ensure(n); L.t32.ensure(n); }
    L.cf.ensure(n); L.strong.ensure(acap); L.tpos.ensure(acap);
    L.nc = 0; L.rounds = 0;
    if (n <= o.coarse_max || l == o.max_levels - 1) {      // coarsest: no split (all marks 0)
      k_l1<<<grid_for(n, 256), 256, 0, s>>>(n, L.A.rp.p, L.A.ci.p, L.A.v.p, L.dinv.p, mixed ? L.dinv32.p : nullptr);
      RS_LAUNCHED(1);
      RS_CUDA(cudaMemsetAsync(L.cf.p, 0, (size_t)n, s));
      h.coarse_dense = 1;
      break;
    }
    rs_fill_i(F, 0, AF_SLOTS, s);
    rs_fill_i(F + AF_CNT, 0, AF_WORDS - AF_CNT, s);
    if (nnz_hint > 8LL * n) k_tpos_warp<<<grid_for((size_t)n * 32, 128), 128, 0, s>>>(n, L.A.rp.p, L.A.ci.p, L.tpos.p, F + AF_SYM);
    else k_tpos<<<grid_for(n, 128), 128, 0, s>>>(n, L.A.rp.p, L.A.ci.p, L.tpos.p, F + AF_SYM);
    k_strength<<<grid_for(n, 128), 128, 0, s>>>(n, L.A.rp.p, L.A.ci.p, L.A.v.p, o.theta, L.strong.p, L.dinv.p,
                                              mixed ? L.dinv32.p : nullptr);
    h.hashw.ensure(n); h.newc.ensure(n); h.plist.ensure(2 * (size_t)n);
    k_pmis_init<<<grid_for(n, 128), 128, 0, s>>>(n, L.A.rp.p, L.A.ci.p, L.strong.p, L.tpos.p, o.seed, l,
                                                 h.hashw.p, L.cf.p, h.newc.p, F + AF_CNT, h.plist.p);
    RS_LAUNCHED(3);
    RS_CHECK_LAUNCH();
    // full-grid rounds while the lists are long (the previous setup's
    // counts say how many), then the rest in one block until a list is empty
    const int lanes = pmis_lanes(nnz_hint, n);
    const int k = L.tail_r >= 0 ? L.tail_r : ((long long)n * lanes <= PMIS_TAIL_PTS ? 0 : 3);
    pmis_rounds(L, h, n, lanes, 0, k, s);
    pmis_tail(L, h, n, lanes, k, s);
    static thread_local dbuf<int> cidx;      // C flags, then coarse index of each C point
    cidx.ensure(n + 1);
    int pnnz = build_p(L, h, o, n, acap, cidx, s);
    const int *hf = amg_read(h, 0, AF_CNT + PMIS_HINT_ROUNDS, s);   // wait 1
    if (hf[AF_SYM]) RS_FAIL(SIM_ERR_ARG, "AMG: level %d pattern is not structurally symmetric", l);
    if (hf[AF_PCAP]) RS_FAIL(SIM_ERR_ARG, "AMG: level %d interpolation beyond its capacity", l);
    if (hf[AF_PRND] < 0) RS_FAIL(SIM_ERR_TIMEOUT, "AMG: PMIS did not finish in %d rounds", (int)AF_ROUNDS_MAX);
    L.P.nnz = pnnz >= 0 ? pnnz : hf[AF_PNNZ];
    L.rounds = hf[AF_PRND];
    L.tail_r = std::min(L.rounds, PMIS_HINT_ROUNDS - 1);
    for (int r = 0; r < L.tail_r; r++)
      if ((long long)hf[AF_CNT + r] * lanes <= PMIS_TAIL_PTS) { L.tail_r = r; break; }
    if (l > 0) L.A.nnz = hf[AF_LNNZ + l];
    int nc = hf[AF_NC], ap_tot = hf[AF_APTOT], ap_mx = hf[AF_APMX];
    L.nc = nc;
    if (nc == 0) { h.coarse_dense = 0; break; }
    L.P.m = nc;
    static thread_local csr_dev<double> AP;
    spgemm_fill(L.A, L.P, AP, ap_tot, ap_mx, F + AF_APNNZ, s);
    // R = P^T
    L.R.n = nc; L.R.m = n; L.R.nnz = L.P.nnz;
    L.R.rp.ensure(nc + 1); L.R.ci.ensure(L.P.nnz > 0 ? L.P.nnz : 1); L.R.v.ensure(L.P.nnz > 0 ? L.P.nnz : 1);
    static thread_local dbuf<int> fill;
    fill.ensure(nc + 1);
    rs_fill_i(L.R.rp.p, 0, nc + 1, s);
    rs_fill_i(fill.p, 0, nc + 1, s);
    k_col_count<<<grid_for(L.P.nnz, 256), 256, 0, s>>>(L.P.nnz, L.P.ci.p, L.R.rp.p);
    RS_LAUNCHED(1);
    rs_scan_dev(L.R.rp.p, L.R.rp.p, nc, L.R.rp.p + nc, nullptr, s);
    k_transpose_fill<<<grid_for(n, 256), 256, 0, s>>>(n, L.P.rp.p, L.P.ci.p, L.P.v.p, L.R.rp.p, fill.p, L.R.ci.p,
                                                      L.R.v.p);
    {                                                  // rows of R: lanes per row by their mean length
      double avg = nc ? (double)L.P.nnz / nc : 0.0;
      // (a row longer than its group falls to one lane's insertion sort:
      // groups of 16 only where rows average at most 8 entries)
      if (avg <= 4.0) k_sort_rows_g<8><<<grid_for((size_t)nc * 8, 128), 128, 0, s>>>(nc, L.R.rp.p, L.R.ci.p, L.R.v.p);
      else if (avg <= 8.0)
        k_sort_rows_g<16><<<grid_for((size_t)nc * 16, 128), 128, 0, s>>>(nc, L.R.rp.p, L.R.ci.p, L.R.v.p);
      else k_sort_rows_warp<<<grid_for((size_t)nc * 32, 128), 128, 0, s>>>(nc, L.R.rp.p, L.R.ci.p, L.R.v.p);
    }
    RS_LAUNCHED(2);
    // A_{l+1} = R (A P)
    spgemm_count(L.R, AP, F + AF_RAPTOT, F + AF_RAPMX, s);
    hf = amg_read(h, 0, AF_SLOTS, s);                   // wait 2
    AP.nnz = hf[AF_APNNZ];
    spgemm_fill(L.R, AP, h.lev[l + 1].A, hf[AF_RAPTOT], hf[AF_RAPMX], F + AF_LNNZ + l + 1, s);
    if (mixed) { csr_cast(L.P, L.P32, s); csr_cast(L.R, L.R32, s); }
    l++;
  }
  h.nlev = l + 1;
  // nnz of the coarse operators not yet read (the coarsest one's at least)
  bool unknown = false;
  for (int k = 1; k < h.nlev; k++) unknown |= h.lev[k].A.nnz < 0;
  if (unknown) {
    const int *hf = amg_read(h, AF_LNNZ, h.nlev, s);
    for (int k = 1; k < h.nlev; k++) if (h.lev[k].A.nnz < 0) h.lev[k].A.nnz = hf[AF_LNNZ + k];
  }
  for (int k = 0; k < h.nlev; k++) h.lev[k].nnz_prev = h.lev[k].A.nnz;
  for (int k = 0; k < h.nlev && mixed; k++) csr_cast(h.lev[k].A, h.lev[k].A32, s);
  amg_level &C = h.lev[l];
  if (h.coarse_dense) {
    int n = C.A.n;
    if (n > 2048) RS_FAIL(SIM_ERR_ARG, "AMG: coarsest level of %d rows is too large for the dense solve", n);
    dbuf<double> &a = h.dense_a;
    a.ensure((size_t)n * n); h.lu.ensure((size_t)n * n); h.piv.ensure(n);
    k_dense_build<<<grid_for(n, 128), 128, 0, s>>>(n, C.A.rp.p, C.A.ci.p, C.A.v.p, a.p);
    if (n <= 128) {
      static bool attr = false;
      if (!attr) {
        RS_CUDA(cudaFuncSetAttribute(k_dense_lu_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        RS_CUDA(cudaFuncSetAttribute(k_dense_inv_cols<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        RS_CUDA(cudaFuncSetAttribute(k_dense_inv_cols<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        RS_CUDA(cudaFuncSetAttribute(k_dense_inv_cols<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        RS_CUDA(cudaFuncSetAttribute(k_dense_inv_cols<4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
        attr = true;
      }
      h.dense_lu.ensure((size_t)n * n);
      h.dense_rd.ensure(n);
      k_dense_lu_smem<<<1, 512, (size_t)n * n * 8, s>>>(n, a.p, h.piv.p, h.dense_lu.p, h.dense_rd.p);
      const size_t csm = (size_t)n * n * 8 + (size_t)n * 12;
      const unsigned cg = (unsigned)((n + 1) / 2);
      switch ((n + 31) / 32) {
        case 1: k_dense_inv_cols<1><<<cg, 64, csm, s>>>(n, h.dense_lu.p, h.piv.p, h.dense_rd.p, h.lu.p); break;
        case 2: k_dense_inv_cols<2><<<cg, 64, csm, s>>>(n, h.dense_lu.p, h.piv.p, h.dense_rd.p, h.lu.p); break;
        case 3: k_dense_inv_cols<3><<<cg, 64, csm, s>>>(n, h.dense_lu.p, h.piv.p, h.dense_rd.p, h.lu.p); break;
        default: k_dense_inv_cols<4><<<cg, 64, csm, s>>>(n, h.dense_lu.p, h.piv.p, h.dense_rd.p, h.lu.p); break;
      }
      RS_LAUNCHED(1);
    } else {
      k_dense_lu_inv<<<1, 512, 0, s>>>(n, a.p, h.piv.p, h.lu.p);
    }
    RS_LAUNCHED(2);
  }
  RS_CHECK_LAUNCH();
}

// -------------------------------------------------------------- V-cycle ---
template <class T>
__global__ void k_vc_pre(int n, const int *rp, const int *ci, const T *v, const T *dinv, const T *f, T *x, T *r) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  pdl_trigger();
  pdl_wait();
  if (i >= n) return;
  T s = f[i];
  for (int q = rp[i]; q < rp[i + 1]; q++) { int j = ci[q]; s -= v[q] * (f[j] * dinv[j]); }
  x[i] = f[i] * dinv[i];
  r[i] = s;
}
template <class T>
__global__ void k_prolong_add(int n, const int *rp, const int *ci, const T *v, const T *e, const T *x, T *t) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  pdl_trigger();
  pdl_wait();
  if (i >= n) return;
  T s = x[i];
  for (int q = rp[i]; q < rp[i + 1]; q++) s += v[q] * e[ci[q]];
  t[i] = s;
}
template <class T>
__global__ void k_vc_post(int n, const int *rp, const int *ci, const T *v, const T *dinv, const T *f, const T *t, T *x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  pdl_trigger();
  pdl_wait();
  if (i >= n) return;
  T s = f[i];
  for (int q = rp[i]; q < rp[i + 1]; q++) s -= v[q] * t[ci[q]];
  x[i] = t[i] + dinv[i] * s;
}
template <class T>
__global__ void k_restrict_x(int n, const int *rp, const int *ci, const T *v, const T *u, const T *dinv, T *y, T *x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  pdl_trigger();
  pdl_wait();
  if (i >= n) return;
  T s = 0;
  for (int q = rp[i]; q < rp[i + 1]; q++) s += v[q] * u[ci[q]];
  y[i] = s;
  x[i] = s * dinv[i];
}
template <class T>
__global__ void k_jacobi(int n, const int *rp, const int *ci, const T *v, const T *dinv, const T *f, const T *x, T *y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  pdl_trigger();
  pdl_wait();
  if (i >= n) return;
  T s = f[i];
  for (int q = rp[i]; q < rp[i + 1]; q++) s -= v[q] * x[ci[q]];
  y[i] = x[i] + dinv[i] * s;
}
template <class T>
__global__ void k_dense_apply(int n, const double *invT, const T *f, T *x) {
  // x_i = sum_c (A^{-1})_{ic} f_c, invT[c][i]; one warp per row
  pdl_trigger();
  pdl_wait();
  int i = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i >= n) return;
  double s = 0.0;
  for (int c = lane; c < n; c += 32) s += invT[(size_t)c * n + i] * (double)f[c];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if (lane == 0) x[i] = (T)s;
}

// The same four sweeps with L lanes per row (L = 4..32): a row's entries are
// read by consecutive lanes (coalesced), each lane sums a strided part of the
// row and the parts are combined with shuffles.  MODE 0: pre-smoothing
// (x = D^-1 f, r = f - A x; with u given, u already holds D^-1 f); 1: y = A x
// (and, with o2 given, o2 = D_c^-1 y for the coarse level's pre-smoothing);
// 2: t = x + P e; 3: post-smoothing (x = t + D^-1 (f - A t)).
template <class T, int L, int MODE>
__global__ void k_vc_lanes(int n, const int *__restrict__ rp, const int *__restrict__ ci, const T *__restrict__ v,
                           const T *__restrict__ dinv, const T *__restrict__ f, const T *__restrict__ u, T *o1, T *o2) {
  pdl_trigger();
  pdl_wait();
  int g = (blockIdx.x * blockDim.x + threadIdx.x) / L, k = threadIdx.x % L;
  int i = g < n ? g : n - 1;                       // whole groups stay in the shuffles
  int q0 = rp[i], q1 = rp[i + 1];
  T s = 0;
#pragma unroll 4
  for (int q = q0 + k; q < q1; q += L) {
    int j = ci[q];
    T xj = MODE == 0 && !u ? f[j] * dinv[j] : u[j];
    s += v[q] * xj;
  }
#pragma unroll
  for (int o = L / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o, L);
  if (k != 0 || g >= n) return;
  if (MODE == 0) { if (!u) o1[i] = f[i] * dinv[i]; o2[i] = f[i] - s; }   // with u, o1 = u holds it already
  else if (MODE == 1) { o1[i] = s; if (o2) o2[i] = s * dinv[i]; }
  else if (MODE == 2) o1[i] = f[i] + s;            // f = x (the smoothed iterate), u = e
  else o1[i] = u[i] + dinv[i] * (f[i] - s);        // u = t
}

// lanes per row for a matrix's average row length: one thread per row for
// short rows (their loads already coalesce across neighbouring rows), more
// lanes as rows grow (a single thread walking a 40-entry row is latency-bound)
// (measured on the 1M-cell hierarchy: 4 lanes for 9-24 entries per row and
// 16 beyond beat 8/16/32, which left most lanes of a group idle)
static int lanes_for(long long nnz, int n) {
  double avg = n ? (double)nnz / n : 0.0;
  return avg <= 8.0 ? 1 : avg <= 24.0 ? 4 : 16;
}

template <class T>
__global__ void k_vc_pre(int n, const int *rp, const int *ci, const T *v, const T *dinv, const T *f, T *x, T *r);
template <class T>
__global__ void k_prolong_add(int n, const int *rp, const int *ci, const T *v, const T *e, const T *x, T *t);
template <class T>
__global__ void k_vc_post(int n, const int *rp, const int *ci, const T *v, const T *dinv, const T *f, const T *t, T *x);
template <class T>
__global__ void k_csr_spmv(int n, const int *rp, const int *ci, const T *v, const T *x, T *y);

template <class T, int MODE>
static void vc_sweep(int L, int n, const int *rp, const int *ci, const T *v, const T *dinv, const T *f, const T *u,
                     T *o1, T *o2, cudaStream_t s) {
  if (n <= 0) return;
  if (L == 1) {
    unsigned g = grid_for(n, 256);
    if (MODE == 0) launch_pdl(k_vc_pre<T>, g, 256, 0, s, n, rp, ci, v, dinv, f, o1, o2);
    else if (MODE == 1 && o2) launch_pdl(k_restrict_x<T>, g, 256, 0, s, n, rp, ci, v, u, dinv, o1, o2);
    else if (MODE == 1) launch_pdl(k_csr_spmv<T>, g, 256, 0, s, n, rp, ci, v, u, o1);
    else if (MODE == 2) launch_pdl(k_prolong_add<T>, g, 256, 0, s, n, rp, ci, v, u, f, o1);
    else launch_pdl(k_vc_post<T>, g, 256, 0, s, n, rp, ci, v, dinv, f, u, o1);
    RS_LAUNCHED(1);
    return;
  }
  unsigned g = grid_for((size_t)n * L, 256);
  if (L == 4) launch_pdl(k_vc_lanes<T, 4, MODE>, g, 256, 0, s, n, rp, ci, v, dinv, f, u, o1, o2);
  else if (L == 8) launch_pdl(k_vc_lanes<T, 8, MODE>, g, 256, 0, s, n, rp, ci, v, dinv, f, u, o1, o2);
  else if (L == 16) launch_pdl(k_vc_lanes<T, 16, MODE>, g, 256, 0, s, n, rp, ci, v, dinv, f, u, o1, o2);
  else launch_pdl(k_vc_lanes<T, 32, MODE>, g, 256, 0, s, n, rp, ci, v, dinv, f, u, o1, o2);
  RS_LAUNCHED(1);
}

// One level operator as the V-cycle reads it: the FP64 operator's pattern
// with the values of the cycle's precision (the FP32 copies hold values only).
template <class T> struct csr_ref { int n, nnz; const int *rp, *ci; const T *v; };
template <class T> struct lvl_ptrs;
template <> struct lvl_ptrs<double> {
  static csr_ref<double> A(amg_level &L) { return {L.A.n, L.A.nnz, L.A.rp.p, L.A.ci.p, L.A.v.p}; }
  static csr_ref<double> P(amg_level &L) { return {L.P.n, L.P.nnz, L.P.rp.p, L.P.ci.p, L.P.v.p}; }
  static csr_ref<double> R(amg_level &L) { return {L.R.n, L.R.nnz, L.R.rp.p, L.R.ci.p, L.R.v.p}; }
  static double *dinv(amg_level &L) { return L.dinv.p; }
  static double *f(amg_level &L) { return L.f.p; } static double *x(amg_level &L) { return L.x.p; }
  static double *r(amg_level &L) { return L.r.p; } static double *t(amg_level &L) { return L.t.p; }
};
template <> struct lvl_ptrs<float> {
  static csr_ref<float> A(amg_level &L) { return {L.A.n, L.A.nnz, L.A.rp.p, L.A.ci.p, L.A32.v.p}; }
  static csr_ref<float> P(amg_level &L) { return {L.P.n, L.P.nnz, L.P.rp.p, L.P.ci.p, L.P32.v.p}; }
  static csr_ref<float> R(amg_level &L) { return {L.R.n, L.R.nnz, L.R.rp.p, L.R.ci.p, L.R32.v.p}; }
  static float *dinv(amg_level &L) { return L.dinv32.p; }
  static float *f(amg_level &L) { return L.f32.p; } static float *x(amg_level &L) { return L.x32.p; }
  static float *r(amg_level &L) { return L.r32.p; } static float *t(amg_level &L) { return L.t32.p; }
};

template <class T>
int amg_vcycle(amg_hier &h, int l, cudaStream_t s) {
  typedef lvl_ptrs<T> LP;
  amg_level &L = h.lev[l];
  const csr_ref<T> A = LP::A(L);
  int n = A.n;
  if (l == h.nlev - 1) {
    if (h.coarse_dense) {
      launch_pdl(k_dense_apply<T>, grid_for(n, 8), 256, 0, s, n, (const double *)h.lu.p, (const T *)LP::f(L), LP::x(L));
      RS_LAUNCHED(1);
      return 1;
    }
    T *x = LP::x(L), *t = LP::t(L);
    k_vc_pre<T><<<grid_for(n, 256), 256, 0, s>>>(n, A.rp, A.ci, A.v, LP::dinv(L), LP::f(L), x, LP::r(L));
    RS_LAUNCHED(1);
    for (int it = 1; it < 10; it++) {
      k_jacobi<T><<<grid_for(n, 256), 256, 0, s>>>(n, A.rp, A.ci, A.v, LP::dinv(L), LP::f(L), x, t);
      std::swap(x, t);
      RS_LAUNCHED(1);
    }
    if (x != LP::x(L)) RS_CUDA(cudaMemcpyAsync(LP::x(L), x, n * sizeof(T), cudaMemcpyDeviceToDevice, s));
    return 10;
  }
  amg_level &Cl = h.lev[l + 1];
  const csr_ref<T> P = LP::P(L);
  const csr_ref<T> R = LP::R(L);
  int la = lanes_for(A.nnz, n), lr = lanes_for(R.nnz, R.n), lp = lanes_for(P.nnz, n);
  // below level 0 the restriction has already formed x = D^-1 f (pre-smoothing
  // then gathers one vector instead of two; same products, same values)
  vc_sweep<T, 0>(la, n, A.rp, A.ci, A.v, LP::dinv(L), LP::f(L), l > 0 ? LP::x(L) : nullptr, LP::x(L),
                 LP::r(L), s);
  // the coarse level's D^-1 f, unless that level is solved directly
  bool cx = !(l + 1 == h.nlev - 1 && h.coarse_dense);
  vc_sweep<T, 1>(lr, R.n, R.rp, R.ci, R.v, LP::dinv(Cl), nullptr, LP::r(L), LP::f(Cl), cx ? LP::x(Cl) : nullptr, s);
  int k = amg_vcycle<T>(h, l + 1, s);
  vc_sweep<T, 2>(lp, n, P.rp, P.ci, P.v, nullptr, LP::x(L), LP::x(Cl), LP::t(L), nullptr, s);
  vc_sweep<T, 3>(la, n, A.rp, A.ci, A.v, LP::dinv(L), LP::f(L), LP::t(L), LP::x(L), nullptr, s);
  return k + 4;
}
template int amg_vcycle<double>(amg_hier &, int, cudaStream_t);
template int amg_vcycle<float>(amg_hier &, int, cudaStream_t);

// One V-cycle from level 0 as a single graph launch: every buffer it touches
// is fixed between two setups, so the whole recursion (about four kernels per
// level) is recorded once per hierarchy and replayed, which removes the
// per-kernel launch gaps that dominate the small coarse levels.
template <class T>
void amg_vcycle_graph(amg_hier &h, cudaStream_t s) {
  int pi = sizeof(T) == 4 ? 1 : 0;
  if (!h.vc_exec[pi]) {
    if (!h.cap) RS_CUDA(cudaStreamCreateWithFlags(&h.cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    RS_CUDA(cudaStreamBeginCapture(h.cap, cudaStreamCaptureModeThreadLocal));
    int k = 0;
    try {
      k = amg_vcycle<T>(h, 0, h.cap);
    } catch (...) {
      cudaStreamEndCapture(h.cap, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    rs_launches -= k;                              // recorded, not launched
    RS_CUDA(cudaStreamEndCapture(h.cap, &g));
    cudaError_t e = cudaGraphInstantiate(&h.vc_exec[pi], g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { h.vc_exec[pi] = nullptr; RS_CUDA(e); }
    h.vc_launches[pi] = k;
  }
  RS_CUDA(cudaGraphLaunch(h.vc_exec[pi], s));
  RS_LAUNCHED(h.vc_launches[pi]);
}
template void amg_vcycle_graph<double>(amg_hier &, cudaStream_t);
template void amg_vcycle_graph<float>(amg_hier &, cudaStream_t);

template <class T>
__global__ void k_csr_spmv(int n, const int *rp, const int *ci, const T *v, const T *x, T *y) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  pdl_trigger();
  pdl_wait();
  if (i >= n) return;
  T s = 0;
  for (int q = rp[i]; q < rp[i + 1]; q++) s += v[q] * x[ci[q]];
  y[i] = s;
}
template <class T>
void csr_spmv(const int *rp, const int *ci, const T *v, const T *x, T *y, int n, cudaStream_t s) {
  k_csr_spmv<T><<<grid_for(n, 256), 256, 0, s>>>(n, rp, ci, v, x, y);
  RS_LAUNCHED(1);
}
template void csr_spmv<double>(const int *, const int *, const double *, const double *, double *, int, cudaStream_t);
template void csr_spmv<float>(const int *, const int *, const float *, const float *, float *, int, cudaStream_t);
