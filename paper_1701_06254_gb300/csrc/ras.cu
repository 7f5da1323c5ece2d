// Restricted additive Schwarz with block ILU(0) subdomain solves: the
// R(A)^{-1} stages of CPR-FPF (Algorithm 2: the RAS solves that open and
// close it) of arXiv 1701.06254, with the local potential reordering of
// eqs. (30)-(32) applied inside each subdomain.  A subdomain is a column
// tile of tile_x x tile_y cells over all layers (a well goes with the tile
// of its first perforated cell); its local system is the owned rows plus
// every row within graph distance 1 or 2 of them (the overlap, Table 9).  Each subdomain maps to one thread
// block: the potential sort, the level sets of the reordered factors, the
// factorisation and both triangular solves run level by level inside that
// block.
#include "common.cuh"
#include <cuda_bf16.h>
#include <algorithm>
#include <cfloat>
#include <climits>

// Streamed per-subdomain factors for the shared-memory apply.  One warp
// solves one subdomain: its local vector y lives in shared
// memory, and the factors, which each application reads exactly once and in
// a fixed order, flow through a small shared-memory ring filled by bulk
// copies (cp.async.bulk + mbarrier) a few chunks ahead of the sweep.  The
// stream of a subdomain (16-byte aligned pieces):
//   header  {m, L groups, U groups, stream bytes, first group's start and
//           bytes} 32 B
//   groups  the rows of the L sweep (L levels 1.., level 0 has no entries),
//           then the rows of the U sweep (U levels 0..), level by level;
//           a level is split into groups of at most 32 rows (one per lane)
//           and at most one chunk of bytes; a group never straddles the
//           end of the ring (the stream is padded to the next ring period
//           instead), so its pieces are contiguous in shared memory
// A group:
//   {nrows | nent << 16, bytes, next group's start, next group's bytes} 16 B
//   row records: local row, first and end entry   8 B (L) or RREC_U (U, with
//               (group-relative), U: the inverse  the 2x2 block, 4 values)
//               diagonal block
//   cols  u16[nent] | vals [nent][4]   (the row records, the columns and
//   the values each start on a 16-byte boundary)
// The global row of each local row (bit 0: owned) is a separate array
// (gidx), read by the gather and the scatter.
#define RAS_SMEM_BUDGET (200 * 1024)
#define RAS_GROUP_ROWS 32
template <class TB> struct ring_cfg;                       // ring bytes, chunk bytes per stored type
template <> struct ring_cfg<__nv_bfloat16> { static const int R = 4096, C = 1024; };
template <> struct ring_cfg<float> { static const int R = 16384, C = 4096; };
template <> struct ring_cfg<double> { static const int R = 32768, C = 8192; };
// U row record: 8 bytes of indices, then the inverse diagonal block at DOFF
template <class TB> __host__ __device__ constexpr int rrec_doff() { return 4 * (int)sizeof(TB) <= 8 ? 8 : 16; }
template <class TB> __host__ __device__ constexpr int rrec_u() { return (rrec_doff<TB>() + 4 * (int)sizeof(TB) + 15) & ~15; }
// a group's byte cap: one chunk (a group then touches at most two chunks,
// and padding to the next ring period wastes at most a quarter of it)
template <class TB> __host__ __device__ constexpr int group_cap() { return ring_cfg<TB>::C; }
__host__ __device__ inline int al16(int x) { return (x + 15) & ~15; }

// ------------------------------------------------- static partition (host)
void ras_build_static(sim_ls_s *ls) {
  ras_data &R = ls->ras;
  int tx = ls->o.tile_x, ty = ls->o.tile_y;
  int ntx = (ls->nx + tx - 1) / tx, nty = (ls->ny + ty - 1) / ty;
  int nsub = ntx * nty, nb = ls->nb, n = ls->n;
  R.nsub = nsub;
  std::vector<int> owner(nb);
  for (int c = 0; c < n; c++) {
    int i = c % ls->nx, j = (c / ls->nx) % ls->ny;
    owner[c] = (i / tx) + ntx * (j / ty);
  }
  for (int w = 0; w < ls->nw; w++) owner[n + w] = owner[ls->h_wc0[w]];
  std::vector<std::vector<int>> own(nsub);
  for (int r = 0; r < nb; r++) own[owner[r]].push_back(r);
  std::vector<int> sub_ptr(nsub + 1, 0), ext, owned, ncell(nsub), lrp_ptr(nsub + 1, 0), lrlen, lrp, lci, lsrc;
  std::vector<int> mark(nb, 0), loc(nb, -1);
  R.max_ext = 0; R.max_nnz = 0;
  int maxcells = 0;
  for (int s = 0; s < nsub; s++) {
    std::vector<int> list;
    for (int g : own[s])
      if (!mark[g]) { mark[g] = 1; list.push_back(g); }
    // rings of graph neighbours, one per level of overlap (1, or 2: Table 9)
    int ov = ls->o.overlap == 2 ? 2 : 1;
    for (int lev = 0, r0 = 0, r1 = (int)list.size(); lev < ov; lev++, r0 = r1, r1 = (int)list.size())
      for (int a = r0; a < r1; a++) {
        int g = list[a];
        for (int q = ls->h_rp[g]; q < ls->h_rp[g + 1]; q++) {
          int c = ls->h_ci[q];
          if (!mark[c]) { mark[c] = 1; list.push_back(c); }
        }
      }
    std::sort(list.begin(), list.end());      // cells ascending, then wells ascending
    int m = (int)list.size(), base = (int)ext.size(), nc = 0;
    for (int a = 0; a < m; a++) {
      int g = list[a];
      mark[g] = 0; loc[g] = a;
      ext.push_back(g);
      owned.push_back(owner[g] == s);
      nc += g < n;
    }
    ncell[s] = nc;
    maxcells = std::max(maxcells, nc);
    int nnz0 = (int)lci.size();
    for (int a = 0; a < m; a++) {
      int g = list[a], len = 0;
      lrp.push_back((int)lci.size());
      for (int q = ls->h_rp[g]; q < ls->h_rp[g + 1]; q++) {
        int lc = loc[ls->h_ci[q]];
        if (lc < 0) continue;
        lci.push_back(lc); lsrc.push_back(q); len++;
      }
      lrlen.push_back(len);
    }
    for (int a = 0; a < m; a++) loc[list[a]] = -1;
    sub_ptr[s + 1] = base + m;
    lrp_ptr[s + 1] = (int)lci.size();
    R.max_ext = std::max(R.max_ext, m);
    R.max_nnz = std::max(R.max_nnz, (int)lci.size() - nnz0);
  }
  cudaStream_t st = ls->st;
  h2d(R.sub_ptr, sub_ptr, st); h2d(R.ext, ext, st);
  std::vector<uint8_t> ow(owned.begin(), owned.end());
  h2d(R.owned, ow, st); h2d(R.ncell, ncell, st);
  h2d(R.lrp_ptr, lrp_ptr, st); h2d(R.lrlen, lrlen, st); h2d(R.lrp, lrp, st);
  h2d(R.lci, lci, st); h2d(R.lsrc, lsrc, st);
  size_t next_tot = ext.size(), nnz_tot = lci.size();
  R.perm.alloc(next_tot); R.ipos.alloc(next_tot); R.frp.alloc(next_tot + nsub);
  R.fci.alloc(nnz_tot); R.fdiag.alloc(next_tot);
  R.lvl.alloc(2 * next_tot); R.lvl_rows.alloc(2 * next_tot); R.nlev.alloc(2 * nsub);
  R.lvl_ptr.alloc(2 * (next_tot + nsub));
  if (ls->o.precision != SIM_PREC_FP64) { R.fval32.alloc(4 * nnz_tot); R.dinv32.alloc(4 * next_tot); }
  else { R.fval.alloc(4 * nnz_tot); R.dinv.alloc(4 * next_tot); }
  int m = 1;
  while (m < maxcells) m <<= 1;
  R.max_lvl_ptr = m;   // sort width (power of two >= most cells in a subdomain)
  // shared-memory apply: a bound on each subdomain's stream (the grouping
  // follows the level sets of each setup, the bound only rows and entries:
  // at most one group per walked row, each with its header and padding)
  {
    int vb = ls->o.precision == SIM_PREC_FP64 ? 32 : (ls->o.precision == SIM_PREC_MIXED_BF16 ? 8 : 16);
    int ru = ls->o.precision == SIM_PREC_FP64 ? rrec_u<double>()
                                              : (ls->o.precision == SIM_PREC_MIXED_BF16 ? rrec_u<__nv_bfloat16>()
                                                                                        : rrec_u<float>());
    int ring = ls->o.precision == SIM_PREC_FP64 ? ring_cfg<double>::R
                                                : (ls->o.precision == SIM_PREC_MIXED_BF16 ? ring_cfg<__nv_bfloat16>::R
                                                                                          : ring_cfg<float>::R);
    int yb = ls->o.precision == SIM_PREC_FP64 ? 16 : 8;   // local vector: double2 or float2 per row
    std::vector<long long> boff(nsub + 1, 0);
    int mmax = 0;
    bool fits16 = true;
    for (int s2 = 0; s2 < nsub; s2++) {
      long long ms = sub_ptr[s2 + 1] - sub_ptr[s2], nz = lrp_ptr[s2 + 1] - lrp_ptr[s2], e = nz - ms;
      if (ms >= 65535) fits16 = false;
      long long bound = 16 + 2 * ms * (16 + 48) + ms * (8 + ru) + e * (2 + vb);   // header + 3 paddings per group
      bound = bound + bound / 3 + ring;                     // ring-period padding: <= one chunk per ring
      boff[s2 + 1] = boff[s2] + ((bound + 15) & ~15LL);
      mmax = std::max(mmax, (int)ms);
    }
    R.m_max = mmax;
    // the ring, then the local vector, then one product per entry of a group
    // (a group holds at most a chunk: 16-bit column + block per entry)
    int chunk = ring / 4, pmax = chunk / (2 + vb) + 1;
    R.smem_bytes = ((size_t)mmax * yb + 15) / 16 * 16 + ring + (size_t)pmax * yb;
    R.smem_path = fits16 && R.smem_bytes <= RAS_SMEM_BUDGET;
    if (R.smem_path) {
      h2d(R.blob_off, boff, st); R.blob.alloc(boff[nsub]);
      R.gidx.alloc(ext.size()); R.gdesc.alloc(2 * ext.size() + 2 * (size_t)nsub);
    }
  }
  if ((size_t)m * 12 > 200 * 1024) RS_FAIL(SIM_ERR_ARG, "RAS: %d cells per subdomain is too many (reduce tile_x/tile_y)", maxcells);
  if ((size_t)R.max_ext * 16 > 200 * 1024) RS_FAIL(SIM_ERR_ARG, "RAS: subdomain too large");
}

// --------------------------------------------- potential ordering (eq. 30)
// Sort the cells of each subdomain by descending oil potential; equal keys
// keep ascending natural order (ext indices of cells ascend with the natural
// index).  Wells keep their place after the cells (eq. 32).
__global__ void k_ras_order(const int *sub_ptr, const int *ext, const int *ncell, const double *key, int reorder,
                            int *perm, int *ipos) {
  extern __shared__ unsigned char smem[];
  int s = blockIdx.x, base = sub_ptr[s], m = sub_ptr[s + 1] - base, nc = ncell[s];
  int w = 1;
  while (w < nc) w <<= 1;
  long long *k = reinterpret_cast<long long *>(smem);   // integer keys (dkey) of the potentials
  int *id = reinterpret_cast<int *>(k + w);
  if (reorder) {
    const long long kmin = dkey(-DBL_MAX);
    for (int i = threadIdx.x; i < w; i += blockDim.x) {
      if (i < nc) {
        double kv = key[ext[base + i]];
        k[i] = kv > -DBL_MAX ? dkey(kv) : kmin;   // NaN / -inf sort with the padding, before it
        id[i] = i;
      }
      else { k[i] = kmin; id[i] = INT_MAX; }
    }
    __syncthreads();
    for (int kk = 2; kk <= w; kk <<= 1)
      for (int j = kk >> 1; j > 0; j >>= 1) {
        for (int i = threadIdx.x; i < w; i += blockDim.x) {
          int ixj = i ^ j;
          if (ixj > i) {
            // "a before b": larger key first, then smaller index
            long long ka = k[i], kb = k[ixj]; int ia = id[i], ib = id[ixj];
            bool a_first = (ka > kb) || (ka == kb && ia < ib);
            bool up = (i & kk) == 0;
            if (a_first != up) { k[i] = kb; k[ixj] = ka; id[i] = ib; id[ixj] = ia; }
          }
        }
        __syncthreads();
      }
    for (int i = threadIdx.x; i < nc; i += blockDim.x) { perm[base + i] = id[i]; ipos[base + id[i]] = i; }
  } else {
    for (int i = threadIdx.x; i < nc; i += blockDim.x) { perm[base + i] = i; ipos[base + i] = i; }
  }
  for (int i = nc + threadIdx.x; i < m; i += blockDim.x) { perm[base + i] = i; ipos[base + i] = i; }
}

// local pattern in position order; columns sorted by position
__global__ void k_ras_pattern(const int *sub_ptr, const int *lrp_ptr, const int *lrp, const int *lrlen,
                              const int *lci, const int *lsrc, const int *perm, const int *ipos, int *frp, int *fci,
                              int *fdiag, int *fsrc) {
  __shared__ int warp_tot[32];
  __shared__ int carry;
  int s = blockIdx.x, base = sub_ptr[s], m = sub_ptr[s + 1] - base, pbase = lrp_ptr[s];
  int fbase = base + s;                   // frp segment has m + 1 entries
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int c0 = 0; c0 < m; c0 += blockDim.x) {
    int pos = c0 + threadIdx.x, len = pos < m ? lrlen[base + perm[base + pos]] : 0;
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, x = len;
    for (int o = 1; o < 32; o <<= 1) { int y = __shfl_up_sync(0xffffffffu, x, o); if (lane >= o) x += y; }
    if (lane == 31) warp_tot[wid] = x;
    __syncthreads();
    if (wid == 0) {
      int nw = blockDim.x >> 5, v = lane < nw ? warp_tot[lane] : 0, z = v;
      for (int o = 1; o < 32; o <<= 1) { int y = __shfl_up_sync(0xffffffffu, z, o); if (lane >= o) z += y; }
      if (lane < nw) warp_tot[lane] = z - v;
    }
    __syncthreads();
    int excl = carry + warp_tot[wid] + x - len;
    if (pos < m) frp[fbase + pos] = excl;
    __syncthreads();
    if (threadIdx.x == blockDim.x - 1) carry = excl + len;
    __syncthreads();
  }
  if (threadIdx.x == 0) frp[fbase + m] = carry;
  __syncthreads();
  for (int pos = threadIdx.x; pos < m; pos += blockDim.x) {
    int e = perm[base + pos], src0 = lrp[base + e], len = lrlen[base + e], o = pbase + frp[fbase + pos];
    for (int a = 0; a < len; a++) {         // insertion by position
      int c = ipos[base + lci[src0 + a]], q = lsrc[src0 + a], b = o + a - 1;
      while (b >= o && fci[b] > c) { fci[b + 1] = fci[b]; fsrc[b + 1] = fsrc[b]; b--; }
      fci[b + 1] = c; fsrc[b + 1] = q;
    }
    for (int a = 0; a < len; a++) if (fci[o + a] == pos) fdiag[base + pos] = o + a;
  }
}

// Level sets of the subdomain's factors: L level of row i = 1 + the largest
// L level among its columns c < i (0 without such a column), U level the
// same over c > i; rows of a level in ascending position.  The levels are
// the longest paths of the two DAGs, computed for all rows in parallel from
// the pattern in shared memory, each row once its predecessors are done,
// then counted, scanned and filled by one warp each for L and U (ranks
// within a chunk of 32 rows by matching levels, so the fill keeps the
// ascending order).  Blocks
// whose pattern does not fit in shared memory take k_ras_levels_serial.
__global__ void __launch_bounds__(128) k_ras_levels(const int *sub_ptr, const int *lrp_ptr, const int *frp,
                                                    const int *fci, int *lvl, int *lvl_rows, int *nlev,
                                                    int *lvl_ptr, int *err) {
  extern __shared__ int lsm[];
  int s = blockIdx.x, base = sub_ptr[s], m = sub_ptr[s + 1] - base, pbase = lrp_ptr[s], fbase = base + s;
  int nnz = frp[fbase + m] - frp[fbase];
  const int *rpg = frp + fbase, *cig = fci + pbase + frp[fbase];
  int *srp = lsm, *sci = srp + (m + 1), *LvL = sci + nnz, *LvU = LvL + m, *cnt = LvU + m;   // cnt: 2 (m + 1)
  for (int k = threadIdx.x; k <= m; k += blockDim.x) srp[k] = rpg[k] - rpg[0];
  for (int k = threadIdx.x; k < nnz; k += blockDim.x) sci[k] = cig[k];
  for (int k = threadIdx.x; k < m; k += blockDim.x) { LvL[k] = -1; LvU[k] = -1; }
  for (int k = threadIdx.x; k < 2 * (m + 1); k += blockDim.x) cnt[k] = 0;
  __syncthreads();
  // L levels: thread t takes rows t, t + nt, ... ascending and waits (in
  // shared memory) for each column c < i to have its level; every wait is
  // on a lower row, taken earlier by its thread, so the waits end.  U levels
  // the same from the last row down.  Each wait is bounded: past the limit
  // the kernel records code 5 and takes 0 for that level.
  volatile int *vL = LvL, *vU = LvU;
  const int LIMIT = 1 << 22;
  bool bad = false;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    int l = 0;
    for (int q = srp[i]; q < srp[i + 1]; q++) {
      int c = sci[q];
      if (c >= i) break;                            // columns ascending
      int v, spins = 0;
      while ((v = vL[c]) < 0 && ++spins < LIMIT) {}
      if (v < 0) { bad = true; v = 0; }
      l = max(l, v + 1);
    }
    vL[i] = l;
  }
  for (int i = m - 1 - (int)threadIdx.x; i >= 0; i -= blockDim.x) {
    int u = 0;
    for (int q = srp[i + 1] - 1; q >= srp[i]; q--) {
      int c = sci[q];
      if (c <= i) break;
      int v, spins = 0;
      while ((v = vU[c]) < 0 && ++spins < LIMIT) {}
      if (v < 0) { bad = true; v = 0; }
      u = max(u, v + 1);
    }
    vU[i] = u;
  }
  if (bad) atomicExch(err, 5);
  __syncthreads();
  // counts per level, then per warp (0: L, 1: U) the scan and the fill
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    atomicAdd(&cnt[LvL[i]], 1);
    atomicAdd(&cnt[(m + 1) + LvU[i]], 1);
  }
  __syncthreads();
  int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = threadIdx.x; k < m; k += blockDim.x) { lvl[2 * base + k] = LvL[k]; lvl[2 * base + m + k] = LvU[k]; }
  if (wid > 1) return;
  bool upper = wid == 1;
  const int *Lv = upper ? LvU : LvL;
  int *c = cnt + (upper ? m + 1 : 0);
  int *pp = lvl_ptr + 2 * (base + s) + (upper ? m + 1 : 0);
  int *rr = lvl_rows + 2 * base + (upper ? m : 0);
  // number of levels: one past the last non-empty count
  int nl = 0;
  for (int k = lane; k < m; k += 32) if (c[k]) nl = max(nl, k + 1);
  for (int o = 16; o > 0; o >>= 1) nl = max(nl, __shfl_xor_sync(0xffffffffu, nl, o));
  // exclusive scan of the counts into pp[0..nl] and the cursors c[0..nl)
  int run = 0;
  for (int k0 = 0; k0 <= nl; k0 += 32) {
    int k = k0 + lane, v = k < nl ? c[k] : 0, x = v;
    for (int o = 1; o < 32; o <<= 1) { int y = __shfl_up_sync(0xffffffffu, x, o); if (lane >= o) x += y; }
    if (k <= nl) pp[k] = run + x - v;
    if (k < nl) c[k] = run + x - v;
    run += __shfl_sync(0xffffffffu, x, 31);
  }
  __syncwarp();
  for (int i0 = 0; i0 < m; i0 += 32) {
    int i = i0 + lane, lv = i < m ? Lv[i] : -1 - lane;
    unsigned grp = __match_any_sync(0xffffffffu, lv);
    if (i < m) rr[c[lv] + __popc(grp & ((1u << lane) - 1u))] = i;
    __syncwarp();
    if (i < m && lane == __ffs(grp) - 1) c[lv] += __popc(grp);
    __syncwarp();
  }
  if (lane == 0) nlev[2 * s + (upper ? 1 : 0)] = nl;
}

// the same, one thread per triangle walking the rows serially from global
// memory (subdomains whose pattern does not fit in shared memory)
__global__ void k_ras_levels_serial(const int *sub_ptr, const int *lrp_ptr, const int *frp, const int *fci,
                                    int *lvl, int *lvl_rows, int *nlev, int *lvl_ptr) {
  int s = blockIdx.x, base = sub_ptr[s], m = sub_ptr[s + 1] - base, pbase = lrp_ptr[s], fbase = base + s;
  const int *rp_ = frp + fbase, *ci_ = fci + pbase;
  bool upper;
  if (threadIdx.x == 0) upper = false;
  else if (threadIdx.x == 32) upper = true;
  else return;
  int *Lv = lvl + 2 * base + (upper ? m : 0);
  int nl = 0;
  for (int t = 0; t < m; t++) {
    int i = upper ? m - 1 - t : t;
    int lv = 0;
    for (int q = rp_[i]; q < rp_[i + 1]; q++) {
      int c = ci_[q];
      if ((upper ? c > i : c < i) && Lv[c] + 1 > lv) lv = Lv[c] + 1;
    }
    Lv[i] = lv; if (lv + 1 > nl) nl = lv + 1;
  }
  nlev[2 * s + (upper ? 1 : 0)] = nl;
  int *pp = lvl_ptr + 2 * (base + s) + (upper ? m + 1 : 0);
  int *rr = lvl_rows + 2 * base + (upper ? m : 0);
  for (int l = 0; l <= nl; l++) pp[l] = 0;
  for (int i = 0; i < m; i++) pp[Lv[i] + 1]++;
  for (int l = 0; l < nl; l++) pp[l + 1] += pp[l];
  for (int i = 0; i < m; i++) rr[pp[Lv[i]]++] = i;       // counts reused as cursors
  for (int l = nl; l > 0; l--) pp[l] = pp[l - 1];
  pp[0] = 0;
}

// launch order of the apply: subdomains by descending L + U level count
// (a CTA's time grows with its levels; starting the longest first keeps them
// out of the last wave).  One block: counting sort on the clamped key; the
// order within a key is whatever the atomics give (each subdomain writes only
// its own rows, so the order changes no result).
#define RAS_KEYS 4096
__global__ void __launch_bounds__(1024) k_ras_lpt(int nsub, const int *nlev, int *order) {
  __shared__ int cnt[RAS_KEYS];
  for (int k = threadIdx.x; k < RAS_KEYS; k += blockDim.x) cnt[k] = 0;
  __syncthreads();
  for (int s = threadIdx.x; s < nsub; s += blockDim.x) {
    int key = min(nlev[2 * s] + nlev[2 * s + 1], RAS_KEYS - 1);
    atomicAdd(&cnt[RAS_KEYS - 1 - key], 1);                 // descending keys
  }
  __syncthreads();
  if (threadIdx.x == 0) {                                   // exclusive scan (4096 entries)
    int run = 0;
    for (int k = 0; k < RAS_KEYS; k++) { int c = cnt[k]; cnt[k] = run; run += c; }
  }
  __syncthreads();
  for (int s = threadIdx.x; s < nsub; s += blockDim.x) {
    int key = min(nlev[2 * s] + nlev[2 * s + 1], RAS_KEYS - 1);
    order[atomicAdd(&cnt[RAS_KEYS - 1 - key], 1)] = s;
  }
}

template <class T> __device__ __forceinline__ void inv2x2(const T *M, T *I) {
  T det = M[0] * M[3] - M[1] * M[2];
  T r = T(1) / det;
  I[0] = M[3] * r; I[1] = -M[1] * r; I[2] = -M[2] * r; I[3] = M[0] * r;
}

// block ILU(0), level by level (IKJ form per row): for each k < i in the
// row, L_ik = A_ik U_kk^{-1}; A_ij -= L_ik U_kj for j > k present in row i.
template <class T>
__global__ void k_ras_factor(const int *sub_ptr, const int *lrp_ptr, const int *frp, const int *fci, const int *fdiag,
                             const int *fsrc, const double *val, const int *lvl_rows, const int *nlev,
                             const int *lvl_ptr, T *fv, T *dinv, const int *order) {
  int s = order[blockIdx.x], base = sub_ptr[s], m = sub_ptr[s + 1] - base, pbase = lrp_ptr[s], fbase = base + s;
  int q0 = pbase + frp[fbase], q1 = pbase + frp[fbase + m];
  for (int q = q0 + threadIdx.x; q < q1; q += blockDim.x) {   // gather values in factor order
    const double *src = val + 4 * (size_t)fsrc[q];
    fv[4 * (size_t)q + 0] = (T)src[0]; fv[4 * (size_t)q + 1] = (T)src[1];
    fv[4 * (size_t)q + 2] = (T)src[2]; fv[4 * (size_t)q + 3] = (T)src[3];
  }
  __syncthreads();
  const int *pL = lvl_ptr + 2 * (base + s), *rL = lvl_rows + 2 * base;
  int nL = nlev[2 * s];
  for (int l = 0; l < nL; l++) {
    for (int a = pL[l] + threadIdx.x; a < pL[l + 1]; a += blockDim.x) {
      int i = rL[a];
      int r0 = pbase + frp[fbase + i], r1 = pbase + frp[fbase + i + 1];
      for (int q = r0; q < r1; q++) {
        int k = fci[q];
        if (k >= i) break;
        T *Aq = fv + 4 * (size_t)q;
        const T *Dk = dinv + 4 * (size_t)(base + k);
        T l0 = Aq[0] * Dk[0] + Aq[1] * Dk[2], l1 = Aq[0] * Dk[1] + Aq[1] * Dk[3];
        T l2 = Aq[2] * Dk[0] + Aq[3] * Dk[2], l3 = Aq[2] * Dk[1] + Aq[3] * Dk[3];
        Aq[0] = l0; Aq[1] = l1; Aq[2] = l2; Aq[3] = l3;
        int k1 = pbase + frp[fbase + k + 1];
        int qi = q + 1;
        for (int qk = fdiag[base + k] + 1; qk < k1; qk++) {
          int j = fci[qk];
          while (qi < r1 && fci[qi] < j) qi++;
          if (qi >= r1) break;
          if (fci[qi] != j) continue;
          const T *U = fv + 4 * (size_t)qk;
          T *A = fv + 4 * (size_t)qi;
          A[0] -= l0 * U[0] + l1 * U[2]; A[1] -= l0 * U[1] + l1 * U[3];
          A[2] -= l2 * U[0] + l3 * U[2]; A[3] -= l2 * U[1] + l3 * U[3];
        }
      }
      inv2x2(fv + 4 * (size_t)fdiag[base + i], dinv + 4 * (size_t)(base + i));
    }
    __syncthreads();
  }
}

void ras_pack(sim_ls_s *ls);
void ras_setup(sim_ls_s *ls) {
  ras_data &R = ls->ras;
  cudaStream_t s = ls->st;
  int w = R.max_lvl_ptr;
  size_t smem = (size_t)w * 12;
  static bool attr = false;
  if (!attr) {
    RS_CUDA(cudaFuncSetAttribute(k_ras_order, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr = true;
  }
  k_ras_order<<<R.nsub, 512, smem, s>>>(R.sub_ptr.p, R.ext.p, R.ncell.p, ls->key.p, ls->o.reorder, R.perm.p, R.ipos.p);
  static thread_local dbuf<int> fsrc;
  fsrc.ensure(R.lci.n);
  k_ras_pattern<<<R.nsub, 256, 0, s>>>(R.sub_ptr.p, R.lrp_ptr.p, R.lrp.p, R.lrlen.p, R.lci.p, R.lsrc.p, R.perm.p,
                                       R.ipos.p, R.frp.p, R.fci.p, R.fdiag.p, fsrc.p);
  // level sets from shared memory when the largest pattern fits
  size_t lsmem = (5 * (size_t)R.max_ext + 3 + (size_t)R.max_nnz) * sizeof(int);
  static bool lattr = false;
  if (!lattr) {
    RS_CUDA(cudaFuncSetAttribute(k_ras_levels, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    lattr = true;
  }
  if (lsmem <= 200 * 1024)
    k_ras_levels<<<R.nsub, 128, lsmem, s>>>(R.sub_ptr.p, R.lrp_ptr.p, R.frp.p, R.fci.p, R.lvl.p, R.lvl_rows.p,
                                            R.nlev.p, R.lvl_ptr.p, ls->errw_dev);
  else
    k_ras_levels_serial<<<R.nsub, 64, 0, s>>>(R.sub_ptr.p, R.lrp_ptr.p, R.frp.p, R.fci.p, R.lvl.p, R.lvl_rows.p,
                                              R.nlev.p, R.lvl_ptr.p);
  // longest subdomains first for the factorisation and the applies (their
  // CTAs' times grow with the level counts)
  R.order.ensure(R.nsub);
  k_ras_lpt<<<1, 1024, 0, s>>>(R.nsub, R.nlev.p, R.order.p);
  if (ls->o.precision != SIM_PREC_FP64)
    k_ras_factor<float><<<R.nsub, 128, 0, s>>>(R.sub_ptr.p, R.lrp_ptr.p, R.frp.p, R.fci.p, R.fdiag.p, fsrc.p,
                                               ls->val.p, R.lvl_rows.p, R.nlev.p, R.lvl_ptr.p, R.fval32.p, R.dinv32.p,
                                               R.order.p);
  else
    k_ras_factor<double><<<R.nsub, 128, 0, s>>>(R.sub_ptr.p, R.lrp_ptr.p, R.frp.p, R.fci.p, R.fdiag.p, fsrc.p,
                                                ls->val.p, R.lvl_rows.p, R.nlev.p, R.lvl_ptr.p, R.fval.p, R.dinv.p,
                                                R.order.p);
  // (measured: the same factorisation with the subdomain in shared memory
  // took 4.2 against 1.2 ms on the 1M-cell case: 94 KB per block left two
  // blocks per SM, and the level loop's time is not its loads')
  RS_LAUNCHED(5);
  ras_pack(ls);
  R.built = true;
  RS_CHECK_LAUNCH();
}

// x = R(A)^{-1} f: gather the local right-hand side in position order,
// forward solve with L (unit diagonal) level by level, backward solve with U,
// write back the owned rows only.
template <class T>
__global__ void k_ras_apply(const int *sub_ptr, const int *ext, const uint8_t *owned, const int *lrp_ptr,
                            const int *frp, const int *fci, const int *fdiag, const int *perm, const int *lvl_rows,
                            const int *nlev, const int *lvl_ptr, const T *fv, const T *dinv, const T *f, T *x) {
  extern __shared__ unsigned char smem_raw[];
  T *y = reinterpret_cast<T *>(smem_raw);
  int s = blockIdx.x, base = sub_ptr[s], m = sub_ptr[s + 1] - base, pbase = lrp_ptr[s], fbase = base + s;
  for (int pos = threadIdx.x; pos < m; pos += blockDim.x) {
    int g = ext[base + perm[base + pos]];
    y[2 * pos] = f[2 * (size_t)g]; y[2 * pos + 1] = f[2 * (size_t)g + 1];
  }
  __syncthreads();
  const int *pL = lvl_ptr + 2 * (base + s), *pU = pL + (m + 1);
  const int *rL = lvl_rows + 2 * base, *rU = rL + m;
  int nL = nlev[2 * s], nU = nlev[2 * s + 1];
  for (int l = 1; l < nL; l++) {                 // level 0 rows have no L entries
    for (int a = pL[l] + threadIdx.x; a < pL[l + 1]; a += blockDim.x) {
      int i = rL[a];
      T y0 = y[2 * i], y1 = y[2 * i + 1];
      for (int q = pbase + frp[fbase + i]; q < fdiag[base + i]; q++) {
        const T *B = fv + 4 * (size_t)q; int c = fci[q];
        T c0 = y[2 * c], c1 = y[2 * c + 1];
        y0 -= B[0] * c0 + B[1] * c1; y1 -= B[2] * c0 + B[3] * c1;
      }
      y[2 * i] = y0; y[2 * i + 1] = y1;
    }
    __syncthreads();
  }
  for (int l = 0; l < nU; l++) {
    for (int a = pU[l] + threadIdx.x; a < pU[l + 1]; a += blockDim.x) {
      int i = rU[a];
      T y0 = y[2 * i], y1 = y[2 * i + 1];
      int r1 = pbase + frp[fbase + i + 1];
      for (int q = fdiag[base + i] + 1; q < r1; q++) {
        const T *B = fv + 4 * (size_t)q; int c = fci[q];
        T c0 = y[2 * c], c1 = y[2 * c + 1];
        y0 -= B[0] * c0 + B[1] * c1; y1 -= B[2] * c0 + B[3] * c1;
      }
      const T *D = dinv + 4 * (size_t)(base + i);
      y[2 * i] = D[0] * y0 + D[1] * y1; y[2 * i + 1] = D[2] * y0 + D[3] * y1;
    }
    __syncthreads();
  }
  for (int pos = threadIdx.x; pos < m; pos += blockDim.x) {
    int e = perm[base + pos];
    if (owned[base + e]) {
      int g = ext[base + e];
      x[2 * (size_t)g] = y[2 * pos]; x[2 * (size_t)g + 1] = y[2 * pos + 1];
    }
  }
}

// pack the factors of each subdomain into its blob (one block per subdomain)
template <class TB> __device__ __forceinline__ TB to_blob(float v);
template <> __device__ __forceinline__ float to_blob<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 to_blob<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }
template <class TB> __device__ __forceinline__ TB to_blob_d(double v) { return to_blob<TB>((float)v); }
template <> __device__ __forceinline__ double to_blob_d<double>(double v) { return v; }
__device__ __forceinline__ float from_blob(float v) { return v; }
__device__ __forceinline__ double from_blob(double v) { return v; }
__device__ __forceinline__ float from_blob(__nv_bfloat16 v) { return __bfloat162float(v); }
// one 2x2 block of the packed factors in a single shared-memory load
__device__ __forceinline__ void blk4(const __nv_bfloat16 *B, float &b0, float &b1, float &b2, float &b3) {
  uint2 u = *reinterpret_cast<const uint2 *>(B);
  __nv_bfloat162 lo = *reinterpret_cast<__nv_bfloat162 *>(&u.x), hi = *reinterpret_cast<__nv_bfloat162 *>(&u.y);
  b0 = __low2float(lo); b1 = __high2float(lo); b2 = __low2float(hi); b3 = __high2float(hi);
}
__device__ __forceinline__ void blk4(const float *B, float &b0, float &b1, float &b2, float &b3) {
  float4 v = *reinterpret_cast<const float4 *>(B);
  b0 = v.x; b1 = v.y; b2 = v.z; b3 = v.w;
}
__device__ __forceinline__ void blk4(const double *B, double &b0, double &b1, double &b2, double &b3) {
  double2 u = reinterpret_cast<const double2 *>(B)[0], v = reinterpret_cast<const double2 *>(B)[1];
  b0 = u.x; b1 = u.y; b2 = v.x; b3 = v.y;
}
// a -= sum over q in [q0, q1) of B_q y[cols[q]], in the order of q; the
// entries are taken four at a time so that their column and block loads,
// then their y loads, are in flight together
template <class T, class T2, class TB>
__device__ __forceinline__ void row_sub(T2 &a, int q0, int q1, const uint16_t *cols, const TB *vals, const T2 *y) {
  for (int q = q0; q < q1; q += 4) {
    int c[4];
    T bb[4][4];
#pragma unroll
    for (int u = 0; u < 4; u++)
      if (q + u < q1) { c[u] = cols[q + u]; blk4(vals + 4 * (q + u), bb[u][0], bb[u][1], bb[u][2], bb[u][3]); }
    T2 yc[4];
#pragma unroll
    for (int u = 0; u < 4; u++)
      if (q + u < q1) yc[u] = y[c[u]];
#pragma unroll
    for (int u = 0; u < 4; u++)
      if (q + u < q1) { a.x -= bb[u][0] * yc[u].x + bb[u][1] * yc[u].y; a.y -= bb[u][2] * yc[u].x + bb[u][3] * yc[u].y; }
  }
}

// T: factor type (FP32 or FP64), TB: stored value type (T, or BF16).
// One block per subdomain.  Thread 0 splits the levels into groups (at most
// 32 rows and group_cap bytes each) and lays them out; then each warp fills
// whole groups: row records (with the inverse diagonal block for U rows),
// columns and values in the row's entry order.
template <class T, class TB>
__global__ void k_ras_pack(const int *sub_ptr, const int *lrp_ptr, const int *ext, const uint8_t *owned,
                           const int *perm, const int *frp, const int *fci, const int *fdiag, const T *fv,
                           const T *dinv, const int *lvl_rows, const int *nlev, const int *lvl_ptr,
                           const long long *blob_off, unsigned char *blobs, int *gidx, int4 *gdesc,
                           const int *order, int *err) {
  int s = order[blockIdx.x], base = sub_ptr[s], m = sub_ptr[s + 1] - base, pbase = lrp_ptr[s], fbase = base + s;
  const int *pL = lvl_ptr + 2 * (base + s), *pU = pL + (m + 1);
  const int *rL = lvl_rows + 2 * base, *rU = rL + m;
  int nL = nlev[2 * s], nU = nlev[2 * s + 1];
  unsigned char *b = blobs + blob_off[s];
  int4 *gd = gdesc + 2 * (base + s);                 // room for 2 (m + 1) groups
  const int VB = 4 * (int)sizeof(TB), RU = rrec_u<TB>(), CAP = group_cap<TB>(), RB = ring_cfg<TB>::R;
  __shared__ int ngr[3];
  // dynamic shared memory: per level its group count (then the first group's
  // index), per group its bytes
  extern __shared__ int psm[];
  const int nlevels = (nL > 1 ? nL - 1 : 0) + nU;
  int *lgc = psm, *gby = psm + nlevels + 1;
  // row i's entries in the factor: [frp, diag) lower, (diag, frp next) upper
  auto nlo = [&](int i) { return fdiag[base + i] - pbase - frp[fbase + i]; };
  auto nup = [&](int i) { return frp[fbase + i + 1] - (fdiag[base + i] - pbase) - 1; };
  // level lv of the sweep order: L levels 1..nL-1, then U levels 0..nU-1
  auto level_of = [&](int lv, int &sweep, int &a, int &a1) {
    int nLw = nL > 1 ? nL - 1 : 0;
    sweep = lv >= nLw;
    int l = sweep ? lv - nLw : lv + 1;
    const int *pp = sweep ? pU : pL;
    a = pp[l]; a1 = pp[l + 1];
  };
  // split one level into groups of at most RAS_GROUP_ROWS rows and CAP bytes;
  // emit(first, rows, entries) for each group in order
  auto split = [&](int lv, auto emit) {
    int sweep, a, a1;
    level_of(lv, sweep, a, a1);
    const int *rr = sweep ? rU : rL;
    int rrec = sweep ? RU : 8;
    while (a < a1) {
      int rows = 0, ent = 0;
      for (;;) {
        if (a + rows >= a1 || rows == RAS_GROUP_ROWS) break;
        int i = rr[a + rows], ne = sweep ? nup(i) : nlo(i);
        int nb = 16 + al16((rows + 1) * rrec) + al16(2 * (ent + ne)) + (ent + ne) * VB;
        if (rows > 0 && nb > CAP) break;
        rows++; ent += ne;
      }
      emit(a, rows, ent, sweep);
      a += rows;
    }
  };
  for (int lv = threadIdx.x; lv < nlevels; lv += blockDim.x) {       // groups per level
    int c = 0;
    split(lv, [&](int, int, int, int) { c++; });
    lgc[lv] = c;
  }
  __syncthreads();
  if (threadIdx.x == 0) {                                            // first group of each level
    int acc = 0, nLw = nL > 1 ? nL - 1 : 0, ngL = 0;
    for (int lv = 0; lv < nlevels; lv++) { int c = lgc[lv]; lgc[lv] = acc; acc += c; if (lv == nLw - 1) ngL = acc; }
    lgc[nlevels] = acc;
    ngr[0] = nLw > 0 ? ngL : 0; ngr[1] = acc - ngr[0];
  }
  __syncthreads();
  for (int lv = threadIdx.x; lv < nlevels; lv += blockDim.x) {       // descriptors and bytes
    int g = lgc[lv];
    split(lv, [&](int a, int rows, int ent, int sweep) {
      int rrec = sweep ? RU : 8;
      gd[g] = make_int4(a, rows, ent, sweep);
      gby[g] = al16(16 + al16(rows * rrec) + al16(2 * ent) + ent * VB);
      g++;
    });
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // offsets: groups in order after a 32-byte stream header, none across the
    // end of a ring period (moved to the next period instead)
    int ng = ngr[0] + ngr[1], off = 32;
    for (int g = 0; g < ng; g++) {
      int gb = gby[g];
      if ((off & (RB - 1)) + gb > RB) off = (off + RB - 1) & ~(RB - 1);
      gd[g].w = (off << 1) | gd[g].w;
      off += gb;
    }
    // the stream must fit its bound (rows and entries only); never true by
    // construction, checked so that a violation is an error, not an overrun
    if ((long long)off > blob_off[s + 1] - blob_off[s]) { atomicExch(err, 4); ngr[0] = 0; ngr[1] = 0; off = 32; ng = 0; }
    ngr[2] = off;
    int *hdr = (int *)b;
    hdr[0] = m; hdr[1] = ngr[0]; hdr[2] = ngr[1]; hdr[3] = off;
    // each group records the next one's start and size: the stream header the first's
    hdr[4] = ng ? (gd[0].w >> 1) : 0;
    hdr[5] = ng ? gby[0] : 0;
  }
  __syncthreads();
  int ng = ngr[0] + ngr[1];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  for (int g = wid; g < ng; g += nwarps) {
    int4 d = gd[g];
    int sweep = d.w & 1, goff = d.w >> 1, rows = d.y, ent = d.z, rrec = sweep ? RU : 8;
    const int *rr = sweep ? rU : rL;
    unsigned char *G = b + goff;
    uint16_t *cols = (uint16_t *)(G + 16 + al16(rows * rrec));
    TB *vals = (TB *)(G + 16 + al16(rows * rrec) + al16(2 * ent));
    int i = lane < rows ? rr[d.x + lane] : 0;
    int ne = lane < rows ? (sweep ? nup(i) : nlo(i)) : 0;
    int e0 = ne;                                      // exclusive prefix of the entry counts
    for (int o = 1; o < 32; o <<= 1) { int y = __shfl_up_sync(0xffffffffu, e0, o); if (lane >= o) e0 += y; }
    e0 -= ne;
    if (lane == 0) {
      int *h = (int *)G;
      h[0] = rows | (ent << 16); h[1] = al16(16 + al16(rows * rrec) + al16(2 * ent) + ent * VB);
      h[2] = g + 1 < ng ? (gd[g + 1].w >> 1) : 0;                    // where the next group starts
      h[3] = g + 1 < ng ? gby[g + 1] : 0;                              // and its bytes
    }
    if (lane < rows) {
      uint16_t *rec = (uint16_t *)(G + 16 + lane * rrec);
      rec[0] = (uint16_t)i; rec[1] = (uint16_t)e0; rec[2] = (uint16_t)(e0 + ne); rec[3] = 0;
      if (sweep) {
        TB *dv = (TB *)((unsigned char *)rec + rrec_doff<TB>());
        const T *dsrc = dinv + 4 * (size_t)(base + i);
        for (int u = 0; u < 4; u++) dv[u] = to_blob_d<TB>(dsrc[u]);
      }
      int q0 = sweep ? fdiag[base + i] - pbase + 1 : frp[fbase + i];
      for (int k = 0; k < ne; k++) {
        int q = q0 + k;
        cols[e0 + k] = (uint16_t)fci[pbase + q];
        const T *src = fv + 4 * (size_t)(pbase + q);
        for (int u = 0; u < 4; u++) vals[4 * (e0 + k) + u] = to_blob_d<TB>(src[u]);
      }
    }
  }
  for (int pos = threadIdx.x; pos < m; pos += blockDim.x) {
    int x = perm[base + pos];
    gidx[base + pos] = (ext[base + x] << 1) | (owned[base + x] ? 1 : 0);
  }
}

// one 2x2 block from the ring at stream offset off: a 32-byte FP64 block
// may wrap around the ring's end, so its two 16-byte halves are addressed
// separately (16-byte alignment keeps every other element whole)
template <int RB> __device__ __forceinline__ void ring_blk4(const unsigned char *ring, int off, const __nv_bfloat16 *,
                                                           float &b0, float &b1, float &b2, float &b3) {
  blk4(reinterpret_cast<const __nv_bfloat16 *>(ring + (off & (RB - 1))), b0, b1, b2, b3);
}
template <int RB> __device__ __forceinline__ void ring_blk4(const unsigned char *ring, int off, const float *,
                                                           float &b0, float &b1, float &b2, float &b3) {
  blk4(reinterpret_cast<const float *>(ring + (off & (RB - 1))), b0, b1, b2, b3);
}
template <int RB> __device__ __forceinline__ void ring_blk4(const unsigned char *ring, int off, const double *,
                                                           double &b0, double &b1, double &b2, double &b3) {
  double2 u = *reinterpret_cast<const double2 *>(ring + (off & (RB - 1)));
  double2 v = *reinterpret_cast<const double2 *>(ring + ((off + 16) & (RB - 1)));
  b0 = u.x; b1 = u.y; b2 = v.x; b3 = v.y;
}

// explicit round-to-nearest products and sums (no contraction): the
// entry-parallel sweep forms B_e y_c = fma(b0, y0, b1 y1) and subtracts it
__device__ __forceinline__ float r_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double r_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float r_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double r_fma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float r_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double r_sub(double a, double b) { return __dsub_rn(a, b); }

template <class T> struct v2_t;
template <> struct v2_t<float> { typedef float2 type; };
template <> struct v2_t<double> { typedef double2 type; };

// ------------------------------------------------ bulk copies (TMA) ------
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// bounded wait: gives up after `limit` polls, records `code` in *err and
// returns false (the hardware copies themselves cannot stall forever; the
// bound only turns a fault into an error status instead of a hang)
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, int *err, int code) {
  for (int it = 0; it < (1 << 22); it++)
    if (mbar_try_wait(bar, parity)) return true;
  atomicExch(err, code);
  return false;
}

// x = R(A)^{-1} f, one warp per subdomain (one warp per block).  Lane 0
// keeps the ring NSLOT chunks ahead of the sweep with bulk copies; every lane
// waits on a chunk's mbarrier before reading it (bounded waits).  The sweep
// takes one group at a time: lane r solves row r of the group (its entries
// in stored order), then the warp synchronises; at the end the owned rows
// are written (or added).
template <class T, class Tin, bool ACC, class TB>
__global__ void __launch_bounds__(32) k_ras_apply_stream(const long long *blob_off, const unsigned char *blobs,
                                                        const int *gidx_all, const int *sub_ptr, const int *order,
                                                        const Tin *__restrict__ f, T *__restrict__ x, int *err,
                                                        int m_max_all) {
  constexpr int RB = ring_cfg<TB>::R, CB = ring_cfg<TB>::C, NSLOT = RB / CB, RU = rrec_u<TB>();
  extern __shared__ uint4 sm4[];
  __shared__ uint64_t bar[NSLOT];
  typedef typename v2_t<T>::type T2;
  typedef typename v2_t<Tin>::type Tin2;
  const int lane = threadIdx.x;
  const int s = order[blockIdx.x];
  const unsigned char *st = blobs + blob_off[s];
  const int *gidx = gidx_all + sub_ptr[s];
  unsigned char *ring = reinterpret_cast<unsigned char *>(sm4);
  T2 *y = reinterpret_cast<T2 *>(ring + RB);
  const int m = sub_ptr[s + 1] - sub_ptr[s];
  T2 *P = reinterpret_cast<T2 *>(reinterpret_cast<unsigned char *>(y) + (((size_t)m_max_all * sizeof(T2) + 15) & ~(size_t)15));
  // header: m, L groups, U groups, stream bytes, first group's start and bytes
  const int4 hd = *reinterpret_cast<const int4 *>(st);
  const int ngL = hd.y, ng = hd.y + hd.z, total = hd.w;
  int cons = reinterpret_cast<const int *>(st)[4];
  int cur = reinterpret_cast<const int *>(st)[5];   // the group's bytes (each header names the next one's)
  const int nchunk = (total + CB - 1) / CB;
  if (lane == 0) {
    for (int k = 0; k < NSLOT; k++) mbar_init(&bar[k], 1);
    mbar_fence_init();
  }
  __syncwarp();
  int issued = 0;                                    // lane 0: chunks issued
  auto issue_upto = [&](int lim) {
    for (; issued < lim && issued < nchunk; issued++) {
      int len = total - issued * CB < CB ? total - issued * CB : CB;
      uint64_t *bk = &bar[issued % NSLOT];
      mbar_arrive_expect_tx(bk, (unsigned)len);
      bulk_g2s(ring + (issued % NSLOT) * CB, st + (size_t)issued * CB, (unsigned)len, bk);
    }
  };
  if (lane == 0) issue_upto(NSLOT);
  // gather the extended right-hand side (overlaps the first bulk copies)
  const Tin2 *f2 = reinterpret_cast<const Tin2 *>(f);
  for (int p0 = lane; p0 < m; p0 += 8 * 32) {
    Tin2 v[8];
#pragma unroll
    for (int u = 0; u < 8; u++) { int pos = p0 + u * 32; if (pos < m) v[u] = f2[gidx[pos] >> 1]; }
#pragma unroll
    for (int u = 0; u < 8; u++) {
      int pos = p0 + u * 32;
      if (pos < m) { T2 t; t.x = (T)v[u].x; t.y = (T)v[u].y; y[pos] = t; }
    }
  }
  __syncwarp();
  int landed = 0, freed = 0;                         // chunks waited for; chunks behind the sweep
  bool ok = true;
  for (int g = 0; g < ng; g++) {
    // the whole group, its size known from the previous header
    int need = (cons + cur + CB - 1) / CB;
    for (; landed < need && ok; landed++) ok = mbar_wait_bounded(&bar[landed % NSLOT], (landed / NSLOT) & 1, err, 3);
    if (!__all_sync(0xffffffffu, ok)) return;
    const unsigned char *G = ring + (cons & (RB - 1));         // the group is contiguous in the ring
    const int4 h4 = *reinterpret_cast<const int4 *>(G);
    const int rows = h4.x & 0xffff, ent = h4.x >> 16;
    const bool up = g >= ngL;
    const int rrec = up ? RU : 8;
    const uint16_t *cols = reinterpret_cast<const uint16_t *>(G + 16 + al16(rows * rrec));
    const TB *vals = reinterpret_cast<const TB *>(G + 16 + al16(rows * rrec) + al16(2 * ent));
    // every entry's product B_e y_c with all lanes (the columns belong to
    // earlier levels, final already), then each row subtracts its own
    // products in stored order
    for (int e = lane; e < ent; e += 32) {
      T b0, b1, b2, b3;
      blk4(vals + 4 * e, b0, b1, b2, b3);
      T2 yc = y[cols[e]], pe;
      pe.x = r_fma(b0, yc.x, r_mul(b1, yc.y));
      pe.y = r_fma(b2, yc.x, r_mul(b3, yc.y));
      P[e] = pe;
    }
    __syncwarp();
    if (lane < rows) {
      const unsigned char *rec = G + 16 + lane * rrec;
      const uint2 ri = *reinterpret_cast<const uint2 *>(rec);
      const int i = ri.x & 0xffff, e0 = ri.x >> 16, e1 = ri.y & 0xffff;
      T2 a = y[i];
      for (int e = e0; e < e1; e++) {
        T2 pe = P[e];
        a.x = r_sub(a.x, pe.x);
        a.y = r_sub(a.y, pe.y);
      }
      if (up) {
        T d0, d1, d2, d3;
        blk4(reinterpret_cast<const TB *>(rec + rrec_doff<TB>()), d0, d1, d2, d3);
        T2 o;
        o.x = d0 * a.x + d1 * a.y; o.y = d2 * a.x + d3 * a.y;
        y[i] = o;
      } else {
        y[i] = a;
      }
    }
    cons = h4.z;                                     // the next group's start
    cur = h4.w;                                      // and bytes
    __syncwarp();
    // chunks wholly behind the sweep are free: refill them
    if (lane == 0 && cons / CB > freed) {
      freed = cons / CB;
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      issue_upto(freed + NSLOT);
    }
  }
  for (int pos = lane; pos < m; pos += 32) {
    int gi = gidx[pos];
    if (gi & 1) {
      size_t gg = (size_t)(gi >> 1);
      T2 v = y[pos];
      if (ACC) { x[2 * gg] += v.x; x[2 * gg + 1] += v.y; }
      else { x[2 * gg] = v.x; x[2 * gg + 1] = v.y; }
    }
  }
}

void ras_pack(sim_ls_s *ls) {
  ras_data &R = ls->ras;
  if (!R.smem_path) return;
  size_t psmem = (4 * (size_t)R.m_max + 8) * sizeof(int);      // level group counts and group bytes
  static bool pattr = false;
  if (!pattr) {
    RS_CUDA(cudaFuncSetAttribute(k_ras_pack<float, __nv_bfloat16>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    RS_CUDA(cudaFuncSetAttribute(k_ras_pack<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    RS_CUDA(cudaFuncSetAttribute(k_ras_pack<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    pattr = true;
  }
#define RAS_PACK_ARGS R.sub_ptr.p, R.lrp_ptr.p, R.ext.p, R.owned.p, R.perm.p, R.frp.p, R.fci.p, R.fdiag.p
  if (ls->o.precision == SIM_PREC_MIXED_BF16)
    k_ras_pack<float, __nv_bfloat16><<<R.nsub, 128, psmem, ls->st>>>(RAS_PACK_ARGS, R.fval32.p, R.dinv32.p, R.lvl_rows.p,
                                                                R.nlev.p, R.lvl_ptr.p, R.blob_off.p, R.blob.p,
                                                                R.gidx.p, R.gdesc.p, R.order.p, ls->errw_dev);
  else if (ls->o.precision != SIM_PREC_FP64)
    k_ras_pack<float, float><<<R.nsub, 128, psmem, ls->st>>>(RAS_PACK_ARGS, R.fval32.p, R.dinv32.p, R.lvl_rows.p, R.nlev.p,
                                                        R.lvl_ptr.p, R.blob_off.p, R.blob.p, R.gidx.p, R.gdesc.p,
                                                        R.order.p, ls->errw_dev);
  else
    k_ras_pack<double, double><<<R.nsub, 128, psmem, ls->st>>>(RAS_PACK_ARGS, R.fval.p, R.dinv.p, R.lvl_rows.p, R.nlev.p,
                                                          R.lvl_ptr.p, R.blob_off.p, R.blob.p, R.gidx.p, R.gdesc.p,
                                                          R.order.p, ls->errw_dev);
#undef RAS_PACK_ARGS
  RS_LAUNCHED(1);
}

template <class T, class Tin>
__global__ void k_cast_acc(size_t m, const Tin *a, T *b, bool acc) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < m) b[i] = acc ? b[i] + (T)a[i] : (T)a[i];
}

template <class T, class Tin, class TB>
static void ras_apply_go(sim_ls_s *ls, const Tin *f, T *x, bool acc) {
  ras_data &R = ls->ras;
  if (acc)
    k_ras_apply_stream<T, Tin, true, TB><<<R.nsub, 32, R.smem_bytes, ls->st>>>(R.blob_off.p, R.blob.p, R.gidx.p,
                                                                              R.sub_ptr.p, R.order.p, f, x, ls->errw_dev,
                                                                              R.m_max);
  else
    k_ras_apply_stream<T, Tin, false, TB><<<R.nsub, 32, R.smem_bytes, ls->st>>>(R.blob_off.p, R.blob.p, R.gidx.p,
                                                                               R.sub_ptr.p, R.order.p, f, x, ls->errw_dev,
                                                                               R.m_max);
}
template <class T, class Tin> static void ras_apply_launch(sim_ls_s *ls, const Tin *f, T *x, bool acc);
template <> void ras_apply_launch<double, double>(sim_ls_s *ls, const double *f, double *x, bool acc) {
  ras_apply_go<double, double, double>(ls, f, x, acc);
}
template <> void ras_apply_launch<float, float>(sim_ls_s *ls, const float *f, float *x, bool acc) {
  if (ls->o.precision == SIM_PREC_MIXED_BF16) ras_apply_go<float, float, __nv_bfloat16>(ls, f, x, acc);
  else ras_apply_go<float, float, float>(ls, f, x, acc);
}
template <> void ras_apply_launch<float, double>(sim_ls_s *ls, const double *f, float *x, bool acc) {
  if (ls->o.precision == SIM_PREC_MIXED_BF16) ras_apply_go<float, double, __nv_bfloat16>(ls, f, x, acc);
  else ras_apply_go<float, double, float>(ls, f, x, acc);
}

template <class T, class Tin> void ls_ras_apply(sim_ls_s *ls, const Tin *f, T *x, bool accumulate) {
  ras_data &R = ls->ras;
  cudaStream_t s = ls->st;
  if (R.smem_path) {
    static bool attr = false;
    if (!attr) {
#define RAS_ATTR(...) RS_CUDA(cudaFuncSetAttribute(k_ras_apply_stream<__VA_ARGS__>, cudaFuncAttributeMaxDynamicSharedMemorySize, RAS_SMEM_BUDGET))
      RAS_ATTR(float, float, false, float); RAS_ATTR(float, float, true, float);
      RAS_ATTR(float, double, false, float); RAS_ATTR(float, double, true, float);
      RAS_ATTR(float, float, false, __nv_bfloat16); RAS_ATTR(float, float, true, __nv_bfloat16);
      RAS_ATTR(float, double, false, __nv_bfloat16); RAS_ATTR(float, double, true, __nv_bfloat16);
      RAS_ATTR(double, double, false, double); RAS_ATTR(double, double, true, double);
#undef RAS_ATTR
      attr = true;
    }
    rs_timed tm(ls, SIM_T_RAS);
    ras_apply_launch<T, Tin>(ls, f, x, accumulate);
    RS_LAUNCHED(1);
    return;
  }
  // global-memory path (subdomains too large for shared memory)
  size_t nu = 2 * (size_t)ls->nb;
  static thread_local dbuf<T> tin, tout;
  const T *fin = reinterpret_cast<const T *>(f);
  if (sizeof(Tin) != sizeof(T)) {
    tin.ensure(nu);
    k_cast_acc<T, Tin><<<grid_for(nu, 256), 256, 0, s>>>(nu, f, tin.p, false);
    RS_LAUNCHED(1);
    fin = tin.p;
  }
  T *xout = x;
  if (accumulate) { tout.ensure(nu); xout = tout.p; }
  size_t smem = (size_t)R.max_ext * 2 * sizeof(T);
  static bool attr2 = false;
  if (!attr2) {
    RS_CUDA(cudaFuncSetAttribute(k_ras_apply<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    RS_CUDA(cudaFuncSetAttribute(k_ras_apply<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
    attr2 = true;
  }
  bool mixed = sizeof(T) == 4;
  {
    rs_timed tm(ls, SIM_T_RAS);
    k_ras_apply<T><<<R.nsub, 256, smem, s>>>(R.sub_ptr.p, R.ext.p, R.owned.p, R.lrp_ptr.p, R.frp.p, R.fci.p,
                                             R.fdiag.p, R.perm.p, R.lvl_rows.p, R.nlev.p, R.lvl_ptr.p,
                                             mixed ? (const T *)R.fval32.p : (const T *)R.fval.p,
                                             mixed ? (const T *)R.dinv32.p : (const T *)R.dinv.p, fin, xout);
    RS_LAUNCHED(1);
  }
  if (accumulate) {
    k_cast_acc<T, T><<<grid_for(nu, 256), 256, 0, s>>>(nu, xout, x, true);
    RS_LAUNCHED(1);
  }
}
template void ls_ras_apply<double, double>(sim_ls_s *, const double *, double *, bool);
template void ls_ras_apply<float, float>(sim_ls_s *, const float *, float *, bool);
template void ls_ras_apply<float, double>(sim_ls_s *, const double *, float *, bool);
