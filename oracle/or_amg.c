/* CPU oracle, part 3: algebraic multigrid for the pressure block, the
 * M(A_pp)^{-1} stage of Algorithm 2 (CPR-FPF).
 *
 * TEST INFRASTRUCTURE ONLY (see or_internal.h).
 *
 * The paper calls for "an AMG solver" on A_pp (Sec. "Multi-stage
 * preconditioner") without fixing its parts.  This oracle follows the
 * reading used throughout the project:
 *   strength     S_i = { j != i : -a_ij >= theta * max_{k != i} (-a_ik) }
 *   coarsening   PMIS (parallel modified independent set) with weights
 *                w_i = |S^T_i| + h(i), h a splitmix64 hash in [0, 1)
 *   interpolation direct (Stueben), positive off-diagonals lumped into the
 *                diagonal; or extended+i (De Sterck, Falgout, Nolting and
 *                Yang); R = P^T, Galerkin A_c = R (A P)
 *   cycle        one V(1,1) with l1-Jacobi smoothing, zero initial guess
 *   coarsest     dense LU with partial pivoting
 * Every sum is accumulated left to right in the order of the loops below.
 */
#include "or_internal.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

static void *xc(size_t n, size_t sz) { void *p = calloc(n ? n : 1, sz); if (!p) abort(); return p; }

void or_csr_free(or_csr *a) { free(a->rp); free(a->ci); free(a->v); memset(a, 0, sizeof(*a)); }

void or_amg_free(or_amg *h)
{
  for (int l = 0; l < h->nlev; l++) {
    or_level *L = &h->lev[l];
    or_csr_free(&L->A); or_csr_free(&L->P); or_csr_free(&L->R);
    free(L->cf); free(L->strong); free(L->dl1);
  }
  free(h->lu); free(h->piv);
  memset(h, 0, sizeof(*h));
}

/* splitmix64 (Steele, Lea and Flood 2014): one step of the generator
   seeded with x. */
uint64_t or_splitmix64(uint64_t x)
{
  uint64_t z = x + 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* PMIS tie-breaking weight in [0, 1): the top 53 bits of
   splitmix64(seed ^ (level << 40) ^ i), times 2^-53. */
double or_pmis_hash(uint64_t seed, int level, int i)
{
  uint64_t z = or_splitmix64(seed ^ ((uint64_t)level << 40) ^ (uint64_t)(uint32_t)i);
  return (double)(z >> 11) * (1.0 / 9007199254740992.0);
}

/* strength of connection on -a_ij */
static void strength(const or_csr *A, double theta, unsigned char *S)
{
  for (int i = 0; i < A->n; i++) {
    int have = 0; double mx = 0.0;
    for (int q = A->rp[i]; q < A->rp[i + 1]; q++) {
      if (A->ci[q] == i) continue;
      double v = -A->v[q];
      if (!have || v > mx) { mx = v; have = 1; }
    }
    double thr = theta * mx;
    for (int q = A->rp[i]; q < A->rp[i + 1]; q++)
      S[q] = (unsigned char)(have && mx > 0.0 && A->ci[q] != i && -A->v[q] >= thr);
  }
}

/* PMIS coarsening.  cf: 1 = C, -1 = F.  Returns the number of rounds.
   Synchronous rounds: (1) every undecided point whose weight beats that of
   each undecided neighbour in S_i u S^T_i (ties: lower index wins) becomes
   C; (2) every undecided point with a C point in S_i becomes F.  Points that
   influence no one (|S^T_i| = 0) are F from the start. */
static int pmis(const or_csr *A, const unsigned char *S, uint64_t seed, int level, signed char *cf)
{
  int n = A->n;
  /* S^T as explicit lists: j in ST_i  <=>  i in S_j */
  int *cnt = xc(n + 1, 4);
  for (int j = 0; j < n; j++)
    for (int q = A->rp[j]; q < A->rp[j + 1]; q++) if (S[q]) cnt[A->ci[q] + 1]++;
  for (int i = 0; i < n; i++) cnt[i + 1] += cnt[i];
  int *st = xc(cnt[n], 4), *fill = xc(n, 4);
  for (int j = 0; j < n; j++)
    for (int q = A->rp[j]; q < A->rp[j + 1]; q++)
      if (S[q]) { int i = A->ci[q]; st[cnt[i] + fill[i]++] = j; }
  double *w = xc(n, 8);
  for (int i = 0; i < n; i++) {
    w[i] = (double)(cnt[i + 1] - cnt[i]) + or_pmis_hash(seed, level, i);
    cf[i] = (cnt[i + 1] - cnt[i] == 0) ? -1 : 0;
  }
  signed char *newc = xc(n, 1);
  int rounds = 0;
  for (;;) {
    int und = 0;
    for (int i = 0; i < n; i++) und += (cf[i] == 0);
    if (!und) break;
    rounds++;
    for (int i = 0; i < n; i++) {
      newc[i] = 0;
      if (cf[i] != 0) continue;
      int best = 1;
      for (int q = A->rp[i]; q < A->rp[i + 1] && best; q++) {
        if (!S[q]) continue;
        int j = A->ci[q];
        if (cf[j] == 0 && (w[j] > w[i] || (w[j] == w[i] && j < i))) best = 0;
      }
      for (int q = cnt[i]; q < cnt[i + 1] && best; q++) {
        int j = st[q];
        if (cf[j] == 0 && (w[j] > w[i] || (w[j] == w[i] && j < i))) best = 0;
      }
      newc[i] = (signed char)best;
    }
    for (int i = 0; i < n; i++) if (newc[i]) cf[i] = 1;
    for (int i = 0; i < n; i++) {
      if (cf[i] != 0) continue;
      for (int q = A->rp[i]; q < A->rp[i + 1]; q++)
        if (S[q] && cf[A->ci[q]] == 1) { cf[i] = -1; break; }
    }
  }
  free(cnt); free(st); free(fill); free(w); free(newc);
  return rounds;
}

/* direct interpolation.  C point: P_i = e_{c(i)}.  F point with strong C
   neighbours C_i: w_ij = -(alpha_i a_ij) / (a_ii + sum_{k != i} a_ik^+) for
   j in C_i, alpha_i = sum_{k != i} a_ik^- / sum_{j in C_i} a_ij.
   F point without strong C neighbours: empty row. */
static void interp(const or_csr *A, const unsigned char *S, const signed char *cf, or_csr *P)
{
  int n = A->n;
  int *cidx = xc(n, 4), nc = 0;
  for (int i = 0; i < n; i++) cidx[i] = (cf[i] == 1) ? nc++ : -1;
  P->n = n; P->m = nc;
  P->rp = xc(n + 1, 4);
  for (int i = 0; i < n; i++) {
    int len = 0;
    if (cf[i] == 1) len = 1;
    else for (int q = A->rp[i]; q < A->rp[i + 1]; q++) if (S[q] && cf[A->ci[q]] == 1) len++;
    P->rp[i + 1] = P->rp[i] + len;
  }
  P->nnz = P->rp[n];
  P->ci = xc(P->nnz, 4); P->v = xc(P->nnz, 8);
  for (int i = 0; i < n; i++) {
    int o = P->rp[i];
    if (cf[i] == 1) { P->ci[o] = cidx[i]; P->v[o] = 1.0; continue; }
    if (P->rp[i + 1] == o) continue;
    double sneg = 0.0, spos = 0.0, snegc = 0.0, aii = 0.0;
    for (int q = A->rp[i]; q < A->rp[i + 1]; q++) {
      double a = A->v[q];
      if (A->ci[q] == i) { aii = a; continue; }
      if (a < 0.0) sneg += a; else spos += a;
    }
    for (int q = A->rp[i]; q < A->rp[i + 1]; q++) if (S[q] && cf[A->ci[q]] == 1) snegc += A->v[q];
    double dg = aii + spos, alpha = sneg / snegc;
    for (int q = A->rp[i]; q < A->rp[i + 1]; q++)
      if (S[q] && cf[A->ci[q]] == 1) { P->ci[o] = cidx[A->ci[q]]; P->v[o++] = -(alpha * A->v[q]) / dg; }
  }
  free(cidx);
}

/* value of row k's entry in column col (binary search; rows are sorted),
   found = 0 when the row has no such entry */
static double row_value(const or_csr *A, int k, int col, int *found)
{
  int a = A->rp[k], b = A->rp[k + 1];
  while (a < b) {
    int m = (a + b) / 2;
    if (A->ci[m] == col) { *found = 1; return A->v[m]; }
    if (A->ci[m] < col) a = m + 1; else b = m;
  }
  *found = 0;
  return 0.0;
}

/* the couplings of row k that extended+i distributes: a_kl when it differs
   in sign from the diagonal a_kk, else 0 */
static double hat(double akk, double akl)
{
  if (akk < 0.0) return akl > 0.0 ? akl : 0.0;
  return akl < 0.0 ? akl : 0.0;
}

static int in_sorted(const int *a, int m, int x)
{
  int lo = 0, hi = m;
  while (lo < hi) { int md = (lo + hi) / 2; if (a[md] == x) return 1; if (a[md] < x) lo = md + 1; else hi = md; }
  return 0;
}

/* extended+i interpolation (De Sterck, Falgout, Nolting and Yang, "Distance-
   two interpolation for parallel algebraic multigrid", 2008).  C point: P_i =
   e_{c(i)}.  F point i: the interpolatory set is C^_i = C^s_i united with the
   strong C neighbours C^s_k of every strong F neighbour k in F^s_i.  With
   a^_kl the couplings of row k of the opposite sign to a_kk and, for each k
   in F^s_i, D_k = sum over l in C^_i + {i} of a^_kl (row k's column order):
     at_ii = a_ii + sum_{n weak, n not in C^_i} a_in
                  + sum_{k in F^s_i} a_ik a^_ki / D_k      (a_ik itself when D_k = 0)
     w_ij  = -(a_ij + sum_{k in F^s_i, D_k != 0, j in row k} a_ik a^_kj / D_k) / at_ii
   for j in C^_i ascending (a_ij = 0 when j is no neighbour of i); both sums
   run in row i's column order.  An F point without strong connections has
   an empty row. */
static void interp_exti(const or_csr *A, const unsigned char *S, const signed char *cf, or_csr *P)
{
  int n = A->n;
  int *cidx = xc(n, 4), nc = 0;
  for (int i = 0; i < n; i++) cidx[i] = (cf[i] == 1) ? nc++ : -1;
  int *stamp = xc(n, 4);
  for (int i = 0; i < n; i++) stamp[i] = -1;
  int maxrow = 0;
  for (int i = 0; i < n; i++) if (A->rp[i + 1] - A->rp[i] > maxrow) maxrow = A->rp[i + 1] - A->rp[i];
  /* C^_i of every F row, sorted ascending */
  int **set = xc(n, sizeof(int *)), *len = xc(n, 4), *buf = xc(n, 4);
  for (int i = 0; i < n; i++) {
    if (cf[i] == 1) continue;
    int m = 0;
    for (int q = A->rp[i]; q < A->rp[i + 1]; q++) {
      int j = A->ci[q];
      if (!S[q] || j == i) continue;
      if (cf[j] == 1) { if (stamp[j] != i) { stamp[j] = i; buf[m++] = j; } }
      else for (int r = A->rp[j]; r < A->rp[j + 1]; r++) {
        int l = A->ci[r];
        if (S[r] && cf[l] == 1 && stamp[l] != i) { stamp[l] = i; buf[m++] = l; }
      }
    }
    for (int a = 1; a < m; a++) { int v = buf[a], b = a - 1; while (b >= 0 && buf[b] > v) { buf[b + 1] = buf[b]; b--; } buf[b + 1] = v; }
    set[i] = xc(m, 4); memcpy(set[i], buf, 4 * (size_t)m); len[i] = m;
  }
  P->n = n; P->m = nc;
  P->rp = xc(n + 1, 4);
  for (int i = 0; i < n; i++) P->rp[i + 1] = P->rp[i] + (cf[i] == 1 ? 1 : len[i]);
  P->nnz = P->rp[n];
  P->ci = xc(P->nnz, 4); P->v = xc(P->nnz, 8);
  double *D = xc(maxrow, 8);
  for (int i = 0; i < n; i++) {
    int o = P->rp[i];
    if (cf[i] == 1) { P->ci[o] = cidx[i]; P->v[o] = 1.0; continue; }
    int m = len[i];
    if (m == 0) continue;
    const int *cs = set[i];
    int q0 = A->rp[i], f;
    /* D_k of each strong F neighbour, by its position in row i */
    for (int q = q0; q < A->rp[i + 1]; q++) {
      int k = A->ci[q];
      D[q - q0] = 0.0;
      if (!S[q] || k == i || cf[k] != -1) continue;
      double akk = row_value(A, k, k, &f), d = 0.0;
      for (int r = A->rp[k]; r < A->rp[k + 1]; r++) {
        int l = A->ci[r];
        if (l == i || in_sorted(cs, m, l)) d = d + hat(akk, A->v[r]);
      }
      D[q - q0] = d;
    }
    double at = 0.0;
    at = row_value(A, i, i, &f);
    for (int q = q0; q < A->rp[i + 1]; q++) {
      int j = A->ci[q];
      if (j == i) continue;
      if (S[q]) {
        if (cf[j] == 1) continue;
        if (D[q - q0] == 0.0) at = at + A->v[q];
        else {
          double akk = row_value(A, j, j, &f), aki = row_value(A, j, i, &f);
          at = at + (A->v[q] * hat(akk, aki)) / D[q - q0];
        }
      } else if (!in_sorted(cs, m, j)) at = at + A->v[q];
    }
    for (int a = 0; a < m; a++) {
      int j = cs[a];
      double num = row_value(A, i, j, &f);
      for (int q = q0; q < A->rp[i + 1]; q++) {
        int k = A->ci[q];
        if (!S[q] || k == i || cf[k] != -1 || D[q - q0] == 0.0) continue;
        double akj = row_value(A, k, j, &f);
        if (!f) continue;
        double akk = row_value(A, k, k, &f);
        num = num + (A->v[q] * hat(akk, akj)) / D[q - q0];
      }
      P->ci[o] = cidx[j]; P->v[o++] = -num / at;
    }
  }
  for (int i = 0; i < n; i++) if (cf[i] != 1) free(set[i]);
  free(set); free(len); free(buf); free(stamp); free(cidx); free(D);
}

/* T = A^T; rows of T list their columns in ascending order */
void or_transpose(const or_csr *A, or_csr *T)
{
  T->n = A->m; T->m = A->n; T->nnz = A->nnz;
  T->rp = xc(T->n + 1, 4); T->ci = xc(A->nnz, 4); T->v = xc(A->nnz, 8);
  for (int q = 0; q < A->nnz; q++) T->rp[A->ci[q] + 1]++;
  for (int i = 0; i < T->n; i++) T->rp[i + 1] += T->rp[i];
  int *fill = xc(T->n, 4);
  for (int i = 0; i < A->n; i++)
    for (int q = A->rp[i]; q < A->rp[i + 1]; q++) {
      int j = A->ci[q], o = T->rp[j] + fill[j]++;
      T->ci[o] = i; T->v[o] = A->v[q];
    }
  free(fill);
}

/* C = A B (row by row, dense accumulator).  C_ij = sum over k in row i of
   A (ascending), of A_ik B_kj, added left to right starting from 0.  The
   pattern is the structural one: entries that cancel to 0 are kept. */
void or_spgemm(const or_csr *A, const or_csr *B, or_csr *C)
{
  int n = A->n, m = B->m;
  int *mark = xc(m, 4), *cols = xc(m, 4);
  double *acc = xc(m, 8);
  for (int j = 0; j < m; j++) mark[j] = -1;
  C->n = n; C->m = m; C->rp = xc(n + 1, 4);
  size_t cap = 16; C->ci = xc(cap, 4); C->v = xc(cap, 8);
  int nnz = 0;
  for (int i = 0; i < n; i++) {
    int len = 0;
    for (int q = A->rp[i]; q < A->rp[i + 1]; q++) {
      int k = A->ci[q]; double a = A->v[q];
      for (int r = B->rp[k]; r < B->rp[k + 1]; r++) {
        int j = B->ci[r];
        if (mark[j] != i) { mark[j] = i; acc[j] = 0.0; cols[len++] = j; }
        acc[j] = acc[j] + a * B->v[r];
      }
    }
    /* ascending column order */
    for (int a = 1; a < len; a++) { int v = cols[a], b = a - 1; while (b >= 0 && cols[b] > v) { cols[b + 1] = cols[b]; b--; } cols[b + 1] = v; }
    if ((size_t)(nnz + len) > cap) {
      while ((size_t)(nnz + len) > cap) cap *= 2;
      C->ci = realloc(C->ci, 4 * cap); C->v = realloc(C->v, 8 * cap);
      if (!C->ci || !C->v) abort();
    }
    for (int a = 0; a < len; a++) { C->ci[nnz] = cols[a]; C->v[nnz++] = acc[cols[a]]; }
    C->rp[i + 1] = nnz;
  }
  C->nnz = nnz;
  free(mark); free(cols); free(acc);
}

static void csr_copy(const or_csr *A, or_csr *B)
{
  *B = *A;
  B->rp = xc(A->n + 1, 4); memcpy(B->rp, A->rp, 4 * (size_t)(A->n + 1));
  B->ci = xc(A->nnz, 4); memcpy(B->ci, A->ci, 4 * (size_t)A->nnz);
  B->v = xc(A->nnz, 8); memcpy(B->v, A->v, 8 * (size_t)A->nnz);
}

/* l1-Jacobi diagonal d_i = a_ii + sum_{j != i} |a_ij| */
static void l1diag(const or_csr *A, double *d)
{
  for (int i = 0; i < A->n; i++) {
    double s = 0.0, aii = 0.0;
    for (int q = A->rp[i]; q < A->rp[i + 1]; q++) {
      if (A->ci[q] == i) aii = A->v[q]; else s += fabs(A->v[q]);
    }
    d[i] = aii + s;
  }
}

static void dense_lu(const or_csr *A, double **lu_out, int **piv_out)
{
  int n = A->n;
  double *a = xc((size_t)n * n, 8); int *piv = xc(n, 4);
  for (int i = 0; i < n; i++)
    for (int q = A->rp[i]; q < A->rp[i + 1]; q++) a[(size_t)i * n + A->ci[q]] = A->v[q];
  for (int k = 0; k < n; k++) {
    int p = k; double mx = fabs(a[(size_t)k * n + k]);
    for (int i = k + 1; i < n; i++) if (fabs(a[(size_t)i * n + k]) > mx) { mx = fabs(a[(size_t)i * n + k]); p = i; }
    piv[k] = p;
    if (p != k) for (int j = 0; j < n; j++) { double t = a[(size_t)k * n + j]; a[(size_t)k * n + j] = a[(size_t)p * n + j]; a[(size_t)p * n + j] = t; }
    for (int i = k + 1; i < n; i++) {
      double l = a[(size_t)i * n + k] / a[(size_t)k * n + k];
      a[(size_t)i * n + k] = l;
      for (int j = k + 1; j < n; j++) a[(size_t)i * n + j] = a[(size_t)i * n + j] - l * a[(size_t)k * n + j];
    }
  }
  *lu_out = a; *piv_out = piv;
}

static void dense_solve(int n, const double *a, const int *piv, const double *f, double *x)
{
  for (int i = 0; i < n; i++) x[i] = f[i];
  for (int k = 0; k < n; k++) if (piv[k] != k) { double t = x[k]; x[k] = x[piv[k]]; x[piv[k]] = t; }
  for (int i = 0; i < n; i++) { double s = x[i]; for (int j = 0; j < i; j++) s -= a[(size_t)i * n + j] * x[j]; x[i] = s; }
  for (int i = n - 1; i >= 0; i--) { double s = x[i]; for (int j = i + 1; j < n; j++) s -= a[(size_t)i * n + j] * x[j]; x[i] = s / a[(size_t)i * n + i]; }
}

/* Build the hierarchy from A0 (copied).  Level l is the coarsest when it
   has at most coarse_max rows or l = max_levels - 1 (dense LU), or when
   PMIS finds no coarse point (then the coarsest solve is 10 l1-Jacobi
   sweeps unless the level is small enough for the dense LU). */
int or_amg_setup(or_amg *h, const or_csr *A0, double theta, uint64_t seed, int coarse_max, int max_levels,
                 int interpolation)
{
  memset(h, 0, sizeof(*h));
  if (max_levels > 32) max_levels = 32;
  if (max_levels < 1) max_levels = 1;
  csr_copy(A0, &h->lev[0].A);
  int l = 0;
  for (;;) {
    or_level *L = &h->lev[l];
    int n = L->A.n;
    L->dl1 = xc(n, 8); l1diag(&L->A, L->dl1);
    L->cf = xc(n, 1); L->strong = xc(L->A.nnz, 1);
    if (n <= coarse_max || l == max_levels - 1) { h->coarse_dense = 1; break; }
    strength(&L->A, theta, L->strong);
    L->pmis_rounds = pmis(&L->A, L->strong, seed, l, L->cf);
    int nc = 0; for (int i = 0; i < n; i++) nc += (L->cf[i] == 1);
    if (nc == 0) { h->coarse_dense = 0; break; }
    if (interpolation == 1) interp_exti(&L->A, L->strong, L->cf, &L->P);
    else interp(&L->A, L->strong, L->cf, &L->P);
    or_transpose(&L->P, &L->R);
    or_csr AP; or_spgemm(&L->A, &L->P, &AP);
    or_spgemm(&L->R, &AP, &h->lev[l + 1].A);
    or_csr_free(&AP);
    l++;
  }
  h->nlev = l + 1;
  if (h->coarse_dense) dense_lu(&h->lev[l].A, &h->lu, &h->piv);
  return 0;
}

static void csr_mv(const or_csr *A, const double *x, double *y)
{
  #pragma omp parallel for schedule(static)
  for (int i = 0; i < A->n; i++) { double s = 0.0; for (int q = A->rp[i]; q < A->rp[i + 1]; q++) s += A->v[q] * x[A->ci[q]]; y[i] = s; }
}

/* one V(1,1) cycle from a zero initial guess: x ~ A_l^{-1} f */
void or_amg_vcycle(const or_amg *h, int l, const double *f, double *x)
{
  const or_level *L = &h->lev[l];
  int n = L->A.n;
  if (l == h->nlev - 1) {
    if (h->coarse_dense) { dense_solve(n, h->lu, h->piv, f, x); return; }
    double *t = xc(n, 8);
    for (int i = 0; i < n; i++) x[i] = 0.0;
    for (int it = 0; it < 10; it++) {
      csr_mv(&L->A, x, t);
      for (int i = 0; i < n; i++) x[i] = x[i] + (f[i] - t[i]) / L->dl1[i];
    }
    free(t);
    return;
  }
  int nc = L->P.m;
  double *r = xc(n, 8), *t = xc(n, 8), *fc = xc(nc, 8), *ec = xc(nc, 8);
  for (int i = 0; i < n; i++) x[i] = f[i] / L->dl1[i];            /* pre-smooth  */
  csr_mv(&L->A, x, t);
  for (int i = 0; i < n; i++) r[i] = f[i] - t[i];
  csr_mv(&L->R, r, fc);                                          /* restrict    */
  or_amg_vcycle(h, l + 1, fc, ec);
  csr_mv(&L->P, ec, t);                                          /* prolongate  */
  for (int i = 0; i < n; i++) x[i] += t[i];
  csr_mv(&L->A, x, t);                                           /* post-smooth */
  for (int i = 0; i < n; i++) x[i] = x[i] + (f[i] - t[i]) / L->dl1[i];
  free(r); free(t); free(fc); free(ec);
}

/* ---- standalone AMG for tests ---- */
or_amg *or_amg_new(int n, const int *rp, const int *ci, const double *v, double theta,
                   uint64_t seed, int coarse_max, int max_levels, int interpolation)
{
  or_csr A; A.n = A.m = n; A.nnz = rp[n];
  A.rp = (int *)rp; A.ci = (int *)ci; A.v = (double *)v;
  or_amg *h = xc(1, sizeof(or_amg));
  or_amg_setup(h, &A, theta, seed, coarse_max, max_levels, interpolation);
  return h;
}

/* test hook: strength and interpolation (0 direct, 1 extended+i) of a
   scalar matrix for a given C/F split; *nnz receives the size of P, and
   prp / pci / pv (when not NULL) its rows */
void or_interp_given(int n, const int *rp, const int *ci, const double *v, double theta, const signed char *cf,
                     int interpolation, int *nnz, int *prp, int *pci, double *pv)
{
  or_csr A; A.n = A.m = n; A.nnz = rp[n];
  A.rp = (int *)rp; A.ci = (int *)ci; A.v = (double *)v;
  unsigned char *S = xc(A.nnz, 1);
  strength(&A, theta, S);
  or_csr P;
  memset(&P, 0, sizeof(P));
  if (interpolation == 1) interp_exti(&A, S, cf, &P); else interp(&A, S, cf, &P);
  *nnz = P.nnz;
  if (prp) memcpy(prp, P.rp, 4 * (size_t)(n + 1));
  if (pci) memcpy(pci, P.ci, 4 * (size_t)P.nnz);
  if (pv) memcpy(pv, P.v, 8 * (size_t)P.nnz);
  or_csr_free(&P);
  free(S);
}
void or_amg_delete(or_amg *h) { if (h) { or_amg_free(h); free(h); } }
int or_amg_nlev(const or_amg *h) { return h->nlev; }
void or_amg_level_sizes(const or_amg *h, int l, int *out)
{
  const or_level *L = &h->lev[l];
  out[0] = L->A.n; out[1] = L->A.nnz; out[2] = L->P.nnz; out[3] = L->P.m; out[4] = L->pmis_rounds;
  out[5] = h->coarse_dense;
}
void or_amg_level_get(const or_amg *h, int l, int *rp, int *ci, double *v, signed char *cf,
                      unsigned char *strong, int *prp, int *pci, double *pv, double *dl1)
{
  const or_level *L = &h->lev[l];
  if (rp) memcpy(rp, L->A.rp, 4 * (size_t)(L->A.n + 1));
  if (ci) memcpy(ci, L->A.ci, 4 * (size_t)L->A.nnz);
  if (v) memcpy(v, L->A.v, 8 * (size_t)L->A.nnz);
  if (cf) memcpy(cf, L->cf, (size_t)L->A.n);
  if (strong) memcpy(strong, L->strong, (size_t)L->A.nnz);
  if (prp && L->P.rp) memcpy(prp, L->P.rp, 4 * (size_t)(L->P.n + 1));
  if (pci && L->P.ci) memcpy(pci, L->P.ci, 4 * (size_t)L->P.nnz);
  if (pv && L->P.v) memcpy(pv, L->P.v, 8 * (size_t)L->P.nnz);
  if (dl1) memcpy(dl1, L->dl1, 8 * (size_t)L->A.n);
}
void or_amg_apply(const or_amg *h, const double *f, double *x) { or_amg_vcycle(h, 0, f, x); }
double or_hash(uint64_t seed, int level, int i) { return or_pmis_hash(seed, level, i); }
