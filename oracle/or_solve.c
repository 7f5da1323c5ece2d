/* CPU oracle, part 2: processing and solution of the Newton systems.
 *
 * TEST INFRASTRUCTURE ONLY (see or_internal.h).
 *
 * Passages followed (arXiv 1701.06254):
 *   block structure of A, eq. (28); decoupling D^{-1}A x = D^{-1}b, eq. (29);
 *   ABF operator (Sec. "Matrix decoupling strategy"), Quasi-IMPES operator;
 *   local potential reordering, eqs. (30)-(32) and the worked example that
 *   follows eq. (30); restriction / prolongation eqs. (34)-(35);
 *   CPR-FPF, Algorithm 2; RAS with ILU subdomain solves; GMRES(m) (used here
 *   in its flexible, right-preconditioned form).
 * Storage: 2x2 blocks (cell-interleaved unknowns), which is the paper's
 * field-split system of eq. (20) under a fixed permutation.  Well rows are
 * padded with a dummy second unknown whose equation is 1*x = 0.
 */
#include "or_internal.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

static void *xc(size_t n, size_t sz) { void *p = calloc(n ? n : 1, sz); if (!p) abort(); return p; }

void or_lsys_init_pattern(or_lsys *ls, int nx, int ny, int nz, int nw,
                          const int *rp, const int *ci, const int *well_cell0)
{
  memset(ls, 0, sizeof(*ls));
  ls->nx = nx; ls->ny = ny; ls->nz = nz; ls->n = nx * ny * nz; ls->nw = nw;
  ls->nb = ls->n + nw;
  ls->rp = xc(ls->nb + 1, 4);
  memcpy(ls->rp, rp, 4 * (size_t)(ls->nb + 1));
  ls->nnzb = rp[ls->nb];
  ls->ci = xc(ls->nnzb, 4);
  memcpy(ls->ci, ci, 4 * (size_t)ls->nnzb);
  ls->val = xc(4 * (size_t)ls->nnzb, 8);
  ls->b = xc(2 * (size_t)ls->nb, 8);
  ls->key = xc(ls->n, 8);
  ls->dmat = xc(4 * (size_t)ls->nb, 8);
  ls->well_cell0 = xc(nw, 4);
  if (nw) memcpy(ls->well_cell0, well_cell0, 4 * (size_t)nw);
}

static void free_subs(or_lsys *ls)
{
  for (int s = 0; s < ls->nsub; s++) {
    or_sub *S = &ls->sub[s];
    free(S->own); free(S->ext); free(S->rp); free(S->ci); free(S->lu); free(S->dinv); free(S->diag); free(S->opos);
  }
  free(ls->sub); ls->sub = NULL; ls->nsub = 0;
}

void or_lsys_free(or_lsys *ls)
{
  free(ls->rp); free(ls->ci); free(ls->val); free(ls->b); free(ls->key); free(ls->dmat);
  free(ls->well_cell0);
  free_subs(ls);
  or_amg_free(&ls->amg);
  memset(ls, 0, sizeof(*ls));
}

/* y = A x over the 2x2 block system */
void or_bsr_mv(const or_lsys *ls, const double *x, double *y)
{
  #pragma omp parallel for schedule(static)
  for (int i = 0; i < ls->nb; i++) {
    double y0 = 0, y1 = 0;
    for (int q = ls->rp[i]; q < ls->rp[i + 1]; q++) {
      const double *B = &ls->val[4 * (size_t)q];
      const double *xx = &x[2 * (size_t)ls->ci[q]];
      y0 += B[0] * xx[0] + B[1] * xx[1];
      y1 += B[2] * xx[0] + B[3] * xx[1];
    }
    y[2 * i] = y0; y[2 * i + 1] = y1;
  }
}

/* ---------------- decoupling (eq. 29) ---------------- */

/* ABF: D = the 2x2 diagonal block of each cell row (Diag(A_pp), Diag(A_ps);
   Diag(A_sp), Diag(A_ss)); well rows keep D = I.  Every block of row i and
   b_i are multiplied by D_i^{-1} = [[d, -b], [-c, a]] / (ad - bc).  Each
   entry is formed with separate multiplications, additions and divisions in
   exactly the order written here. */
static void abf(or_lsys *ls)
{
  for (int i = 0; i < ls->nb; i++) {
    double *D = &ls->dmat[4 * (size_t)i];
    if (i >= ls->n) { D[0] = 1; D[1] = 0; D[2] = 0; D[3] = 1; continue; }
    int qd = -1;
    for (int q = ls->rp[i]; q < ls->rp[i + 1]; q++) if (ls->ci[q] == i) qd = q;
    const double *M = &ls->val[4 * (size_t)qd];
    double a = M[0], b = M[1], c = M[2], d = M[3];
    D[0] = a; D[1] = b; D[2] = c; D[3] = d;
    double det = a * d - b * c;
    double i00 = d / det, i01 = -b / det, i10 = -c / det, i11 = a / det;
    for (int q = ls->rp[i]; q < ls->rp[i + 1]; q++) {
      double *B = &ls->val[4 * (size_t)q];
      double b00 = B[0], b01 = B[1], b10 = B[2], b11 = B[3];
      double t0, t1;
      t0 = i00 * b00; t1 = i01 * b10; B[0] = t0 + t1;
      t0 = i00 * b01; t1 = i01 * b11; B[1] = t0 + t1;
      t0 = i10 * b00; t1 = i11 * b10; B[2] = t0 + t1;
      t0 = i10 * b01; t1 = i11 * b11; B[3] = t0 + t1;
    }
    double r0 = ls->b[2 * i], r1 = ls->b[2 * i + 1], t0, t1;
    t0 = i00 * r0; t1 = i01 * r1; ls->b[2 * i] = t0 + t1;
    t0 = i10 * r0; t1 = i11 * r1; ls->b[2 * i + 1] = t0 + t1;
  }
}

/* Quasi-IMPES: the pressure row of each cell loses Diag(A_ps) Diag(A_ss)^{-1}
   times the saturation row; saturation and well rows are unchanged. */
static void quasi_impes(or_lsys *ls)
{
  for (int i = 0; i < ls->nb; i++) {
    double *D = &ls->dmat[4 * (size_t)i];
    D[0] = 1; D[1] = 0; D[2] = 0; D[3] = 1;
    if (i >= ls->n) continue;
    int qd = -1;
    for (int q = ls->rp[i]; q < ls->rp[i + 1]; q++) if (ls->ci[q] == i) qd = q;
    double ratio = ls->val[4 * (size_t)qd + 1] / ls->val[4 * (size_t)qd + 3];
    D[1] = ratio;
    for (int q = ls->rp[i]; q < ls->rp[i + 1]; q++) {
      double *B = &ls->val[4 * (size_t)q];
      B[0] = B[0] - ratio * B[2];
      B[1] = B[1] - ratio * B[3];
    }
    ls->b[2 * i] = ls->b[2 * i] - ratio * ls->b[2 * i + 1];
  }
}

/* ---------------- local potential reordering (eqs. 30-32) ---------------- */

static const double *g_key; static const int *g_idx;
static int cmp_pot(const void *pa, const void *pb)
{
  int a = *(const int *)pa, b = *(const int *)pb;
  double ka = g_key[a], kb = g_key[b];
  if (ka > kb) return -1;                 /* descending potential */
  if (ka < kb) return 1;
  return (g_idx[a] > g_idx[b]) - (g_idx[a] < g_idx[b]);   /* tie: lower index first */
}

/* order[pos] = item whose potential is the (pos+1)-th largest; items with
   equal potential keep the order of their indices idx[].  The inverse,
   Pm(item) = pos + 1, is the mapping of eq. (30). */
void or_potential_rank(int m, const double *key, const int *idx, int *order)
{
  for (int i = 0; i < m; i++) order[i] = i;
  g_key = key; g_idx = idx;
  qsort(order, m, sizeof(int), cmp_pot);
}

/* ---------------- RAS subdomains (overlap 1) ---------------- */

/* Subdomain = column tile of tile_x x tile_y cells over all layers; a well
   belongs to the tile of its first perforated cell.  The local system is
   the rows of the owned unknowns and of every unknown within graph
   distance `overlap` of them in the matrix graph (overlap 1, or 2 as in the
   paper's Table 9), restricted to those rows and columns, with cells ordered by descending
   oil potential (eq. 30, applied per subdomain) and wells last (eq. 32). */
static void build_subs(or_lsys *ls)
{
  free_subs(ls);
  int tx = ls->o.tile_x > 0 ? ls->o.tile_x : 4, ty = ls->o.tile_y > 0 ? ls->o.tile_y : 4;
  int ntx = (ls->nx + tx - 1) / tx, nty = (ls->ny + ty - 1) / ty;
  ls->nsub = ntx * nty;
  ls->sub = xc(ls->nsub, sizeof(or_sub));
  int nb = ls->nb, n = ls->n;
  int *owner = xc(nb, 4), *cnt = xc(ls->nsub, 4);
  for (int c = 0; c < n; c++) {
    int i = c % ls->nx, j = (c / ls->nx) % ls->ny;
    owner[c] = (i / tx) + ntx * (j / ty);
  }
  for (int w = 0; w < ls->nw; w++) owner[n + w] = owner[ls->well_cell0[w]];
  for (int r = 0; r < nb; r++) cnt[owner[r]]++;
  for (int s = 0; s < ls->nsub; s++) { ls->sub[s].own = xc(cnt[s], 4); ls->sub[s].nown = 0; }
  for (int r = 0; r < nb; r++) { or_sub *S = &ls->sub[owner[r]]; S->own[S->nown++] = r; }
  int *mark = xc(nb, 4), *loc = xc(nb, 4), *list = xc(nb, 4), *ord = xc(nb, 4);
  for (int r = 0; r < nb; r++) { mark[r] = 0; loc[r] = -1; }
  for (int s = 0; s < ls->nsub; s++) {
    or_sub *S = &ls->sub[s];
    int m = 0, ov = ls->o.overlap == 2 ? 2 : 1;
    for (int a = 0; a < S->nown; a++) {
      int g = S->own[a];
      if (!mark[g]) { mark[g] = 1; list[m++] = g; }
    }
    /* rings of graph neighbours, one per level of overlap */
    for (int lev = 0, r0 = 0, r1 = m; lev < ov; lev++, r0 = r1, r1 = m)
      for (int a = r0; a < r1; a++) {
        int g = list[a];
        for (int q = ls->rp[g]; q < ls->rp[g + 1]; q++) {
          int c = ls->ci[q];
          if (!mark[c]) { mark[c] = 1; list[m++] = c; }
        }
      }
    /* split into cells and wells, each in ascending global order */
    int mc = 0, mw = 0;
    int *cells = xc(m, 4), *wl = xc(m, 4);
    for (int a = 0; a < m; a++) { if (list[a] < n) cells[mc++] = list[a]; else wl[mw++] = list[a]; mark[list[a]] = 0; }
    /* ascending global order */
    for (int a = 1; a < mc; a++) { int v = cells[a], b = a - 1; while (b >= 0 && cells[b] > v) { cells[b + 1] = cells[b]; b--; } cells[b + 1] = v; }
    for (int a = 1; a < mw; a++) { int v = wl[a], b = a - 1; while (b >= 0 && wl[b] > v) { wl[b + 1] = wl[b]; b--; } wl[b + 1] = v; }
    S->next = m;
    S->ext = xc(m, 4);
    if (ls->o.reorder) {
      double *k = xc(mc, 8);
      for (int a = 0; a < mc; a++) k[a] = ls->key[cells[a]];
      or_potential_rank(mc, k, cells, ord);
      for (int a = 0; a < mc; a++) S->ext[a] = cells[ord[a]];
      free(k);
    } else {
      for (int a = 0; a < mc; a++) S->ext[a] = cells[a];
    }
    for (int a = 0; a < mw; a++) S->ext[mc + a] = wl[a];
    free(cells); free(wl);
    /* local pattern, columns sorted by local position */
    for (int a = 0; a < m; a++) loc[S->ext[a]] = a;
    S->rp = xc(m + 1, 4);
    int nnz = 0;
    for (int a = 0; a < m; a++) {
      int g = S->ext[a];
      for (int q = ls->rp[g]; q < ls->rp[g + 1]; q++) if (loc[ls->ci[q]] >= 0) nnz++;
      S->rp[a + 1] = nnz;
    }
    S->ci = xc(nnz, 4); S->lu = xc(4 * (size_t)nnz, 8);
    S->dinv = xc(4 * (size_t)m, 8); S->diag = xc(m, 4);
    for (int a = 0; a < m; a++) {
      int g = S->ext[a], p0 = S->rp[a], k = p0;
      for (int q = ls->rp[g]; q < ls->rp[g + 1]; q++) {
        int lc = loc[ls->ci[q]];
        if (lc < 0) continue;
        /* insertion by local column */
        int b = k - 1;
        while (b >= p0 && S->ci[b] > lc) {
          S->ci[b + 1] = S->ci[b];
          memcpy(&S->lu[4 * (size_t)(b + 1)], &S->lu[4 * (size_t)b], 32);
          b--;
        }
        S->ci[b + 1] = lc;
        memcpy(&S->lu[4 * (size_t)(b + 1)], &ls->val[4 * (size_t)q], 32);
        k++;
      }
      for (int q = p0; q < k; q++) if (S->ci[q] == a) S->diag[a] = q;
    }
    S->opos = xc(S->nown, 4);
    for (int b = 0; b < S->nown; b++) S->opos[b] = loc[S->own[b]];
    for (int a = 0; a < m; a++) loc[S->ext[a]] = -1;
  }
  free(owner); free(cnt); free(mark); free(loc); free(list); free(ord);
}

static void inv2(const double *M, double *I)
{
  double det = M[0] * M[3] - M[1] * M[2];
  I[0] = M[3] / det; I[1] = -M[1] / det; I[2] = -M[2] / det; I[3] = M[0] / det;
}
static void mul2(const double *A, const double *B, double *C)
{
  double c0 = A[0] * B[0] + A[1] * B[2], c1 = A[0] * B[1] + A[1] * B[3];
  double c2 = A[2] * B[0] + A[3] * B[2], c3 = A[2] * B[1] + A[3] * B[3];
  C[0] = c0; C[1] = c1; C[2] = c2; C[3] = c3;
}

/* block ILU(0) in the local order (row-wise IKJ form): for each row i and
   each k < i in its pattern, L_ik = A_ik U_kk^{-1}, then A_ij -= L_ik U_kj
   for every j > k present in row i.  No fill is kept. */
static void bilu0(or_sub *S)
{
  for (int i = 0; i < S->next; i++) {
    for (int q = S->rp[i]; q < S->rp[i + 1]; q++) {
      int k = S->ci[q];
      if (k >= i) break;
      double L[4];
      mul2(&S->lu[4 * (size_t)q], &S->dinv[4 * (size_t)k], L);
      memcpy(&S->lu[4 * (size_t)q], L, 32);
      for (int qk = S->diag[k] + 1; qk < S->rp[k + 1]; qk++) {
        int j = S->ci[qk];
        for (int qi = q + 1; qi < S->rp[i + 1]; qi++)
          if (S->ci[qi] == j) {
            double P[4]; mul2(L, &S->lu[4 * (size_t)qk], P);
            double *A = &S->lu[4 * (size_t)qi];
            A[0] -= P[0]; A[1] -= P[1]; A[2] -= P[2]; A[3] -= P[3];
            break;
          }
      }
    }
    inv2(&S->lu[4 * (size_t)S->diag[i]], &S->dinv[4 * (size_t)i]);
  }
}

/* x = R(A)^{-1} f: each subdomain solves its local system with the ILU
   factors and writes back only the unknowns it owns (restricted). */
void or_ras_apply(const or_lsys *ls, const double *f, double *x)
{
  #pragma omp parallel for schedule(dynamic, 4)
  for (int s = 0; s < ls->nsub; s++) {
    const or_sub *S = &ls->sub[s];
    int m = S->next;
    double *y = xc(2 * (size_t)m, 8);
    for (int a = 0; a < m; a++) { y[2 * a] = f[2 * (size_t)S->ext[a]]; y[2 * a + 1] = f[2 * (size_t)S->ext[a] + 1]; }
    for (int i = 0; i < m; i++)                      /* L y = f (unit diagonal) */
      for (int q = S->rp[i]; q < S->diag[i]; q++) {
        const double *L = &S->lu[4 * (size_t)q]; const double *yy = &y[2 * (size_t)S->ci[q]];
        double t0 = L[0] * yy[0] + L[1] * yy[1], t1 = L[2] * yy[0] + L[3] * yy[1];
        y[2 * i] -= t0; y[2 * i + 1] -= t1;
      }
    for (int i = m - 1; i >= 0; i--) {                 /* U y = y */
      double r0 = y[2 * i], r1 = y[2 * i + 1];
      for (int q = S->diag[i] + 1; q < S->rp[i + 1]; q++) {
        const double *U = &S->lu[4 * (size_t)q]; const double *yy = &y[2 * (size_t)S->ci[q]];
        r0 -= U[0] * yy[0] + U[1] * yy[1]; r1 -= U[2] * yy[0] + U[3] * yy[1];
      }
      const double *D = &S->dinv[4 * (size_t)i];
      y[2 * i] = D[0] * r0 + D[1] * r1; y[2 * i + 1] = D[2] * r0 + D[3] * r1;
    }
    /* restricted write-back: owned unknowns only */
    for (int b = 0; b < S->nown; b++) {
      int g = S->own[b], a = S->opos[b];
      x[2 * (size_t)g] = y[2 * a]; x[2 * (size_t)g + 1] = y[2 * a + 1];
    }
    free(y);
  }
}

/* ---------------- setup: decouple, reorder, RAS, AMG ---------------- */

int or_lsys_setup(or_lsys *ls)
{
  if (ls->o.decoupling == OR_DEC_ABF) abf(ls);
  else if (ls->o.decoupling == OR_DEC_QI) quasi_impes(ls);
  else for (int i = 0; i < ls->nb; i++) { double *D = &ls->dmat[4 * (size_t)i]; D[0] = 1; D[1] = 0; D[2] = 0; D[3] = 1; }
  build_subs(ls);
  #pragma omp parallel for schedule(dynamic, 4)
  for (int s = 0; s < ls->nsub; s++) bilu0(&ls->sub[s]);
  /* pressure block A_pp: entry [0][0] of every cell-cell block (eq. 34 restricts to cell pressures) */
  or_csr A; A.n = A.m = ls->n;
  A.rp = xc(ls->n + 1, 4);
  int nnz = 0;
  for (int i = 0; i < ls->n; i++) {
    for (int q = ls->rp[i]; q < ls->rp[i + 1]; q++) if (ls->ci[q] < ls->n) nnz++;
    A.rp[i + 1] = nnz;
  }
  A.nnz = nnz; A.ci = xc(nnz, 4); A.v = xc(nnz, 8);
  nnz = 0;
  for (int i = 0; i < ls->n; i++)
    for (int q = ls->rp[i]; q < ls->rp[i + 1]; q++)
      if (ls->ci[q] < ls->n) { A.ci[nnz] = ls->ci[q]; A.v[nnz++] = ls->val[4 * (size_t)q]; }
  or_amg_free(&ls->amg);
  int rc = or_amg_setup(&ls->amg, &A, ls->o.amg_theta, ls->o.seed, ls->o.amg_coarse_max, ls->o.amg_max_levels,
                        ls->o.interp);
  or_csr_free(&A);
  ls->have_setup = 1;
  return rc;
}

/* ---------------- CPR-FPF, Algorithm 2 ---------------- */

void or_cpr_apply(or_lsys *ls, const double *f, double *x)
{
  int nu = 2 * ls->nb, n = ls->n;
  double *r = xc(nu, 8), *t = xc(nu, 8), *pc = xc(n, 8), *xp = xc(n, 8);
  or_ras_apply(ls, f, x);                                /* x = R(A)^{-1} f        */
  or_bsr_mv(ls, x, t);                                   /* r = f - A x            */
  for (int i = 0; i < nu; i++) r[i] = f[i] - t[i];
  for (int c = 0; c < n; c++) pc[c] = r[2 * c];          /*    Pi_r r (eq. 34)     */
  or_amg_vcycle(&ls->amg, 0, pc, xp);                    /* M(A_pp)^{-1}           */
  for (int c = 0; c < n; c++) x[2 * c] += xp[c];         /*    x += Pi_p (eq. 35)  */
  or_bsr_mv(ls, x, t);                                   /* r = f - A x            */
  for (int i = 0; i < nu; i++) r[i] = f[i] - t[i];
  or_ras_apply(ls, r, t);                                /* x += R(A)^{-1} r       */
  for (int i = 0; i < nu; i++) x[i] += t[i];
  free(r); free(t); free(pc); free(xp);
}

/* ---------------- flexible GMRES(m), right preconditioned ---------------- */

static double dot(const double *a, const double *b, int m) { double s = 0; for (int i = 0; i < m; i++) s += a[i] * b[i]; return s; }
static long S_reorth = 0;   /* second Gram-Schmidt passes taken (statistics) */
long or_reorth_count(void) { return S_reorth; }

/* Solves the (decoupled) system A y = b from y = 0 until
   ||b - A y||_2 <= tol ||b||_2 (eq. 24) or max_lin iterations.  Arnoldi
   with classical Gram-Schmidt and a conditional second pass; Givens
   rotations on the Hessenberg matrix.  Returns 0 (converged), 1 (iteration limit) or
   2 (non-finite value). */
/* BiCGSTAB (van der Vorst), right preconditioned by CPR-FPF: the paper's
   other Krylov method (Examples 3, 6 and 7; each iteration applies the
   preconditioner twice).  Solves A M^-1 u = b with x = M^-1 u from x = 0.
   One iteration:
     rho = (rh, r);  beta = (rho / rho_prev) (alpha / omega)
     p = r + beta (p - omega v);  ph = M^-1 p;  v = A ph
     alpha = rho / (rh, v);  s = r - alpha v
     (stop with x += alpha ph when ||s|| <= tol ||b||)
     sh = M^-1 s;  t = A sh;  omega = (t, s) / (t, t)
     x += alpha ph + omega sh;  r = s - omega t
   The iteration stops when the recursive residual meets tol ||b||; the true
   residual b - A x is then checked, and when it does not meet the tolerance
   (or on a breakdown: rho, (rh, v) or omega zero) the method restarts from
   the true residual with rh = r.  At most max_lin iterations. */
static int or_lsys_solve_bicgstab(or_lsys *ls, double tol, double *x, int *its_out, double *relres)
{
  int nu = 2 * ls->nb, maxit = ls->o.max_lin, its = 0, rc = 1;
  double *r = xc(nu, 8), *rh = xc(nu, 8), *p = xc(nu, 8), *v = xc(nu, 8), *s = xc(nu, 8);
  double *t = xc(nu, 8), *ph = xc(nu, 8), *sh = xc(nu, 8);
  for (int i = 0; i < nu; i++) x[i] = 0.0;
  double bn = sqrt(dot(ls->b, ls->b, nu)), rn = bn;
  if (bn == 0.0) { *its_out = 0; *relres = 0.0; rc = 0; goto out; }
  if (bn != bn) { *its_out = 0; *relres = bn; rc = 2; goto out; }
  memcpy(r, ls->b, 8 * (size_t)nu);
  for (;;) {                                   /* (re)start from the residual in r */
    memcpy(rh, r, 8 * (size_t)nu);
    memset(p, 0, 8 * (size_t)nu); memset(v, 0, 8 * (size_t)nu);
    double rho_prev = 1.0, alpha = 1.0, omega = 1.0;
    int broke = 0, done = 0;
    while (its < maxit) {
      double rho = dot(rh, r, nu);
      if (rho == 0.0) { broke = 1; break; }
      double beta = (rho / rho_prev) * (alpha / omega);
      for (int i = 0; i < nu; i++) p[i] = r[i] + beta * (p[i] - omega * v[i]);
      or_cpr_apply(ls, p, ph);
      or_bsr_mv(ls, ph, v);
      double rv = dot(rh, v, nu);
      if (rv == 0.0) { broke = 1; break; }
      alpha = rho / rv;
      for (int i = 0; i < nu; i++) s[i] = r[i] - alpha * v[i];
      its++;
      double sn = sqrt(dot(s, s, nu));
      if (sn != sn) { rc = 2; rn = sn; goto out; }
      if (sn <= tol * bn) {
        for (int i = 0; i < nu; i++) x[i] += alpha * ph[i];
        done = 1; break;
      }
      or_cpr_apply(ls, s, sh);
      or_bsr_mv(ls, sh, t);
      double tt = dot(t, t, nu), ts = dot(t, s, nu);
      omega = tt > 0.0 ? ts / tt : 0.0;
      for (int i = 0; i < nu; i++) x[i] += alpha * ph[i] + omega * sh[i];
      for (int i = 0; i < nu; i++) r[i] = s[i] - omega * t[i];
      rn = sqrt(dot(r, r, nu));
      if (rn != rn) { rc = 2; goto out; }
      if (rn <= tol * bn) { done = 1; break; }
      if (omega == 0.0) { broke = 1; break; }
      rho_prev = rho;
    }
    /* true residual */
    or_bsr_mv(ls, x, t);
    for (int i = 0; i < nu; i++) r[i] = ls->b[i] - t[i];
    rn = sqrt(dot(r, r, nu));
    if (rn != rn) { rc = 2; goto out; }
    if (rn <= tol * bn) { rc = 0; break; }
    if (its >= maxit) { rc = 1; break; }
    if (!done && !broke) { rc = 1; break; }
  }
out:
  if (bn > 0.0 && rc != 2) *relres = rn / bn;
  else if (rc == 2) *relres = NAN;
  *its_out = its;
  free(r); free(rh); free(p); free(v); free(s); free(t); free(ph); free(sh);
  return rc;
}

int or_lsys_solve(or_lsys *ls, double tol, double *y, int *its_out, double *relres)
{
  if (ls->o.krylov == OR_BICGSTAB) return or_lsys_solve_bicgstab(ls, tol, y, its_out, relres);
  int nu = 2 * ls->nb, m = ls->o.restart > 0 ? ls->o.restart : 50, maxit = ls->o.max_lin;
  double *V = xc((size_t)(m + 1) * nu, 8), *Z = xc((size_t)m * nu, 8);
  double *H = xc((size_t)(m + 1) * m, 8), *cs = xc(m, 8), *sn = xc(m, 8), *g = xc(m + 1, 8);
  double *h = xc(m + 1, 8), *h2 = xc(m + 1, 8), *w = xc(nu, 8), *r = xc(nu, 8), *yy = xc(m, 8);
  for (int i = 0; i < nu; i++) y[i] = 0.0;
  double bn = sqrt(dot(ls->b, ls->b, nu));
  int its = 0, rc = 1;
  if (bn == 0.0) { *its_out = 0; *relres = 0.0; rc = 0; goto out; }
  memcpy(r, ls->b, 8 * (size_t)nu);
  double beta = bn;
  for (;;) {
    for (int i = 0; i < nu; i++) V[i] = r[i] / beta;
    memset(g, 0, 8 * (size_t)(m + 1)); g[0] = beta;
    int j, jend = 0, stop = 0;
    for (j = 0; j < m; j++) {
      double *vj = &V[(size_t)j * nu], *zj = &Z[(size_t)j * nu];
      or_cpr_apply(ls, vj, zj);
      or_bsr_mv(ls, zj, w);
      /* classical Gram-Schmidt; a second pass only when the first one
         removed nearly all of w (||w_1|| < 1e-2 ||w||, the Daniel, Gragg,
         Kaufman and Stewart test with a small threshold: a pass that keeps
         at least 1% of w loses at most ~100 eps of orthogonality) */
      double wn2 = dot(w, w, nu);
      for (int k = 0; k <= j; k++) h[k] = dot(&V[(size_t)k * nu], w, nu);
      for (int i = 0; i < nu; i++) { double s = 0; for (int k = 0; k <= j; k++) s += h[k] * V[(size_t)k * nu + i]; w[i] -= s; }
      double hn2 = dot(w, w, nu);
      if (hn2 < 1e-4 * wn2) {
        for (int k = 0; k <= j; k++) h2[k] = dot(&V[(size_t)k * nu], w, nu);
        for (int i = 0; i < nu; i++) { double s = 0; for (int k = 0; k <= j; k++) s += h2[k] * V[(size_t)k * nu + i]; w[i] -= s; }
        for (int k = 0; k <= j; k++) h[k] += h2[k];
        hn2 = dot(w, w, nu);
        S_reorth++;
      }
      double hn = sqrt(hn2);
      if (hn != hn) { rc = 2; goto out; }
      if (hn > 0.0) for (int i = 0; i < nu; i++) V[(size_t)(j + 1) * nu + i] = w[i] / hn;
      /* apply the previous rotations to column j, then a new one */
      for (int k = 0; k < j; k++) {
        double t = cs[k] * h[k] + sn[k] * h[k + 1];
        h[k + 1] = -sn[k] * h[k] + cs[k] * h[k + 1];
        h[k] = t;
      }
      double rr = sqrt(h[j] * h[j] + hn * hn);
      cs[j] = h[j] / rr; sn[j] = hn / rr;
      h[j] = rr;
      g[j + 1] = -sn[j] * g[j];
      g[j] = cs[j] * g[j];
      for (int k = 0; k <= j; k++) H[(size_t)k * m + j] = h[k];
      its++;
      jend = j + 1;
      if (fabs(g[j + 1]) <= tol * bn || its >= maxit || hn == 0.0) { stop = 1; break; }
    }
    /* y_k from the triangular system, x += Z y */
    for (int k = jend - 1; k >= 0; k--) {
      double s = g[k];
      for (int l = k + 1; l < jend; l++) s -= H[(size_t)k * m + l] * yy[l];
      yy[k] = s / H[(size_t)k * m + k];
    }
    for (int i = 0; i < nu; i++) { double s = 0; for (int k = 0; k < jend; k++) s += yy[k] * Z[(size_t)k * nu + i]; y[i] += s; }
    or_bsr_mv(ls, y, w);
    for (int i = 0; i < nu; i++) r[i] = ls->b[i] - w[i];
    beta = sqrt(dot(r, r, nu));
    if (beta != beta) { rc = 2; break; }
    if (beta <= tol * bn) { rc = 0; break; }
    if (its >= maxit) { rc = 1; break; }
    (void)stop;
  }
  *its_out = its; *relres = beta / bn;
out:
  if (bn == 0.0) { *its_out = 0; *relres = 0.0; }
  else if (rc == 2) { *its_out = its; *relres = NAN; }
  free(V); free(Z); free(H); free(cs); free(sn); free(g); free(h); free(h2); free(w); free(r); free(yy);
  return rc;
}

/* ---------------- accessors for the Python binding ---------------- */
or_lsys *or_ls_create(int nx, int ny, int nz, int nw, const int *rp, const int *ci,
                      const int *well_cell0, const or_opts *o)
{
  or_lsys *ls = xc(1, sizeof(or_lsys));
  or_lsys_init_pattern(ls, nx, ny, nz, nw, rp, ci, well_cell0);
  ls->o = *o;
  return ls;
}
void or_ls_destroy(or_lsys *ls) { if (ls) { or_lsys_free(ls); free(ls); } }
void or_ls_set(or_lsys *ls, const double *val, const double *b, const double *key)
{
  memcpy(ls->val, val, 32 * (size_t)ls->nnzb);
  memcpy(ls->b, b, 16 * (size_t)ls->nb);
  memcpy(ls->key, key, 8 * (size_t)ls->n);
  ls->have_setup = 0;
}
void or_ls_set_opts(or_lsys *ls, const or_opts *o) { ls->o = *o; }
int or_ls_setup(or_lsys *ls) { return or_lsys_setup(ls); }
int or_ls_solve(or_lsys *ls, double tol, double *y, int *its, double *relres) { return or_lsys_solve(ls, tol, y, its, relres); }
void or_ls_get(const or_lsys *ls, int *rp, int *ci, double *val, double *b, double *key)
{
  if (rp) memcpy(rp, ls->rp, 4 * (size_t)(ls->nb + 1));
  if (ci) memcpy(ci, ls->ci, 4 * (size_t)ls->nnzb);
  if (val) memcpy(val, ls->val, 32 * (size_t)ls->nnzb);
  if (b) memcpy(b, ls->b, 16 * (size_t)ls->nb);
  if (key) memcpy(key, ls->key, 8 * (size_t)ls->n);
}
void or_ls_sizes(const or_lsys *ls, int *out) { out[0] = ls->n; out[1] = ls->nw; out[2] = ls->nb; out[3] = ls->nnzb; out[4] = ls->nsub; }
void or_ls_mv(const or_lsys *ls, const double *x, double *y) { or_bsr_mv(ls, x, y); }
void or_ls_cpr(or_lsys *ls, const double *f, double *x) { or_cpr_apply(ls, f, x); }
void or_ls_ras(const or_lsys *ls, const double *f, double *x) { or_ras_apply(ls, f, x); }
or_amg *or_ls_amg(or_lsys *ls) { return &ls->amg; }
void or_ls_sub_sizes(const or_lsys *ls, int s, int *out) { out[0] = ls->sub[s].nown; out[1] = ls->sub[s].next; out[2] = ls->sub[s].rp[ls->sub[s].next]; }
void or_ls_sub_get(const or_lsys *ls, int s, int *own, int *ext, int *rp, int *ci, double *lu, double *dinv)
{
  const or_sub *S = &ls->sub[s];
  if (own) memcpy(own, S->own, 4 * (size_t)S->nown);
  if (ext) memcpy(ext, S->ext, 4 * (size_t)S->next);
  if (rp) memcpy(rp, S->rp, 4 * (size_t)(S->next + 1));
  if (ci) memcpy(ci, S->ci, 4 * (size_t)S->rp[S->next]);
  if (lu) memcpy(lu, S->lu, 32 * (size_t)S->rp[S->next]);
  if (dinv) memcpy(dinv, S->dinv, 32 * (size_t)S->next);
}
