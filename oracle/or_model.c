/* CPU oracle, part 1: the two-phase oil-water model, its fully implicit
 * discretisation, Newton's method and the time loop.
 *
 * TEST INFRASTRUCTURE ONLY (see or_internal.h).
 *
 * Passages followed (arXiv 1701.06254):
 *   Sec. "Two-phase oil-water flow model": mass balance eq. (3), no-flow
 *     boundary, porosity eq. (4), phase potential eq. (5), density eq. (6),
 *     viscosity eq. (7), s_o + s_w = 1 eq. (8), Peaceman well rate eq. (10),
 *     BHP constraint eq. (11), water-rate constraint eq. (12);
 *   Sec. "Numerical methods": unknowns (p, s_w, p_b), backward Euler eq. (15),
 *     transmissibility eq. (16), discrete residual eq. (17), upstreaming
 *     eq. (18), F(x) = 0 eqs. (19)-(23);
 *   Sec. "Nonlinear methods": Algorithm 1 (inexact Newton), eqs. (24)-(27).
 * Where the paper is silent (units, gravity sign, relative permeability
 * form, well index, tie rules, scaling, time-step cuts) the reading taken is
 * stated at each use below.
 */
#include "or_internal.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

static void *xc(size_t n, size_t sz) { void *p = calloc(n ? n : 1, sz); if (!p) abort(); return p; }

/* ------------------------------------------------------------------ */
/* Cell properties: eqs. (4), (6), (7), (8) and the Corey relative     */
/* permeabilities (the paper leaves K_r as "user input").              */
/* ------------------------------------------------------------------ */
typedef struct {
  double phi, dphi;                 /* porosity and d/dp              */
  double pc, dpc;                   /* capillary pressure and d/ds_w  */
  double rho[2], drho[2], drhos[2]; /* density (water, oil), d/dp, d/ds_w */
  double mu[2], dmu[2], dmus[2];    /* viscosity, d/dp, d/ds_w        */
  double kr[2], dkr[2];             /* rel. perm. and d/ds_w          */
  double m[2], dmp[2], dms[2];      /* mobility rho*kr/mu, d/dp, d/ds */
  double pot[2], dpot[2], dpots[2]; /* potential eq. (5), d/dp, d/ds  */
} props_t;

/* Capillary pressure p_c(s_w) of eq. (9), "user input": the table's points
   joined by straight lines, constant beyond its first and last points.  The
   segment is the last k with sw[k] <= s; its slope is the derivative (0
   outside the table). */
static void capillary(const or_fluid *f, double s, double *pc, double *dpc)
{
  int n = f->pc_n;
  if (n <= 0) { *pc = 0.0; *dpc = 0.0; return; }
  if (n == 1 || s < f->pc_sw[0]) { *pc = f->pc_val[0]; *dpc = 0.0; return; }
  if (s >= f->pc_sw[n - 1]) { *pc = f->pc_val[n - 1]; *dpc = 0.0; return; }
  int k = 0;
  while (s >= f->pc_sw[k + 1]) k++;
  double slope = (f->pc_val[k + 1] - f->pc_val[k]) / (f->pc_sw[k + 1] - f->pc_sw[k]);
  *pc = f->pc_val[k] + (s - f->pc_sw[k]) * slope;
  *dpc = slope;
}

static void cell_props(const or_sim *S, int c, double p, double sw, props_t *P)
{
  const or_fluid *f = &S->f;
  double dp = p - f->p_ref;
  P->phi = S->phi[c] * (1.0 + f->c_r * dp);                     /* eq. (4) */
  P->dphi = S->phi[c] * f->c_r;
  capillary(f, sw, &P->pc, &P->dpc);
  double span = 1.0 - f->swc - f->sor;
  double sh = (sw - f->swc) / span, dsh = 1.0 / span;
  if (sh < 0.0) { sh = 0.0; dsh = 0.0; } else if (sh > 1.0) { sh = 1.0; dsh = 0.0; }
  P->kr[0] = f->krw_max * pow(sh, f->nw);
  P->dkr[0] = f->krw_max * f->nw * pow(sh, f->nw - 1.0) * dsh;
  P->kr[1] = f->kro_max * pow(1.0 - sh, f->no);
  P->dkr[1] = -f->kro_max * f->no * pow(1.0 - sh, f->no - 1.0) * dsh;
  double gz5 = f->g * S->z[c] * OR_PA2BAR;                      /* rho g z in bar per kg/m3 */
  for (int a = 0; a < 2; a++) {
    /* phase pressure, eq. (9): p_w = p_o - p_c(s_w), p_o = p */
    double pa = a == 0 ? p - P->pc : p;
    double dpa_s = a == 0 ? -P->dpc : 0.0;
    P->rho[a] = f->rho_ref[a] * (1.0 + f->c_f[a] * (pa - f->p_ref));   /* eq. (6) */
    P->drho[a] = f->rho_ref[a] * f->c_f[a];
    P->drhos[a] = P->drho[a] * dpa_s;
    P->mu[a] = f->mu_ref[a] + f->c_mu[a] * (pa - f->p_ref);           /* eq. (7) */
    P->dmu[a] = f->c_mu[a];
    P->dmus[a] = f->c_mu[a] * dpa_s;
    P->m[a] = P->rho[a] * P->kr[a] / P->mu[a];
    P->dmp[a] = P->drho[a] * P->kr[a] / P->mu[a] - P->rho[a] * P->kr[a] * P->dmu[a] / (P->mu[a] * P->mu[a]);
    P->dms[a] = P->rho[a] * P->dkr[a] / P->mu[a] + P->drhos[a] * P->kr[a] / P->mu[a]
                - P->rho[a] * P->kr[a] * P->dmus[a] / (P->mu[a] * P->mu[a]);
    /* eq. (5) with z = depth (positive downwards): the potential falls
       with depth, so a hydrostatic column has a constant potential. */
    P->pot[a] = pa - P->rho[a] * gz5;
    P->dpot[a] = 1.0 - P->drho[a] * gz5;
    P->dpots[a] = dpa_s - P->drhos[a] * gz5;
  }
}

/* block position of column `col` in block row `row` (linear search) */
static int bpos(const or_lsys *ls, int row, int col)
{
  for (int q = ls->rp[row]; q < ls->rp[row + 1]; q++) if (ls->ci[q] == col) return q;
  abort();
}

static int cmp_int(const void *a, const void *b) { int x = *(const int *)a, y = *(const int *)b; return (x > y) - (x < y); }

/* ------------------------------------------------------------------ */
/* Creation: geometry, transmissibilities, well indices, pattern.      */
/* ------------------------------------------------------------------ */
or_sim *or_sim_create(const or_grid *g, const double *kx, const double *ky, const double *kz,
                      const double *phi, const or_fluid *f, const or_well *wells, int nw,
                      const or_opts *o)
{
  or_sim *S = xc(1, sizeof(or_sim));
  S->g = *g; S->f = *f; S->o = *o;
  if (f->pc_n > 0) {                       /* own copy of the capillary pressure table */
    S->pc_sw = xc(f->pc_n, 8); S->pc_val = xc(f->pc_n, 8);
    memcpy(S->pc_sw, f->pc_sw, 8 * (size_t)f->pc_n); memcpy(S->pc_val, f->pc_val, 8 * (size_t)f->pc_n);
    S->f.pc_sw = S->pc_sw; S->f.pc_val = S->pc_val;
  }
  int nx = g->nx, ny = g->ny, nz = g->nz, n = nx * ny * nz;
  S->n = n;
  S->kx = xc(n, 8); S->ky = xc(n, 8); S->kz = xc(n, 8); S->phi = xc(n, 8);
  memcpy(S->kx, kx, 8 * (size_t)n); memcpy(S->ky, ky, 8 * (size_t)n);
  memcpy(S->kz, kz, 8 * (size_t)n); memcpy(S->phi, phi, 8 * (size_t)n);
  S->z = xc(n, 8); S->vol = xc(n, 8);
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        int c = i + nx * (j + ny * k);
        S->z[c] = g->top + ((double)k + 0.5) * g->dz;            /* cell-centre depth */
        S->vol[c] = g->dx * g->dy * g->dz;
      }
  /* interior faces (c < d) with the two-point (harmonic) geometric
     transmissibility; the mobility factor of eq. (16) is upstreamed
     separately per eq. (18). */
  S->nf = (nx - 1) * ny * nz + nx * (ny - 1) * nz + nx * ny * (nz - 1);
  S->fc = xc(S->nf, 4); S->fd = xc(S->nf, 4); S->ft = xc(S->nf, 8);
  int nf = 0;
  for (int k = 0; k < nz; k++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) {
        int c = i + nx * (j + ny * k);
        if (i + 1 < nx) {
          int d = c + 1;
          S->fc[nf] = c; S->fd[nf] = d;
          S->ft[nf++] = OR_CDARCY * (g->dy * g->dz) / (g->dx / (2.0 * kx[c]) + g->dx / (2.0 * kx[d]));
        }
        if (j + 1 < ny) {
          int d = c + nx;
          S->fc[nf] = c; S->fd[nf] = d;
          S->ft[nf++] = OR_CDARCY * (g->dx * g->dz) / (g->dy / (2.0 * ky[c]) + g->dy / (2.0 * ky[d]));
        }
        if (k + 1 < nz) {
          int d = c + nx * ny;
          S->fc[nf] = c; S->fd[nf] = d;
          S->ft[nf++] = OR_CDARCY * (g->dx * g->dy) / (g->dz / (2.0 * kz[c]) + g->dz / (2.0 * kz[d]));
        }
      }
  /* wells and perforations; Peaceman's well index when none is given */
  S->nw = nw;
  S->wkind = xc(nw, 4); S->wctrl = xc(nw, 4); S->wtarget = xc(nw, 8); S->wzref = xc(nw, 8);
  S->wctrl0 = xc(nw, 4); S->wtarget0 = xc(nw, 8); S->wlimit = xc(nw, 8); S->wswitched = xc(nw, 4);
  S->pptr = xc(nw + 1, 4);
  for (int w = 0; w < nw; w++) S->pptr[w + 1] = S->pptr[w] + wells[w].n_perf;
  S->pcell = xc(S->pptr[nw], 4); S->pwi = xc(S->pptr[nw], 8);
  for (int w = 0; w < nw; w++) {
    S->wkind[w] = wells[w].kind; S->wctrl[w] = wells[w].control;
    S->wtarget[w] = wells[w].target; S->wzref[w] = wells[w].z_ref;
    S->wctrl0[w] = wells[w].control; S->wtarget0[w] = wells[w].target; S->wlimit[w] = wells[w].bhp_limit;
    for (int q = 0; q < wells[w].n_perf; q++) {
      int c = wells[w].perf_cell[q];
      S->pcell[S->pptr[w] + q] = c;
      double wi;
      if (wells[w].wi) wi = wells[w].wi[q];
      else {
        double a = kx[c], b = ky[c];
        double ro = 0.28 * sqrt(sqrt(b / a) * g->dx * g->dx + sqrt(a / b) * g->dy * g->dy)
                    / (pow(b / a, 0.25) + pow(a / b, 0.25));
        wi = 2.0 * M_PI * OR_CDARCY * sqrt(a * b) * g->dz / (log(ro / wells[w].r_w) + wells[w].skin);
      }
      S->pwi[S->pptr[w] + q] = wi;
    }
  }
  /* block pattern: cell rows (stencil neighbours + perforating wells),
     then one row per well (perforated cells + itself); sorted columns */
  int nb = n + nw;
  int *rp = xc(nb + 1, 4);
  int cap = 7 * n + 2 * S->pptr[nw] + nw;
  int *ci = xc(cap, 4);
  int *tmp = xc(7 + nw + 1 + S->pptr[nw], 4);
  int nnz = 0;
  for (int c = 0; c < n; c++) {
    int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny), m = 0;
    if (k > 0) tmp[m++] = c - nx * ny;
    if (j > 0) tmp[m++] = c - nx;
    if (i > 0) tmp[m++] = c - 1;
    tmp[m++] = c;
    if (i + 1 < nx) tmp[m++] = c + 1;
    if (j + 1 < ny) tmp[m++] = c + nx;
    if (k + 1 < nz) tmp[m++] = c + nx * ny;
    for (int w = 0; w < nw; w++)
      for (int q = S->pptr[w]; q < S->pptr[w + 1]; q++)
        if (S->pcell[q] == c) { tmp[m++] = n + w; break; }
    qsort(tmp, m, 4, cmp_int);
    for (int q = 0; q < m; q++) ci[nnz++] = tmp[q];
    rp[c + 1] = nnz;
  }
  for (int w = 0; w < nw; w++) {
    int m = 0;
    for (int q = S->pptr[w]; q < S->pptr[w + 1]; q++) tmp[m++] = S->pcell[q];
    tmp[m++] = n + w;
    qsort(tmp, m, 4, cmp_int);
    for (int q = 0; q < m; q++) ci[nnz++] = tmp[q];
    rp[n + w + 1] = nnz;
  }
  free(tmp);
  int *wc0 = xc(nw, 4);
  for (int w = 0; w < nw; w++) wc0[w] = S->pcell[S->pptr[w]];
  or_lsys_init_pattern(&S->ls, nx, ny, nz, nw, rp, ci, wc0);
  S->ls.o = *o;
  free(rp); free(ci); free(wc0);
  S->p = xc(n, 8); S->s = xc(n, 8); S->pb = xc(nw ? nw : 1, 8);
  S->acc0 = xc(2 * (size_t)n, 8);
  S->y = xc(2 * (size_t)nb, 8);
  S->dt = o->dt;
  return S;
}

void or_sim_destroy(or_sim *S)
{
  if (!S) return;
  free(S->kx); free(S->ky); free(S->kz); free(S->phi); free(S->z); free(S->vol);
  free(S->fc); free(S->fd); free(S->ft);
  free(S->wkind); free(S->wctrl); free(S->wtarget); free(S->wzref);
  free(S->wctrl0); free(S->wtarget0); free(S->wlimit); free(S->wswitched); free(S->pc_sw); free(S->pc_val);
  free(S->pptr); free(S->pcell); free(S->pwi);
  or_lsys_free(&S->ls);
  free(S->p); free(S->s); free(S->pb); free(S->acc0); free(S->y);
  free(S);
}

/* Wellbore pressure from which a rate-controlled (or shut) well starts:
   10 bar above the oil pressure of its first perforated cell for an
   injector, 10 bar below for a producer, so that it flows from the first
   Newton iteration. */
static double rate_start_pb(const or_sim *S, int w)
{
  double p0 = S->p[S->pcell[S->pptr[w]]];
  return S->wkind[w] == OR_PROD ? p0 - 10.0 : p0 + 10.0;
}

/* Initial equilibrium: every cell gets the oil potential of the datum
   (eq. 5 with the cell's own density, eq. 6, solved exactly because rho is
   linear in p); s_w = sw0.  BHP wells start at their target, rate wells
   10 bar above the oil pressure of their first perforated cell. */
void or_sim_init_hydrostatic(or_sim *S, double p_datum, double sw0)
{
  const or_fluid *f = &S->f;
  double G0 = f->g * S->g.top * OR_PA2BAR;
  double rho0 = f->rho_ref[1] * (1.0 + f->c_f[1] * (p_datum - f->p_ref));
  double pot = p_datum - rho0 * G0;
  for (int c = 0; c < S->n; c++) {
    double G = f->g * S->z[c] * OR_PA2BAR;
    /* p - rho_r (1 + c (p - p_ref)) G = pot  ->  linear in p */
    double a = 1.0 - f->rho_ref[1] * f->c_f[1] * G;
    double r = pot + f->rho_ref[1] * (1.0 - f->c_f[1] * f->p_ref) * G;
    S->p[c] = r / a;
    S->s[c] = sw0;
  }
  for (int w = 0; w < S->nw; w++) {
    S->wctrl[w] = S->wctrl0[w]; S->wtarget[w] = S->wtarget0[w]; S->wswitched[w] = 0;
    S->pb[w] = (S->wctrl[w] == OR_BHP) ? S->wtarget[w] : rate_start_pb(S, w);
  }
  S->t = 0.0;
}

void or_sim_set_state(or_sim *S, const double *p, const double *s, const double *pb, double t)
{
  memcpy(S->p, p, 8 * (size_t)S->n); memcpy(S->s, s, 8 * (size_t)S->n);
  if (S->nw) memcpy(S->pb, pb, 8 * (size_t)S->nw);
  S->t = t;
}

void or_sim_get_state(const or_sim *S, double *p, double *s, double *pb, double *t)
{
  memcpy(p, S->p, 8 * (size_t)S->n); memcpy(s, S->s, 8 * (size_t)S->n);
  if (S->nw) memcpy(pb, S->pb, 8 * (size_t)S->nw);
  if (t) *t = S->t;
}

/* accumulation (phi rho_a s_a) of the current state, stored as the old
   time level for eq. (15) */
void or_sim_store_old(or_sim *S)
{
  for (int c = 0; c < S->n; c++) {
    props_t P; cell_props(S, c, S->p[c], S->s[c], &P);
    S->acc0[2 * c + 0] = P.phi * P.rho[1] * (1.0 - S->s[c]);   /* oil   */
    S->acc0[2 * c + 1] = P.phi * P.rho[0] * S->s[c];           /* water */
  }
}

/* Mass rates of one perforation (eq. 10) for both phases (0 = water,
   1 = oil; + = into the cell) and their derivatives with respect to the
   cell's p and s_w and to p_b.  The drawdown of phase a is
   dd = p_b - p_a + rho_a g (z - z_ref) (z = depth), p_a the phase pressure
   of eq. (9).  Producer: each phase with its own mobility, outflow only
   (q = 0 when dd > 0).  Injector, dd >= 0: water only, with the total cell
   mobility (kr_w/mu_w + kr_o/mu_o), so water can enter a cell at connate
   saturation.  Injector, dd < 0 (crossflow into the wellbore): upstream
   from the cell as for the faces (eq. 18), each phase with its own
   mobility.  A shut well has no flow. */
static void perf_flow(const or_sim *S, int w, int c, double wi, const props_t *P,
                      double q[2], double dqp[2], double dqs[2], double dqb[2])
{
  double dz5 = S->f.g * (S->z[c] - S->wzref[w]) * OR_PA2BAR;
  for (int a = 0; a < 2; a++) {
    q[a] = dqp[a] = dqs[a] = dqb[a] = 0.0;
    if (S->wctrl[w] == OR_SHUT) continue;
    double pa = a == 0 ? S->p[c] - P->pc : S->p[c];
    double dd = (S->pb[w] - pa) + P->rho[a] * dz5;
    double dd_dp = -1.0 + P->drho[a] * dz5;
    double dd_ds = (a == 0 ? P->dpc : 0.0) + P->drhos[a] * dz5;
    if (S->wkind[w] == OR_PROD) {
      if (dd <= 0.0) {            /* at dd = 0: q = 0 with the flowing-side derivative */
        q[a] = wi * P->m[a] * dd;
        dqp[a] = wi * (P->dmp[a] * dd + P->m[a] * dd_dp);
        dqs[a] = wi * (P->dms[a] * dd + P->m[a] * dd_ds);
        dqb[a] = wi * P->m[a];
      }
    } else if (dd < 0.0) {        /* injector crossflow: as a producer perforation */
      q[a] = wi * P->m[a] * dd;
      dqp[a] = wi * (P->dmp[a] * dd + P->m[a] * dd_dp);
      dqs[a] = wi * (P->dms[a] * dd + P->m[a] * dd_ds);
      dqb[a] = wi * P->m[a];
    } else if (a == 0) {          /* at dd = 0: q = 0 with the injecting-side derivative */
      double lt = P->kr[0] / P->mu[0] + P->kr[1] / P->mu[1];
      double lt_p = -P->kr[0] * P->dmu[0] / (P->mu[0] * P->mu[0])
                    - P->kr[1] * P->dmu[1] / (P->mu[1] * P->mu[1]);
      double lt_s = P->dkr[0] / P->mu[0] - P->kr[0] * P->dmus[0] / (P->mu[0] * P->mu[0])
                    + P->dkr[1] / P->mu[1] - P->kr[1] * P->dmus[1] / (P->mu[1] * P->mu[1]);
      q[a] = wi * P->rho[0] * lt * dd;
      dqp[a] = wi * (P->drho[0] * lt * dd + P->rho[0] * lt_p * dd + P->rho[0] * lt * dd_dp);
      dqs[a] = wi * (P->drhos[0] * lt * dd + P->rho[0] * lt_s * dd + P->rho[0] * lt * dd_ds);
      dqb[a] = wi * P->rho[0] * lt;
    }
  }
}

/* Weights of the phase mass rates in a rate-controlled well's equation,
   scaled by the target: eq. (12) water rate, eq. (13) oil rate, eq. (14)
   liquid rate, each in surface volumes (mass / rho_ref) against the target
   in sm3/day; production counts positive for a producer.  The equation is
   sum_m (cw q_w,m + co q_o,m) - 1 = 0. */
static void rate_weights(const or_sim *S, int w, double *cw, double *co)
{
  double sgn = S->wkind[w] == OR_PROD ? -1.0 : 1.0, T = S->wtarget[w];
  *cw = *co = 0.0;
  if (S->wctrl[w] == OR_WRATE || S->wctrl[w] == OR_LRATE) *cw = sgn / (S->f.rho_ref[0] * T);
  if (S->wctrl[w] == OR_ORATE || S->wctrl[w] == OR_LRATE) *co = sgn / (S->f.rho_ref[1] * T);
}

/* ------------------------------------------------------------------ */
/* Residual and Jacobian (eq. 17 with eq. 18 upstreaming and eq. 10    */
/* wells).  Block row = (oil eq, water eq) of a cell; block column =   */
/* (d/dp, d/ds_w).  Well rows are padded to 2x2: (well eq, dummy s).   */
/* b = -R.                                                             */
/* ------------------------------------------------------------------ */
void or_sim_assemble(or_sim *S)
{
  or_lsys *ls = &S->ls;
  int n = S->n;
  double *R = xc(2 * (size_t)ls->nb, 8);
  memset(ls->val, 0, 32 * (size_t)ls->nnzb);
  props_t *P = xc(n, sizeof(props_t));
  #pragma omp parallel for schedule(static)
  for (int c = 0; c < n; c++) cell_props(S, c, S->p[c], S->s[c], &P[c]);
  /* accumulation: (V/dt)[(phi rho s)^{n+1} - (phi rho s)^n] */
  #pragma omp parallel for schedule(static)
  for (int c = 0; c < n; c++) {
    double vt = S->vol[c] / S->dt, sw = S->s[c], so = 1.0 - sw;
    double *J = &ls->val[4 * (size_t)bpos(ls, c, c)];
    R[2 * c + 0] += vt * (P[c].phi * P[c].rho[1] * so - S->acc0[2 * c + 0]);
    R[2 * c + 1] += vt * (P[c].phi * P[c].rho[0] * sw - S->acc0[2 * c + 1]);
    J[0] += vt * (P[c].dphi * P[c].rho[1] + P[c].phi * P[c].drho[1]) * so;
    J[1] += vt * (-P[c].phi * P[c].rho[1]);
    J[2] += vt * (P[c].dphi * P[c].rho[0] + P[c].phi * P[c].drho[0]) * sw;
    J[3] += vt * (P[c].phi * P[c].rho[0] + P[c].phi * P[c].drhos[0] * sw);
  }
  /* face fluxes: flux into c from d is T m_u (Pot_d - Pot_c), with the
     upstream cell u = c if Pot_c >= Pot_d else d (per face, c < d); the
     same value leaves d, so mass is conserved face by face. */
  for (int f = 0; f < S->nf; f++) {
    int c = S->fc[f], d = S->fd[f];
    double T = S->ft[f];
    double *Jcc = &ls->val[4 * (size_t)bpos(ls, c, c)], *Jcd = &ls->val[4 * (size_t)bpos(ls, c, d)];
    double *Jdc = &ls->val[4 * (size_t)bpos(ls, d, c)], *Jdd = &ls->val[4 * (size_t)bpos(ls, d, d)];
    for (int a = 0; a < 2; a++) {
      int e = 1 - a;                       /* equation row: oil 0, water 1 */
      int upc = P[c].pot[a] >= P[d].pot[a];
      const props_t *U = upc ? &P[c] : &P[d];
      double dpot = P[d].pot[a] - P[c].pot[a];
      double Tm = T * U->m[a];
      double F = Tm * dpot;
      double dFdpc = T * ((upc ? P[c].dmp[a] : 0.0) * dpot) - Tm * P[c].dpot[a];
      double dFdsc = T * ((upc ? P[c].dms[a] : 0.0) * dpot) - Tm * P[c].dpots[a];
      double dFdpd = T * ((upc ? 0.0 : P[d].dmp[a]) * dpot) + Tm * P[d].dpot[a];
      double dFdsd = T * ((upc ? 0.0 : P[d].dms[a]) * dpot) + Tm * P[d].dpots[a];
      R[2 * c + e] -= F;
      R[2 * d + e] += F;
      Jcc[2 * e + 0] -= dFdpc; Jcc[2 * e + 1] -= dFdsc;
      Jcd[2 * e + 0] -= dFdpd; Jcd[2 * e + 1] -= dFdsd;
      Jdc[2 * e + 0] += dFdpc; Jdc[2 * e + 1] += dFdsc;
      Jdd[2 * e + 0] += dFdpd; Jdd[2 * e + 1] += dFdsd;
    }
  }
  /* wells: perforation rates of eq. (10) in the cell equations; the well's
     own row is its control: eq. (11) p_b = c scaled by c, or a rate
     equation (12)-(14) scaled by the target mass rate; a shut well keeps
     p_b (row 1 * p_b = current value). */
  for (int w = 0; w < S->nw; w++) {
    int wr = n + w;
    double *Jww = &ls->val[4 * (size_t)bpos(ls, wr, wr)];
    double cw, co;
    rate_weights(S, w, &cw, &co);
    for (int q = S->pptr[w]; q < S->pptr[w + 1]; q++) {
      int c = S->pcell[q];
      double *Jcc = &ls->val[4 * (size_t)bpos(ls, c, c)], *Jcw = &ls->val[4 * (size_t)bpos(ls, c, wr)];
      double *Jwc = &ls->val[4 * (size_t)bpos(ls, wr, c)];
      double qa[2], dqp[2], dqs[2], dqb[2];
      perf_flow(S, w, c, S->pwi[q], &P[c], qa, dqp, dqs, dqb);
      for (int a = 0; a < 2; a++) {
        int e = 1 - a;
        double cwt = a == 0 ? cw : co;
        R[2 * c + e] -= qa[a];
        Jcc[2 * e + 0] -= dqp[a]; Jcc[2 * e + 1] -= dqs[a];
        Jcw[2 * e + 0] -= dqb[a];
        if (cwt != 0.0) {
          R[2 * wr] += cwt * qa[a];
          Jwc[0] += cwt * dqp[a]; Jwc[1] += cwt * dqs[a];
          Jww[0] += cwt * dqb[a];
        }
      }
    }
    if (S->wctrl[w] == OR_BHP) {
      R[2 * wr] = (S->pb[w] - S->wtarget[w]) / S->wtarget[w];   /* eq. (11), scaled */
      Jww[0] = 1.0 / S->wtarget[w];
    } else if (S->wctrl[w] == OR_SHUT) {
      R[2 * wr] = 0.0; Jww[0] = 1.0;
    } else R[2 * wr] -= 1.0;
    Jww[3] = 1.0;                                                    /* padded dummy unknown */
  }
  for (int r = 0; r < 2 * ls->nb; r++) ls->b[r] = -R[r];
  /* potential key for the local reordering: oil potential, eq. (5) */
  for (int c = 0; c < n; c++) ls->key[c] = P[c].pot[1];
  ls->have_setup = 0;
  free(P); free(R);
}

/* Newton convergence measure: max over cells and phases of
   |R| dt / (rho_ref V phi_ref) (a saturation change), and |R| of the
   (already dimensionless) well rows. */
double or_sim_residual_norm(const or_sim *S)
{
  double mx = 0.0;
  for (int c = 0; c < S->n; c++)
    for (int e = 0; e < 2; e++) {
      double rr = fabs(S->ls.b[2 * c + e]) * S->dt / (S->f.rho_ref[1 - e] * S->vol[c] * S->phi[c]);
      if (!(rr <= mx)) mx = rr;          /* propagates NaN */
    }
  for (int w = 0; w < S->nw; w++) {
    double rr = fabs(S->ls.b[2 * (S->n + w)]);
    if (!(rr <= mx)) mx = rr;
  }
  return mx;
}

/* Forcing term of the inexact Newton method: eq. (26), second choice,
   eta_l = (||b(x^l)|| - ||r^{l-1}||) / ||b(x^{l-1})||, forced into
   [0.01, 0.1]; the first iteration uses eta_0 = 0.1.  Norms are 2-norms of
   the decoupled system (which the paper also writes A x = b). */
double or_forcing(int l, double bn, double rprev, double bprev)
{
  if (l == 0) return 0.1;
  double eta = (bn - rprev) / bprev;
  if (eta < 0.01) eta = 0.01;
  if (eta > 0.1) eta = 0.1;
  return eta;
}

/* Control switching with BHP limits (the paper's "various operation
   constraints ... at different time stage"; reading R22).
   Rate to BHP: after each Newton update, a rate-controlled well with a
   limit whose wellbore pressure has passed it (injector above its maximum,
   producer below its minimum) switches to BHP control at the limit, and
   p_b is set to the limit.  Returns the number of wells switched. */
static int limits_rate_to_bhp(or_sim *S)
{
  int k = 0;
  for (int w = 0; w < S->nw; w++) {
    int c = S->wctrl[w];
    if (!(c == OR_WRATE || c == OR_ORATE || c == OR_LRATE) || !(S->wlimit[w] > 0.0)) continue;
    int past = S->wkind[w] == OR_INJ ? S->pb[w] > S->wlimit[w] : S->pb[w] < S->wlimit[w];
    if (!past) continue;
    S->wctrl[w] = OR_BHP; S->wtarget[w] = S->wlimit[w]; S->pb[w] = S->wlimit[w];
    S->wswitched[w] = 1; k++;
  }
  return k;
}

/* BHP back to rate: at the start of a time step, a well held at its limit
   returns to its requested rate when, at the limit, it would deliver more
   than that rate (the rate equation's residual is positive there). */
static void limits_bhp_to_rate(or_sim *S)
{
  int any = 0;
  for (int w = 0; w < S->nw; w++)
    if (S->wswitched[w]) { S->wctrl[w] = S->wctrl0[w]; S->wtarget[w] = S->wtarget0[w]; any = 1; }
  if (!any) return;
  or_sim_assemble(S);
  for (int w = 0; w < S->nw; w++) {
    if (!S->wswitched[w]) continue;
    double r = -S->ls.b[2 * (S->n + w)];
    if (r > 0.0) S->wswitched[w] = 0;
    else { S->wctrl[w] = OR_BHP; S->wtarget[w] = S->wlimit[w]; }
  }
}

/* A new control for well w from now on (a schedule change between steps):
   the control, its target (bar or sm3/day) and the BHP limit of a rate
   control (0 = none).  A well put on a rate control starts from the
   wellbore pressure rate_start_pb. */
void or_sim_set_well(or_sim *S, int w, int control, double target, double limit)
{
  S->wctrl[w] = S->wctrl0[w] = control;
  S->wtarget[w] = S->wtarget0[w] = target;
  S->wlimit[w] = limit; S->wswitched[w] = 0;
  if (control == OR_BHP) S->pb[w] = target;
  else if (control != OR_SHUT) S->pb[w] = rate_start_pb(S, w);
}

static double nrm2(const double *v, int m) { double s = 0; for (int i = 0; i < m; i++) s += v[i] * v[i]; return sqrt(s); }

/* One time step at S->dt by Algorithm 1.  Returns 0 on convergence, 1 when
   max_newton iterations did not converge, 2 on a NaN. */
int or_sim_newton(or_sim *S, int *iters)
{
  or_sim_assemble(S);
  double bprev = 0, rprev = 0;
  int l;
  for (l = 0;; l++) {
    double nr = or_sim_residual_norm(S);
    S->last_norm = nr;
    if (nr != nr) { *iters = l; return 2; }
    if (nr <= S->o.newton_tol) { *iters = l; return 0; }
    if (l >= S->o.max_newton) { *iters = l; return 1; }
    or_lsys_setup(&S->ls);
    int nu = 2 * S->ls.nb;
    double bn = nrm2(S->ls.b, nu);
    double eta = (S->o.newton == OR_INEXACT) ? or_forcing(l, bn, rprev, bprev) : S->o.lin_tol;
    int its; double rel;
    int rc = or_lsys_solve(&S->ls, eta, S->y, &its, &rel);
    S->n_lin += its; S->last_its = its; S->last_relres = rel;
    if (rc == 2) { *iters = l; return 2; }
    bprev = bn; rprev = rel * bn;
    for (int c = 0; c < S->n; c++) {           /* x^{l+1} = x^l + y */
      double ds = S->y[2 * c + 1];
      if (S->o.sat_chop > 0.0) {                 /* optional saturation chop */
        if (ds > S->o.sat_chop) ds = S->o.sat_chop;
        if (ds < -S->o.sat_chop) ds = -S->o.sat_chop;
      }
      S->p[c] += S->y[2 * c];
      S->s[c] += ds;
      if (S->s[c] < 0.0) S->s[c] = 0.0;
      if (S->s[c] > 1.0) S->s[c] = 1.0;
    }
    for (int w = 0; w < S->nw; w++) S->pb[w] += S->y[2 * (S->n + w)];
    S->n_newton++;
    S->n_switch += limits_rate_to_bhp(S);
    or_sim_assemble(S);
  }
}

/* Time loop.  Each step covers dt; a failed Newton solve halves the step
   (at most max_cuts times per step) and the rest of the interval is
   covered with the cut step. Returns 0 or the failing Newton code. */
int or_sim_advance(or_sim *S, int nsteps)
{
  int n = S->n, nw = S->nw;
  double *p0 = xc(n, 8), *s0 = xc(n, 8), *b0 = xc(nw ? nw : 1, 8), *t0 = xc(nw ? nw : 1, 8);
  int *c0 = xc(nw ? nw : 1, 4), *w0 = xc(nw ? nw : 1, 4);
  int rc = 0;
  for (int st = 0; st < nsteps && rc == 0; st++) {
    double rem = S->o.dt, h = S->o.dt;
    int cuts = 0;
    while (rem > 0.0) {
      double dt = h < rem ? h : rem;
      memcpy(p0, S->p, 8 * (size_t)n); memcpy(s0, S->s, 8 * (size_t)n);
      if (nw) memcpy(b0, S->pb, 8 * (size_t)nw);
      or_sim_store_old(S);
      S->dt = dt;
      limits_bhp_to_rate(S);
      if (nw) { memcpy(c0, S->wctrl, 4 * (size_t)nw); memcpy(t0, S->wtarget, 8 * (size_t)nw);
                memcpy(w0, S->wswitched, 4 * (size_t)nw); }
      int its;
      int r = or_sim_newton(S, &its);
      if (r == 0) { S->t += dt; rem -= dt; S->n_steps++; continue; }
      memcpy(S->p, p0, 8 * (size_t)n); memcpy(S->s, s0, 8 * (size_t)n);
      if (nw) { memcpy(S->pb, b0, 8 * (size_t)nw); memcpy(S->wctrl, c0, 4 * (size_t)nw);
                memcpy(S->wtarget, t0, 8 * (size_t)nw); memcpy(S->wswitched, w0, 4 * (size_t)nw); }
      S->n_cuts++; cuts++;
      if (cuts > S->o.max_cuts) { rc = r; break; }
      h = 0.5 * h;
    }
  }
  free(p0); free(s0); free(b0); free(t0); free(c0); free(w0);
  return rc;
}

/* plain linear solve of the currently assembled system (test hook) */
int or_sim_linear_solve(or_sim *S, double tol, double *y, int *its, double *relres)
{
  or_lsys_setup(&S->ls);
  int rc = or_lsys_solve(&S->ls, tol, S->y, its, relres);
  memcpy(y, S->y, 16 * (size_t)S->ls.nb);
  return rc;
}

/* ---- small accessors for the Python binding ---- */
or_lsys *or_sim_lsys(or_sim *S) { return &S->ls; }
void or_sim_set_dt(or_sim *S, double dt) { S->dt = dt; }
void or_sim_stats(const or_sim *S, double *out)
{
  out[0] = (double)S->n_steps; out[1] = (double)S->n_newton; out[2] = (double)S->n_lin;
  out[3] = (double)S->n_cuts; out[4] = S->last_relres; out[5] = S->last_its; out[6] = S->last_norm;
  out[7] = S->t; out[8] = (double)S->n_switch;
}
void or_sim_well_controls(const or_sim *S, int *ctrl, double *target)
{
  for (int w = 0; w < S->nw; w++) { ctrl[w] = S->wctrl[w]; target[w] = S->wtarget[w]; }
}
void or_sim_well_rates(const or_sim *S, double *qw, double *qo)
{
  /* total mass rates per well at the current state (kg/day, + = injection) */
  for (int w = 0; w < S->nw; w++) {
    qw[w] = qo[w] = 0.0;
    for (int q = S->pptr[w]; q < S->pptr[w + 1]; q++) {
      int c = S->pcell[q];
      props_t P; cell_props(S, c, S->p[c], S->s[c], &P);
      double qa[2], d1[2], d2[2], d3[2];
      perf_flow(S, w, c, S->pwi[q], &P, qa, d1, d2, d3);
      qw[w] += qa[0]; qo[w] += qa[1];
    }
  }
}
void or_sim_mass(const or_sim *S, double *mw, double *mo)
{
  /* fluid mass in place, sum over cells of V phi rho_a s_a */
  *mw = *mo = 0.0;
  for (int c = 0; c < S->n; c++) {
    props_t P; cell_props(S, c, S->p[c], S->s[c], &P);
    *mw += S->vol[c] * P.phi * P.rho[0] * S->s[c];
    *mo += S->vol[c] * P.phi * P.rho[1] * (1.0 - S->s[c]);
  }
}
void or_sim_get_wi(const or_sim *S, double *wi) { memcpy(wi, S->pwi, 8 * (size_t)S->pptr[S->nw]); }
