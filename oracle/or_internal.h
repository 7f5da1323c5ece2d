/* Internal declarations of the CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow, single-threaded
 * FP64 restatement of the method of Liu et al., "A Parallel Simulator for
 * Massive Reservoir Models Utilizing Distributed-Memory Parallel Systems"
 * (arXiv 1701.06254).  Only the test suite, __graft_entry__.smoke() and the
 * CPU-baseline leg of bench.py load it.  It shares no code with the CUDA
 * library.  Built with -O2 -ffp-contract=off: every a*b+c rounds twice.
 * A second build with -fopenmp (liboracle_omp.so, for timing the oracle on
 * all host cores) runs the loops marked "omp parallel for" on several
 * threads: each of those writes disjoint outputs and sums nothing across
 * iterations, so both builds give bit-identical results.
 */
#ifndef OR_INTERNAL_H
#define OR_INTERNAL_H
#include <stdint.h>
#include <stddef.h>

/* Darcy constant for k[mD]*A[m2]/L[m]*dp[bar]/mu[cP] -> m3/day:
   9.869233e-16 m2/mD * 1e5 Pa/bar / 1e-3 Pa s/cP * 86400 s/day. */
#define OR_CDARCY (9.869233e-16 * 1e5 / 1e-3 * 86400.0)
#define OR_PA2BAR 1e-5

enum { OR_INJ = 0, OR_PROD = 1 };
enum { OR_BHP = 0, OR_WRATE = 1, OR_ORATE = 2, OR_LRATE = 3, OR_SHUT = 4 };
enum { OR_DEC_NONE = 0, OR_DEC_ABF = 1, OR_DEC_QI = 2 };
enum { OR_STANDARD = 0, OR_INEXACT = 1 };
enum { OR_FGMRES = 0, OR_BICGSTAB = 1 };

typedef struct {
  int nx, ny, nz;
  double dx, dy, dz, top;
} or_grid;

typedef struct {          /* index 0 = water, 1 = oil */
  double rho_ref[2], c_f[2], mu_ref[2], c_mu[2];
  double p_ref, c_r, swc, sor, nw, no, krw_max, kro_max, g;
  int pc_n;                        /* capillary pressure table (eq. 9): points, 0 = p_c = 0 */
  const double *pc_sw, *pc_val;    /* s_w ascending, p_c in bar */
} or_fluid;

typedef struct {
  int kind, control;
  double target, r_w, skin, z_ref;
  int n_perf;
  const int *perf_cell;
  const double *wi;       /* NULL -> Peaceman well index */
  double bhp_limit;       /* rate wells: injector maximum / producer minimum p_b, 0 = none */
} or_well;

typedef struct {
  int decoupling, reorder, newton;
  double newton_tol, lin_tol;
  int max_newton, restart, max_lin;
  int tile_x, tile_y;
  double amg_theta;
  int amg_max_levels, amg_coarse_max;
  uint64_t seed;
  int max_cuts;
  double dt;
  double sat_chop;       /* max |ds_w| per Newton update, 0 = full step */
  int krylov;            /* OR_FGMRES or OR_BICGSTAB */
  int overlap;           /* RAS overlap (graph distance), 1 or 2 */
  int interp;            /* AMG interpolation: 0 direct, 1 extended+i */
} or_opts;

/* ---- compressed sparse rows (scalar) ---- */
typedef struct { int n, m, nnz; int *rp, *ci; double *v; } or_csr;

/* ---- AMG hierarchy on the pressure block ---- */
typedef struct {
  or_csr A, P, R;         /* A: n x n, P: n x nc, R = P^T */
  signed char *cf;        /* 1 = C, -1 = F */
  unsigned char *strong;  /* per nonzero of A */
  double *dl1;            /* l1-Jacobi diagonal */
  int pmis_rounds;
} or_level;

typedef struct {
  int nlev;               /* levels 0..nlev-1, the last one is the coarsest */
  or_level lev[32];
  int coarse_dense;       /* 1: dense LU on the coarsest level, 0: Jacobi sweeps */
  double *lu; int *piv;   /* dense LU of the coarsest level */
} or_amg;

/* ---- RAS subdomain ---- */
typedef struct {
  int nown, next;         /* owned unknown rows, extended (owned + overlap) rows */
  int *own;               /* global block rows owned */
  int *ext;               /* global block rows of the local system, in local order */
  int *rp, *ci;           /* local block CSR (columns sorted by local index) */
  double *lu;             /* 4 per block: L (strict lower) and U (upper) in place */
  double *dinv;           /* 4 per row: inverse of the U diagonal block */
  int *diag;              /* position of the diagonal block in each row */
  int *opos;              /* local position of each owned row */
} or_sub;

/* ---- linear system: 2x2 block CSR over n cells + nw well rows ---- */
typedef struct {
  int nx, ny, nz, n, nw, nb;   /* nb = n + nw block rows */
  int *rp, *ci, nnzb;          /* pattern */
  double *val;                 /* 4 per block, row-major; decoupled after setup */
  double *b;                   /* 2 per block row */
  double *key;                 /* oil potential per cell (reordering key) */
  int *well_cell0;             /* first perforated cell of each well */
  int nsub; or_sub *sub;
  or_amg amg;
  double *dmat;                /* 4 per block row: decoupling operator D (for r = D r~) */
  or_opts o;
  int have_setup;
} or_lsys;

/* ---- simulator ---- */
typedef struct {
  or_grid g; int n;
  double *kx, *ky, *kz, *phi, *z, *vol;
  or_fluid f;
  int nw; int *wkind, *wctrl; double *wtarget, *wzref;
  int *wctrl0; double *wtarget0, *wlimit;  /* requested control and target, BHP limit */
  int *wswitched;                          /* 1: on BHP at its limit instead of its rate */
  double *pc_sw, *pc_val;                  /* copy of the capillary pressure table */
  int *pptr, *pcell; double *pwi;        /* perforations, CSR by well */
  int nf; int *fc, *fd; double *ft;      /* interior faces c < d, geometric transmissibility */
  or_opts o;
  or_lsys ls;                            /* pattern + storage of the Jacobian */
  double *p, *s, *pb;                    /* current iterate */
  double *acc0;                          /* 2 per cell: (phi rho s)^n for oil, water */
  double t, dt;
  double *y;                             /* last Newton update (2 per block row) */
  /* statistics */
  long n_newton, n_lin, n_steps, n_cuts, n_switch;
  double last_relres; int last_its;
  double last_norm;
} or_sim;

/* or_amg.c */
void or_csr_free(or_csr *a);
void or_amg_free(or_amg *h);
int  or_amg_setup(or_amg *h, const or_csr *A0, double theta, uint64_t seed,
                  int coarse_max, int max_levels, int interpolation);
void or_amg_vcycle(const or_amg *h, int l, const double *f, double *x);
uint64_t or_splitmix64(uint64_t x);
double or_pmis_hash(uint64_t seed, int level, int i);
void or_spgemm(const or_csr *A, const or_csr *B, or_csr *C);
void or_transpose(const or_csr *A, or_csr *T);

/* or_solve.c */
void or_lsys_init_pattern(or_lsys *ls, int nx, int ny, int nz, int nw,
                          const int *rp, const int *ci, const int *well_cell0);
void or_lsys_free(or_lsys *ls);
int  or_lsys_setup(or_lsys *ls);
int  or_lsys_solve(or_lsys *ls, double tol, double *y, int *its, double *relres);
void or_bsr_mv(const or_lsys *ls, const double *x, double *y);
void or_cpr_apply(or_lsys *ls, const double *f, double *x);
void or_ras_apply(const or_lsys *ls, const double *f, double *x);
void or_potential_rank(int m, const double *key, const int *idx, int *order);

#endif
