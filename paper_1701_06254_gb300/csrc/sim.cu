// The fully implicit oil-water model on the GPU and the C ABI.
//
// Model (arXiv 1701.06254, Sec. "Two-phase oil-water flow model"): mass
// balance eq. (3) with porosity eq. (4), potential eq. (5) (z = depth),
// density eq. (6), viscosity eq. (7), s_o = 1 - s_w eq. (8), Corey relative
// permeabilities, Peaceman wells eq. (10) with BHP eq. (11) and water-rate
// eq. (12) constraints.  Discretisation (Sec. "Numerical methods"): backward
// Euler eq. (15), two-point fluxes with the geometric transmissibility times
// the upstream mobility (eqs. 16-18; upstream cell of face (c, d), c < d:
// c if Phi_c >= Phi_d, else d), residual eq. (17).  Newton: Algorithm 1,
// forcing term eq. (26) second choice, clamped to [0.01, 0.1].  Also the
// oil-rate (13) and liquid-rate (14) constraints, BHP limits with control
// switching, schedule changes and shut wells, and a capillary pressure
// table (eq. 9: p_w = p_o - p_c(s_w)).
#include "common.cuh"
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <new>

#define PC_MAX 16                      // points of the capillary pressure table
struct fluid_c {
  double rho_ref[2], c_f[2], mu_ref[2], c_mu[2];
  double p_ref, c_r, swc, sor, nw, no, krw_max, kro_max, g;
  double span, inv_span;               // 1 - swc - sor and its reciprocal (formed once, IEEE)
  int pc_n;                            // 0: no capillary pressure
  double pc_sw[PC_MAX], pc_val[PC_MAX];
};

struct sim_s {
  int nx, ny, nz, n, nw, np_;
  double dx, dy, dz, top;
  fluid_c fl;
  rs_opts o;
  cudaStream_t st;
  std::vector<int> wkind, wctrl, pptr;
  std::vector<double> wtarget, wzref;
  // requested control and target, BHP limit, held at the limit (switching)
  std::vector<int> wctrl0, wswitched;
  std::vector<double> wtarget0, wlimit;
  bool any_limit = false;
  dbuf<double> kx, ky, kz, phi, tx, ty, tz;
  dbuf<int> pcell, pwell, ppos_cw, ppos_wc, cpp, cpi, wpptr, wdiag, wkind_d, wctrl_d;
  dbuf<double> pwi, wtarget_d, wzref_d;
  dbuf<double> p, s, pb, acc0, props, p0, s0, pb0, red;
  double t = 0.0, dt = 1.0;
  sim_ls_s *ls = nullptr;
  sim_stats stats;
  // learned warm start: the network used for initial guesses, the one that
  // records (features, target) pairs, the previous solve's update and the
  // scales [rms b_p, rms b_s, rms y_p, rms y_s (of the solved update), rms y_prev_p, rms y_prev_s]
  sim_ws_s *ws = nullptr, *rec = nullptr;
  dbuf<double> yprev, wsc, dws, u, yfirst;
  bool have_prev = false, have_first = false, first_pending = false;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  ~sim_s() { delete ls; if (e0) cudaEventDestroy(e0); if (e1) cudaEventDestroy(e1); }
};

// ----------------------------------------------------------- properties --
struct cprops {
  double phi, dphi, pc, dpc, rho[2], drho[2], drhos[2], mu[2], dmu[2], dmus[2], kr[2], dkr[2], m[2], dmp[2], dms[2],
      pot[2], dpot[2], dpots[2];
};

__device__ __forceinline__ double corey(double x, double e) {
  if (e == 2.0) return x * x;
  if (e == 1.0) return x;
  if (e == 3.0) return x * x * x;
  return pow(x, e);
}

// Values that decide an integer (the upstream cell via the potential, the
// relative-permeability clamp, the producer cut-off via the density) are
// formed with round-to-nearest operations in the order of the plain
// formulas, so equal inputs give equal decisions in any implementation that
// evaluates the same formulas in IEEE arithmetic.
__device__ __forceinline__ double rho_of(const fluid_c &f, int a, double p) {
  return mul_rn(f.rho_ref[a], add_rn(1.0, mul_rn(f.c_f[a], sub_rn(p, f.p_ref))));
}
// capillary pressure of eq. (9) from the table: straight lines between its
// points, constant beyond its ends; the segment is the last k with
// sw[k] <= s, its slope the derivative (0 outside)
__device__ __forceinline__ void capillary(const fluid_c &f, double s, double &pc, double &dpc) {
  int n = f.pc_n;
  if (n <= 0) { pc = 0.0; dpc = 0.0; return; }
  if (n == 1 || s < f.pc_sw[0]) { pc = f.pc_val[0]; dpc = 0.0; return; }
  if (s >= f.pc_sw[n - 1]) { pc = f.pc_val[n - 1]; dpc = 0.0; return; }
  int k = 0;
  while (s >= f.pc_sw[k + 1]) k++;
  double slope = div_rn(sub_rn(f.pc_val[k + 1], f.pc_val[k]), sub_rn(f.pc_sw[k + 1], f.pc_sw[k]));
  pc = add_rn(f.pc_val[k], mul_rn(sub_rn(s, f.pc_sw[k]), slope));
  dpc = slope;
}

__device__ __forceinline__ void cell_props(const fluid_c &f, double phir, double z, double p, double sw, cprops &P) {
  double dp = p - f.p_ref;
  P.phi = phir * (1.0 + f.c_r * dp);
  P.dphi = phir * f.c_r;
  capillary(f, sw, P.pc, P.dpc);
  double sh = div_rn(sub_rn(sw, f.swc), f.span), dsh = f.inv_span;
  if (sh < 0.0) { sh = 0.0; dsh = 0.0; } else if (sh > 1.0) { sh = 1.0; dsh = 0.0; }
  P.kr[0] = f.krw_max * corey(sh, f.nw);
  P.dkr[0] = f.krw_max * f.nw * corey(sh, f.nw - 1.0) * dsh;
  P.kr[1] = f.kro_max * corey(1.0 - sh, f.no);
  P.dkr[1] = -f.kro_max * f.no * corey(1.0 - sh, f.no - 1.0) * dsh;
  double gz5 = mul_rn(mul_rn(f.g, z), RS_PA2BAR);
#pragma unroll
  for (int a = 0; a < 2; a++) {
    // phase pressure, eq. (9): p_w = p_o - p_c(s_w)
    double pa = a == 0 ? sub_rn(p, P.pc) : p, dpa_s = a == 0 ? -P.dpc : 0.0;
    P.rho[a] = rho_of(f, a, pa);
    P.drho[a] = f.rho_ref[a] * f.c_f[a];
    P.drhos[a] = P.drho[a] * dpa_s;
    P.mu[a] = f.mu_ref[a] + f.c_mu[a] * (pa - f.p_ref);
    P.dmu[a] = f.c_mu[a];
    P.dmus[a] = f.c_mu[a] * dpa_s;
    double imu = 1.0 / P.mu[a];
    P.m[a] = P.rho[a] * P.kr[a] * imu;
    P.dmp[a] = P.drho[a] * P.kr[a] * imu - P.rho[a] * P.kr[a] * P.dmu[a] * imu * imu;
    P.dms[a] = P.rho[a] * P.dkr[a] * imu + P.drhos[a] * P.kr[a] * imu - P.rho[a] * P.kr[a] * P.dmus[a] * imu * imu;
    P.pot[a] = sub_rn(pa, mul_rn(P.rho[a], gz5));
    P.dpot[a] = 1.0 - P.drho[a] * gz5;
    P.dpots[a] = dpa_s - P.drhos[a] * gz5;
  }
}

__device__ __forceinline__ double depth(double top, double dz, int k) { return add_rn(top, mul_rn((double)k + 0.5, dz)); }

// per-cell table (SoA, 15 x n): mobilities, potentials and their
// derivatives for the face terms (rows 0-10), and for the accumulation term
// phi, rho_w, rho_o and d rho_w / d s_w (rows 11-14)
__global__ void k_props(int n, int nxy, fluid_c f, double top, double dz, const double *phi, const double *p,
                        const double *s, double *pr) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  cprops P;
  cell_props(f, phi[c], depth(top, dz, c / nxy), p[c], s[c], P);
  pr[0 * (size_t)n + c] = P.m[0]; pr[1 * (size_t)n + c] = P.m[1];
  pr[2 * (size_t)n + c] = P.dmp[0]; pr[3 * (size_t)n + c] = P.dmp[1];
  pr[4 * (size_t)n + c] = P.dms[0]; pr[5 * (size_t)n + c] = P.dms[1];
  pr[6 * (size_t)n + c] = P.pot[0]; pr[7 * (size_t)n + c] = P.pot[1];
  pr[8 * (size_t)n + c] = P.dpot[0]; pr[9 * (size_t)n + c] = P.dpot[1];
  pr[10 * (size_t)n + c] = P.dpots[0];                // the oil potential does not depend on s_w
  pr[11 * (size_t)n + c] = P.phi; pr[12 * (size_t)n + c] = P.rho[0]; pr[13 * (size_t)n + c] = P.rho[1];
  pr[14 * (size_t)n + c] = P.drhos[0];
}

// geometric two-point transmissibility of the +x, +y, +z face of each cell
__global__ void k_trans(int nx, int ny, int nz, double dx, double dy, double dz, const double *kx, const double *ky,
                        const double *kz, double *tx, double *ty, double *tz) {
  int c = blockIdx.x * blockDim.x + threadIdx.x, n = nx * ny * nz;
  if (c >= n) return;
  int i = c % nx, j = (c / nx) % ny, k = c / (nx * ny);
  tx[c] = i + 1 < nx ? RS_CDARCY * (dy * dz) / (dx / (2.0 * kx[c]) + dx / (2.0 * kx[c + 1])) : 0.0;
  ty[c] = j + 1 < ny ? RS_CDARCY * (dx * dz) / (dy / (2.0 * ky[c]) + dy / (2.0 * ky[c + nx])) : 0.0;
  tz[c] = k + 1 < nz ? RS_CDARCY * (dx * dy) / (dz / (2.0 * kz[c]) + dz / (2.0 * kz[c + nx * ny])) : 0.0;
}

// Peaceman well index per perforation
__global__ void k_peaceman(int np_, double dx, double dy, double dz, const int *pcell, const int *pwell,
                           const double *rw, const double *skin, const double *kx, const double *ky, double *wi) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= np_) return;
  if (wi[q] >= 0.0) return;                 // given by the caller
  int c = pcell[q], w = pwell[q];
  double a = kx[c], b = ky[c];
  double ro = 0.28 * sqrt(sqrt(b / a) * dx * dx + sqrt(a / b) * dy * dy) / (pow(b / a, 0.25) + pow(a / b, 0.25));
  wi[q] = 2.0 * M_PI * RS_CDARCY * sqrt(a * b) * dz / (log(ro / rw[w]) + skin[w]);
}

// Mass rates of one perforation (eq. 10) for both phases (0 = water, 1 =
// oil; + = into the cell) and their derivatives with respect to the cell's
// p, s_w and to p_b.  Drawdown of phase a: dd = p_b - p_a + rho_a g (z -
// z_ref).  Producer: own phase mobility, outflow only; injector (dd >= 0):
// water only with the total cell mobility; injector crossflow (dd < 0):
// upstream from the cell like a producer; a shut well carries nothing.
struct pflow { double q[2], dqp[2], dqs[2], dqb[2]; };
__device__ __forceinline__ void perf_flow(const fluid_c &f, int kind, int ctrl, double wi, const cprops &P, double pc_,
                                          double pbw, double dz5, pflow &F) {
#pragma unroll
  for (int a = 0; a < 2; a++) {
    F.q[a] = F.dqp[a] = F.dqs[a] = F.dqb[a] = 0.0;
    if (ctrl == SIM_SHUT) continue;
    double pa = a == 0 ? sub_rn(pc_, P.pc) : pc_;
    double dd = add_rn(sub_rn(pbw, pa), mul_rn(P.rho[a], dz5));
    double dd_dp = -1.0 + P.drho[a] * dz5, dd_ds = (a == 0 ? P.dpc : 0.0) + P.drhos[a] * dz5;
    if (kind == SIM_PROD || dd < 0.0) {         // producer, or injector crossflow: upstream = cell
      if (dd <= 0.0) {
        F.q[a] = wi * P.m[a] * dd; F.dqp[a] = wi * (P.dmp[a] * dd + P.m[a] * dd_dp);
        F.dqs[a] = wi * (P.dms[a] * dd + P.m[a] * dd_ds); F.dqb[a] = wi * P.m[a];
      }
    } else if (a == 0) {                          // injection; at dd = 0 the injecting-side derivative
      double lt = P.kr[0] / P.mu[0] + P.kr[1] / P.mu[1];
      double lt_p = -P.kr[0] * P.dmu[0] / (P.mu[0] * P.mu[0]) - P.kr[1] * P.dmu[1] / (P.mu[1] * P.mu[1]);
      double lt_s = P.dkr[0] / P.mu[0] - P.kr[0] * P.dmus[0] / (P.mu[0] * P.mu[0]) + P.dkr[1] / P.mu[1] -
                    P.kr[1] * P.dmus[1] / (P.mu[1] * P.mu[1]);
      F.q[a] = wi * P.rho[0] * lt * dd;
      F.dqp[a] = wi * (P.drho[0] * lt * dd + P.rho[0] * lt_p * dd + P.rho[0] * lt * dd_dp);
      F.dqs[a] = wi * (P.drhos[0] * lt * dd + P.rho[0] * lt_s * dd + P.rho[0] * lt * dd_ds);
      F.dqb[a] = wi * P.rho[0] * lt;
    }
  }
}

// --------------------------------------------------------------- assembly --
// One thread per cell: accumulation, the six faces (evaluated from this
// cell's side; the neighbour evaluates the same face with the same
// transmissibility and upstream choice, so the two fluxes are exact
// negatives), and the cell's perforations.  Writes the whole block row.
__global__ void __launch_bounds__(128)
k_assemble(int nx, int ny, int nz, fluid_c f, double top, double dz, double vol_dt, const double *__restrict__ phi,
           const double *__restrict__ p, const double *__restrict__ s, const double *__restrict__ pbh,
           const double *__restrict__ acc0, const double *__restrict__ pr, const double *__restrict__ tx,
           const double *__restrict__ ty, const double *__restrict__ tz, const int *__restrict__ rp,
           const int *__restrict__ cpp, const int *__restrict__ cpi, const int *__restrict__ pwell,
           const double *__restrict__ pwi, const int *__restrict__ ppos_cw, const int *__restrict__ wkind,
           const int *__restrict__ wctrl, const double *__restrict__ wzref, double *__restrict__ val,
           double *__restrict__ b) {
  int n = nx * ny * nz, c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  int nxy = nx * ny, i = c % nx, j = (c / nx) % ny, k = c / nxy;
  double z = depth(top, dz, k);
  double pc = p[c], sc = s[c];
  // the accumulation term from the table k_props wrote (the same cell_props
  // values); the full properties only for a perforated cell
  double Pphi = pr[11 * (size_t)n + c], Prho0 = pr[12 * (size_t)n + c], Prho1 = pr[13 * (size_t)n + c];
  double Pdrhos0 = pr[14 * (size_t)n + c], Pdphi = phi[c] * f.c_r;
  double Pdrho0 = f.rho_ref[0] * f.c_f[0], Pdrho1 = f.rho_ref[1] * f.c_f[1];
  double so = 1.0 - sc;
  double R0 = vol_dt * (Pphi * Prho1 * so - acc0[2 * (size_t)c]);
  double R1 = vol_dt * (Pphi * Prho0 * sc - acc0[2 * (size_t)c + 1]);
  double D[4];
  D[0] = vol_dt * (Pdphi * Prho1 + Pphi * Pdrho1) * so;
  D[1] = vol_dt * (-Pphi * Prho1);
  D[2] = vol_dt * (Pdphi * Prho0 + Pphi * Pdrho0) * sc;
  D[3] = vol_dt * (Pphi * Prho0 + Pphi * Pdrhos0 * sc);
  // neighbours in ascending column order: -z, -y, -x, (self), +x, +y, +z
  int nb_[6] = {k > 0 ? c - nxy : -1, j > 0 ? c - nx : -1, i > 0 ? c - 1 : -1,
                i + 1 < nx ? c + 1 : -1, j + 1 < ny ? c + nx : -1, k + 1 < nz ? c + nxy : -1};
  double T_[6] = {k > 0 ? tz[c - nxy] : 0.0, j > 0 ? ty[c - nx] : 0.0, i > 0 ? tx[c - 1] : 0.0, tx[c], ty[c], tz[c]};
  int slot = rp[c], diag_slot = -1;
  for (int t = 0; t < 6; t++) {
    if (t == 3) diag_slot = slot++;
    int d = nb_[t];
    if (d < 0) continue;
    double T = T_[t];
    double O[4];
#pragma unroll
    for (int a = 0; a < 2; a++) {
      int e = 1 - a;
      double md = pr[(size_t)a * n + d], dmpd = pr[(size_t)(2 + a) * n + d], dmsd = pr[(size_t)(4 + a) * n + d];
      double potd = pr[(size_t)(6 + a) * n + d], dpotd = pr[(size_t)(8 + a) * n + d];
      double mc = pr[(size_t)a * n + c], dmpc = pr[(size_t)(2 + a) * n + c], dmsc = pr[(size_t)(4 + a) * n + c];
      double potc = pr[(size_t)(6 + a) * n + c], dpotc = pr[(size_t)(8 + a) * n + c];
      double dpotsc = a == 0 ? pr[(size_t)10 * n + c] : 0.0, dpotsd = a == 0 ? pr[(size_t)10 * n + d] : 0.0;
      // upstream side by the potentials (compared on integer keys: the same
      // decision as the IEEE comparison, off the FP64 pipe); the mobility
      // derivative terms only on the upstream side, so each derivative is one
      // product plus, upstream, one more (T dpot shared)
      long long kc = dkey(potc), kd = dkey(potd);
      bool upc = (c < d) ? (kc >= kd) : !(kd >= kc);
      double dpot = potd - potc;
      double Tm = T * (upc ? mc : md);
      double F = Tm * dpot;
      double X = T * dpot;
      double up_p = (upc ? dmpc : dmpd) * X, up_s = (upc ? dmsc : dmsd) * X;
      double dFdpc = (upc ? up_p : 0.0) - Tm * dpotc;
      double dFdsc = (upc ? up_s : 0.0) - Tm * dpotsc;
      double dFdpd = (upc ? 0.0 : up_p) + Tm * dpotd;
      double dFdsd = (upc ? 0.0 : up_s) + Tm * dpotsd;
      if (e == 0) R0 -= F; else R1 -= F;
      D[2 * e] -= dFdpc; D[2 * e + 1] -= dFdsc;
      O[2 * e] = -dFdpd; O[2 * e + 1] = -dFdsd;
    }
    double *Bo = val + 4 * (size_t)slot++;
    reinterpret_cast<double2 *>(Bo)[0] = make_double2(O[0], O[1]);
    reinterpret_cast<double2 *>(Bo)[1] = make_double2(O[2], O[3]);
  }
  // perforations of this cell (eq. 10)
  cprops P;
  if (cpp[c + 1] > cpp[c]) cell_props(f, phi[c], z, pc, sc, P);
  for (int a2 = cpp[c]; a2 < cpp[c + 1]; a2++) {
    int q = cpi[a2], w = pwell[q];
    double dz5 = mul_rn(mul_rn(f.g, sub_rn(z, wzref[w])), RS_PA2BAR);
    pflow F;
    perf_flow(f, wkind[w], wctrl[w], pwi[q], P, pc, pbh[w], dz5, F);
    double W[4] = {0, 0, 0, 0};
#pragma unroll
    for (int a = 0; a < 2; a++) {
      int e = 1 - a;
      if (e == 0) R0 -= F.q[a]; else R1 -= F.q[a];
      D[2 * e] -= F.dqp[a]; D[2 * e + 1] -= F.dqs[a];
      W[2 * e] = -F.dqb[a];
    }
    double *Bw = val + 4 * (size_t)ppos_cw[q];
    Bw[0] = W[0]; Bw[1] = 0.0; Bw[2] = W[2]; Bw[3] = 0.0;
  }
  double *Bd = val + 4 * (size_t)diag_slot;
  reinterpret_cast<double2 *>(Bd)[0] = make_double2(D[0], D[1]);
  reinterpret_cast<double2 *>(Bd)[1] = make_double2(D[2], D[3]);
  reinterpret_cast<double2 *>(b)[c] = make_double2(-R0, -R1);
}

// well rows, one warp per well (lanes over its perforations, partial sums
// combined by shuffles in a fixed order): BHP control eq. (11) scaled by the
// target; a rate control sum_m (cw q_w + co q_o) - 1 with the weights of
// eq. (12) water, (13) oil or (14) liquid rate in surface volumes over the
// target (production positive for a producer); a shut well keeps p_b
// (1 * p_b, residual 0)
__global__ void k_wells(int n, int nw, fluid_c f, double top, double dz, int nxy, const double *phi, const double *p,
                        const double *s, const double *pbh, const int *wpptr, const int *pcell, const double *pwi,
                        const int *ppos_wc, const int *wdiag, const int *wkind, const int *wctrl, const double *wtarget,
                        const double *wzref, double *val, double *b) {
  int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (w >= nw) return;                               // the whole warp
  int ctrl = wctrl[w];
  double sgn = wkind[w] == SIM_PROD ? -1.0 : 1.0, T = wtarget[w];
  double cw = (ctrl == SIM_WRATE || ctrl == SIM_LRATE) ? sgn / (f.rho_ref[0] * T) : 0.0;
  double co = (ctrl == SIM_ORATE || ctrl == SIM_LRATE) ? sgn / (f.rho_ref[1] * T) : 0.0;
  bool rate = cw != 0.0 || co != 0.0;
  double R = 0.0, Jww = 0.0;
  for (int q = wpptr[w] + lane; q < wpptr[w + 1]; q += 32) {
    int c = pcell[q];
    double *B = val + 4 * (size_t)ppos_wc[q];
    double b0 = 0, b1 = 0;
    if (rate) {
      cprops P;
      double z = depth(top, dz, c / nxy);
      cell_props(f, phi[c], z, p[c], s[c], P);
      double dz5 = mul_rn(mul_rn(f.g, sub_rn(z, wzref[w])), RS_PA2BAR);
      pflow F;
      perf_flow(f, wkind[w], ctrl, pwi[q], P, p[c], pbh[w], dz5, F);
      R += cw * F.q[0] + co * F.q[1];
      b0 = cw * F.dqp[0] + co * F.dqp[1];
      b1 = cw * F.dqs[0] + co * F.dqs[1];
      Jww += cw * F.dqb[0] + co * F.dqb[1];
    }
    B[0] = b0; B[1] = b1; B[2] = 0.0; B[3] = 0.0;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    R += __shfl_xor_sync(0xffffffffu, R, o);
    Jww += __shfl_xor_sync(0xffffffffu, Jww, o);
  }
  if (lane != 0) return;
  if (rate) R -= 1.0;
  else if (ctrl == SIM_SHUT) { R = 0.0; Jww = 1.0; }
  else { R = (pbh[w] - wtarget[w]) / wtarget[w]; Jww = 1.0 / wtarget[w]; }
  double *Bd = val + 4 * (size_t)wdiag[w];
  Bd[0] = Jww; Bd[1] = 0.0; Bd[2] = 0.0; Bd[3] = 1.0;
  b[2 * (size_t)(n + w)] = -R; b[2 * (size_t)(n + w) + 1] = 0.0;
}

// reordering key: oil potential, eq. (5), evaluated in a fixed IEEE order
__global__ void k_key(int n, int nxy, fluid_c f, double top, double dz, const double *p, double *key) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  double z = depth(top, dz, c / nxy);
  double gz5 = mul_rn(mul_rn(f.g, z), RS_PA2BAR);
  double rho = mul_rn(f.rho_ref[1], add_rn(1.0, mul_rn(f.c_f[1], sub_rn(p[c], f.p_ref))));
  key[c] = sub_rn(p[c], mul_rn(rho, gz5));
}

// scaled residual norm (max), one partial per block, then a max in order
__global__ void k_norm_part(int n, int nw, double dt_vol_inv, const fluid_c f, const double *phi, const double *b,
                            double *part) {
  __shared__ double sh[256];
  double mx = 0.0;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n + nw; c += gridDim.x * blockDim.x) {
    double r0, r1;
    if (c < n) {
      r0 = fabs(b[2 * (size_t)c]) * dt_vol_inv / (f.rho_ref[1] * phi[c]);
      r1 = fabs(b[2 * (size_t)c + 1]) * dt_vol_inv / (f.rho_ref[0] * phi[c]);
    } else { r0 = fabs(b[2 * (size_t)c]); r1 = 0.0; }
    if (!(r0 <= mx)) mx = r0;
    if (!(r1 <= mx)) mx = r1;
  }
  sh[threadIdx.x] = mx;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) { double x = sh[threadIdx.x + o]; if (!(x <= sh[threadIdx.x])) sh[threadIdx.x] = x; }
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = sh[0];
}
__global__ void k_max_part(int m, const double *part, double *out) {
  int lane = threadIdx.x;
  double mx = 0.0;
  for (int k = lane; k < m; k += 32) { double x = part[k]; if (!(x <= mx)) mx = x; }
  for (int o = 16; o > 0; o >>= 1) { double y = __shfl_down_sync(0xffffffffu, mx, o); if (!(y <= mx)) mx = y; }
  if (lane == 0) *out = mx;
}

// x += y (Algorithm 1), with the optional saturation chop, then s_w in [0, 1]
__global__ void k_update(int n, int nw, double chop, const double *y, double *p, double *s, double *pb) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n) {
    p[c] += y[2 * (size_t)c];
    double ds = y[2 * (size_t)c + 1];
    if (chop > 0.0) ds = ds > chop ? chop : (ds < -chop ? -chop : ds);
    double v = s[c] + ds;
    s[c] = v < 0.0 ? 0.0 : (v > 1.0 ? 1.0 : v);
  } else if (c < n + nw) {
    pb[c - n] += y[2 * (size_t)c];
  }
}

__global__ void k_store_old(int n, int nxy, fluid_c f, double top, double dz, const double *phi, const double *p,
                            const double *s, double *acc0) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  cprops P;
  cell_props(f, phi[c], depth(top, dz, c / nxy), p[c], s[c], P);
  acc0[2 * (size_t)c] = P.phi * P.rho[1] * (1.0 - s[c]);
  acc0[2 * (size_t)c + 1] = P.phi * P.rho[0] * s[c];
}

__global__ void k_hydrostatic(int n, int nxy, fluid_c f, double top, double dz, double p_datum, double sw0, double *p,
                              double *s) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  double G0 = mul_rn(mul_rn(f.g, top), RS_PA2BAR);
  double rho0 = rho_of(f, 1, p_datum);
  double pot = sub_rn(p_datum, mul_rn(rho0, G0));
  double G = mul_rn(mul_rn(f.g, depth(top, dz, c / nxy)), RS_PA2BAR);
  double a = sub_rn(1.0, mul_rn(mul_rn(f.rho_ref[1], f.c_f[1]), G));
  double r = add_rn(pot, mul_rn(mul_rn(f.rho_ref[1], sub_rn(1.0, mul_rn(f.c_f[1], f.p_ref))), G));
  p[c] = div_rn(r, a);
  s[c] = sw0;
}
// initial wellbore pressure: a BHP well at its target, a rate (or shut)
// well 10 bar above (injector) or below (producer) the oil pressure of its
// first perforated cell
__global__ void k_init_pb(int nw, const int *wkind, const int *wctrl, const double *wtarget, const int *wpptr,
                          const int *pcell, const double *p, double *pb) {
  int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nw) return;
  double p0 = p[pcell[wpptr[w]]];
  pb[w] = wctrl[w] == SIM_BHP ? wtarget[w] : (wkind[w] == SIM_PROD ? sub_rn(p0, 10.0) : add_rn(p0, 10.0));
}

// ------------------------------------------------------------- host side --
static void s_props_assemble(sim_s *h) {
  cudaStream_t s = h->st;
  int n = h->n, nxy = h->nx * h->ny;
  sim_ls_s *ls = h->ls;
  rs_timed tm(ls, SIM_T_ASSEMBLE);
  k_props<<<grid_for(n, 256), 256, 0, s>>>(n, nxy, h->fl, h->top, h->dz, h->phi.p, h->p.p, h->s.p, h->props.p);
  k_assemble<<<grid_for(n, 128), 128, 0, s>>>(h->nx, h->ny, h->nz, h->fl, h->top, h->dz, h->dx * h->dy * h->dz / h->dt,
                                              h->phi.p, h->p.p, h->s.p, h->pb.p, h->acc0.p, h->props.p, h->tx.p,
                                              h->ty.p, h->tz.p, ls->rp.p, h->cpp.p, h->cpi.p, h->pwell.p, h->pwi.p,
                                              h->ppos_cw.p, h->wkind_d.p, h->wctrl_d.p, h->wzref_d.p, ls->val.p,
                                              ls->b.p);
  RS_LAUNCHED(2);
  if (h->nw) {
    k_wells<<<grid_for((size_t)h->nw * 32, 128), 128, 0, s>>>(
        n, h->nw, h->fl, h->top, h->dz, nxy, h->phi.p, h->p.p, h->s.p, h->pb.p, h->wpptr.p, h->pcell.p, h->pwi.p,
        h->ppos_wc.p, h->wdiag.p, h->wkind_d.p, h->wctrl_d.p, h->wtarget_d.p, h->wzref_d.p, ls->val.p, ls->b.p);
    RS_LAUNCHED(1);
  }
  k_key<<<grid_for(n, 256), 256, 0, s>>>(n, nxy, h->fl, h->top, h->dz, h->p.p, ls->key.p);
  RS_LAUNCHED(1);
  RS_CHECK_LAUNCH();
  ls->have_setup = false;
}

static double s_norm(sim_s *h) {
  cudaStream_t s = h->st;
  int nb = 120;
  h->red.ensure(nb + 1);
  double dvi = h->dt / (h->dx * h->dy * h->dz);
  k_norm_part<<<nb, 256, 0, s>>>(h->n, h->nw, dvi, h->fl, h->phi.p, h->ls->b.p, h->red.p);
  k_max_part<<<1, 32, 0, s>>>(nb, h->red.p, h->red.p + nb);
  RS_LAUNCHED(2);
  return d2h(h->red.p + nb, 1, s)[0];
}

static double s_forcing(int l, double bn, double rprev, double bprev) {
  if (l == 0) return 0.1;
  double eta = (bn - rprev) / bprev;
  return eta < 0.01 ? 0.01 : (eta > 0.1 ? 0.1 : eta);
}

static float ev_ms(sim_s *h) {
  float ms = 0;
  RS_CUDA(cudaEventRecord(h->e1, h->st));
  RS_CUDA(cudaEventSynchronize(h->e1));
  RS_CUDA(cudaEventElapsedTime(&ms, h->e0, h->e1));
  return ms;
}

// Algorithm 1 for one time step at h->dt.  0 = converged, 1 = iteration cap,
// 2 = non-finite value.
__global__ void k_f2d(size_t n, const float *a, double *b) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}

// x = sum_k beta_k c_k (k < m <= 3)
__global__ void k_lincomb(int nu, int m, const double *c0, const double *c1, const double *c2, double b0, double b1,
                          double b2, double *x) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nu) return;
  double v = b0 * c0[i];
  if (m > 1) v += b1 * c1[i];
  if (m > 2) v += b2 * c2[i];
  x[i] = v;
}

// Least squares over the span of m candidate guesses: G beta = r with
// G_ij = (A c_i).(A c_j), r_i = (A c_i).b; returns ||b - A x||^2 =
// ||b||^2 - r.beta.  Cholesky with candidates whose pivot is below 1e-12 of
// their diagonal dropped (beta = 0).
static double ls_fit(int m, const double G[3][3], const double r[3], double bb, double beta[3]) {
  double L[3][3] = {{0}}, z[3] = {0};
  bool keep[3] = {false, false, false};
  for (int i = 0; i < m; i++) {
    double d = G[i][i];
    for (int k = 0; k < i; k++) if (keep[k]) d -= L[i][k] * L[i][k];
    keep[i] = G[i][i] > 0.0 && d > 1e-12 * G[i][i];
    if (!keep[i]) continue;
    L[i][i] = std::sqrt(d);
    for (int j = i + 1; j < m; j++) {
      double v = G[j][i];
      for (int k = 0; k < i; k++) if (keep[k]) v -= L[j][k] * L[i][k];
      L[j][i] = v / L[i][i];
    }
  }
  for (int i = 0; i < m; i++) {
    if (!keep[i]) continue;
    double v = r[i];
    for (int k = 0; k < i; k++) if (keep[k]) v -= L[i][k] * z[k];
    z[i] = v / L[i][i];
  }
  for (int i = m - 1; i >= 0; i--) {
    beta[i] = 0.0;
    if (!keep[i]) continue;
    double v = z[i];
    for (int k = i + 1; k < m; k++) if (keep[k]) v -= L[k][i] * beta[k];
    beta[i] = v / L[i][i];
  }
  double rb = 0.0;
  for (int i = 0; i < m; i++) rb += r[i] * beta[i];
  return bb - rb;
}

// One linear solve of the Newton system on the device (after ls_setup).
// With a network attached, the initial guess is the least-squares
// combination, on the decoupled system, of the network's predicted update,
// taken as two candidates (its pressure part and its saturation part, each
// predicted with unit rms, so the fit sets both scales) and, at the first
// Newton iteration of a step, the previous step's first update.  The
// network's terms are kept only when they lower ||b - A x0|| below what the
// other candidate reaches without them (otherwise that plain guess, or zero,
// is the fallback); any such combination has ||b - A x0|| <= ||b||, the
// zero guess's.  Recording needs the rms of b, of the previous update and of
// the solved update (the target is the solved update over its rms).
static int s_solve(sim_s *h, double eta, double bn, int *its, double *rel) {
  sim_ls_s *ls = h->ls;
  cudaStream_t st = h->st;
  int nb = ls->nb, nu = 2 * nb;
  bool x0 = false;
  bool learn = h->ws || h->rec;
  bool first = h->first_pending;
  h->first_pending = false;
  rs_timed tm_ws(ls, h->ws ? SIM_T_WARMSTART : 0);
  if (learn) {
    ws_rms2(h->n, ls->b.p, h->wsc.p, st);
    if (!h->have_prev) RS_CUDA(cudaMemsetAsync(h->wsc.p + 4, 0, 2 * sizeof(double), st));
  }
  if (h->ws) {
    h->dws.ensure(2 * (size_t)nu); h->u.ensure(3 * (size_t)nu);
    {
      rs_timed tm_net(ls, SIM_T_NETWORK);
      ws_predict(h->ws, h->nx, h->ny, h->nz, nb, ls->b.p, h->kx.p, h->s.p, h->yprev.p, h->wsc.p, h->dws.p, st);
    }
    // candidates: the previous step's first update (if any), then the
    // network's pressure and saturation parts
    const double *c[3];
    int m = 0;
    if (first && h->have_first) c[m++] = h->yfirst.p;
    int id = m;
    c[m++] = h->dws.p;
    c[m++] = h->dws.p + nu;
    double *u[3];
    for (int k = 0; k < m; k++) { u[k] = h->u.p + (size_t)k * nu; ls_spmv64_untimed(ls, c[k], u[k]); }
    const double *xs[9], *ys[9];
    int q = 0;
    for (int i = 0; i < m; i++) for (int j = 0; j <= i; j++) { xs[q] = u[i]; ys[q] = u[j]; q++; }
    for (int i = 0; i < m; i++) { xs[q] = u[i]; ys[q] = ls->b.p; q++; }
    double dv[9];
    rs_dots(xs, ys, q, nu, dv, st);
    double G[3][3] = {{0}}, r[3] = {0};
    q = 0;
    for (int i = 0; i < m; i++) for (int j = 0; j <= i; j++) { G[i][j] = G[j][i] = dv[q]; q++; }
    for (int i = 0; i < m; i++) r[i] = dv[q++];
    double bb = bn * bn, beta_p[3] = {0, 0, 0}, beta_d[3] = {0, 0, 0};
    double res_p = id ? ls_fit(id, G, r, bb, beta_p) : bb;   // without the network's term
    double res_d = ls_fit(m, G, r, bb, beta_d);        // with it
    const double *beta = beta_p;
    double res = res_p;
    if (std::isfinite(res_d) && res_d < res_p * (1.0 - 1e-6)) { beta = beta_d; res = res_d; h->stats.ws_used++; }
    else h->stats.ws_fallback++;
    int mm = beta == beta_d ? m : id;
    if (std::isfinite(res) && res < bb) {
      k_lincomb<<<grid_for(nu, 256), 256, 0, st>>>(nu, mm, c[0], mm > 1 ? c[1] : c[0], mm > 2 ? c[2] : c[0],
                                                   beta[0], beta[1], beta[2], ls->y.p);
      RS_LAUNCHED(1);
      x0 = true;
      h->stats.ws_r0 += std::sqrt(std::max(res, 0.0)) / bn;
    } else {
      h->stats.ws_r0 += 1.0;
    }
  }
  tm_ws.stop();
  int rc = ls_solve(ls, eta, its, rel, x0);
  if (rc == 2) return rc;
  if (learn) ws_rms2(h->n, ls->y.p, h->wsc.p + 2, st);        // the solved update's scales
  if (h->rec)
    ws_record(h->rec, h->nx, h->ny, h->nz, ls->b.p, h->kx.p, h->s.p, h->yprev.p, h->wsc.p, ls->y.p, st);
  if (learn) {
    RS_CUDA(cudaMemcpyAsync(h->yprev.p, ls->y.p, nu * sizeof(double), cudaMemcpyDeviceToDevice, st));
    RS_CUDA(cudaMemcpyAsync(h->wsc.p + 4, h->wsc.p + 2, 2 * sizeof(double), cudaMemcpyDeviceToDevice, st));
    h->have_prev = true;
    if (first) {
      h->yfirst.ensure(nu);
      RS_CUDA(cudaMemcpyAsync(h->yfirst.p, ls->y.p, nu * sizeof(double), cudaMemcpyDeviceToDevice, st));
      h->have_first = true;
    }
  }
  return rc;
}

// ------------------------------------------------ well control switching --
// The host keeps each well's current control and target; the device copies
// are refreshed after every change.
static void s_controls_upload(sim_s *h) {
  if (!h->nw) return;
  RS_CUDA(cudaMemcpyAsync(h->wctrl_d.p, h->wctrl.data(), h->nw * sizeof(int), cudaMemcpyHostToDevice, h->st));
  RS_CUDA(cudaMemcpyAsync(h->wtarget_d.p, h->wtarget.data(), h->nw * sizeof(double), cudaMemcpyHostToDevice, h->st));
  RS_CUDA(cudaStreamSynchronize(h->st));      // the host vectors may change right after
}
static void s_controls_reset(sim_s *h) {
  for (int w = 0; w < h->nw; w++) { h->wctrl[w] = h->wctrl0[w]; h->wtarget[w] = h->wtarget0[w]; h->wswitched[w] = 0; }
  s_controls_upload(h);
}
static bool is_rate(int c) { return c == SIM_WRATE || c == SIM_ORATE || c == SIM_LRATE; }

// Rate to BHP, after a Newton update: a rate-controlled well with a BHP limit
// whose p_b has passed it (injector above its maximum, producer below its
// minimum) goes on BHP control at the limit and p_b is set to the limit.
static int s_limits_rate_to_bhp(sim_s *h) {
  if (!h->any_limit) return 0;
  std::vector<double> pb = d2h(h->pb.p, h->nw, h->st);
  int k = 0;
  for (int w = 0; w < h->nw; w++) {
    if (!is_rate(h->wctrl[w]) || !(h->wlimit[w] > 0.0)) continue;
    bool past = h->wkind[w] == SIM_INJ ? pb[w] > h->wlimit[w] : pb[w] < h->wlimit[w];
    if (!past) continue;
    h->wctrl[w] = SIM_BHP; h->wtarget[w] = h->wlimit[w]; h->wswitched[w] = 1;
    RS_CUDA(cudaMemcpyAsync(h->pb.p + w, &h->wlimit[w], sizeof(double), cudaMemcpyHostToDevice, h->st));
    k++;
  }
  if (k) s_controls_upload(h);
  return k;
}

static void s_props_assemble(sim_s *h);
// BHP back to rate, at the start of a time step (after the old accumulation
// is stored): a well held at its limit returns to its requested rate when,
// at the limit, its rate equation's residual is positive (it would deliver
// more than the target).
static void s_limits_bhp_to_rate(sim_s *h) {
  bool any = false;
  for (int w = 0; w < h->nw; w++)
    if (h->wswitched[w]) { h->wctrl[w] = h->wctrl0[w]; h->wtarget[w] = h->wtarget0[w]; any = true; }
  if (!any) return;
  s_controls_upload(h);
  s_props_assemble(h);
  std::vector<double> b = d2h(h->ls->b.p + 2 * (size_t)h->n, 2 * (size_t)h->nw, h->st);
  for (int w = 0; w < h->nw; w++) {
    if (!h->wswitched[w]) continue;
    if (-b[2 * w] > 0.0) h->wswitched[w] = 0;
    else { h->wctrl[w] = SIM_BHP; h->wtarget[w] = h->wlimit[w]; }
  }
  s_controls_upload(h);
}

static int s_newton(sim_s *h, int *iters) {
  RS_CUDA(cudaEventRecord(h->e0, h->st));
  s_props_assemble(h);
  double nr = s_norm(h);
  h->stats.ms_assemble += ev_ms(h);
  double bprev = 0, rprev = 0;
  for (int l = 0;; l++) {
    h->stats.last_norm = nr;
    if (!std::isfinite(nr)) { *iters = l; return 2; }
    if (nr <= h->o.newton_tol) { *iters = l; return 0; }
    if (l >= h->o.max_newton) { *iters = l; return 1; }
    RS_CUDA(cudaEventRecord(h->e0, h->st));
    ls_setup(h->ls);
    int nu = 2 * h->ls->nb;
    double bn = rs_norm2(h->ls->b.p, nu, h->st);
    h->stats.ms_setup += ev_ms(h);
    double eta = h->o.newton == SIM_NEWTON_INEXACT ? s_forcing(l, bn, rprev, bprev) : h->o.lin_tol;
    int its; double rel;
    RS_CUDA(cudaEventRecord(h->e0, h->st));
    int rc = s_solve(h, eta, bn, &its, &rel);
    h->stats.ms_solve += ev_ms(h);
    h->stats.linear_its += its; h->stats.linear_solves++;
    h->stats.last_its = its; h->stats.last_relres = rel;
    if (rc == 2) { *iters = l; return 2; }
    bprev = bn; rprev = rel * bn;
    k_update<<<grid_for(h->n + h->nw, 256), 256, 0, h->st>>>(h->n, h->nw, h->o.sat_chop, h->ls->y.p, h->p.p, h->s.p, h->pb.p);
    RS_LAUNCHED(1);
    h->stats.newton++;
    h->stats.switches += s_limits_rate_to_bhp(h);
    RS_CUDA(cudaEventRecord(h->e0, h->st));
    s_props_assemble(h);
    nr = s_norm(h);
    h->stats.ms_assemble += ev_ms(h);
  }
}

static void s_store_old(sim_s *h) {
  k_store_old<<<grid_for(h->n, 256), 256, 0, h->st>>>(h->n, h->nx * h->ny, h->fl, h->top, h->dz, h->phi.p, h->p.p,
                                                      h->s.p, h->acc0.p);
  RS_LAUNCHED(1);
}

// ------------------------------------------------------------------ ABI ---
#define ABI_BEGIN try {
#define ABI_END                                                       \
  }                                                                   \
  catch (const rs_error &e) { return e.code; }                        \
  catch (const std::bad_alloc &) { rs_set_error("host allocation failed"); return SIM_ERR_OOM; } \
  catch (...) { rs_set_error("unexpected exception"); return SIM_ERR_CUDA; }                       \
  return SIM_OK;

static void copy_in(dbuf<double> &d, const double *src, size_t m, cudaStream_t s) {
  d.alloc(m);
  if (m) RS_CUDA(cudaMemcpyAsync(d.p, src, m * sizeof(double), cudaMemcpyDefault, s));
}

// host check of a well control (eqs. 11-14, shut): NULL when valid
static const char *well_control_invalid(int kind, int control, double target, double limit) {
  if (kind != SIM_INJ && kind != SIM_PROD) return "bad kind";
  if (control < SIM_BHP || control > SIM_SHUT) return "unknown control";
  if ((control == SIM_ORATE || control == SIM_LRATE) && kind != SIM_PROD)
    return "oil- and liquid-rate controls need a producer (injectors inject water)";
  if (control != SIM_SHUT && !(target > 0 && target < HUGE_VAL)) return "target must be finite and positive";
  if (!(limit >= 0 && limit < HUGE_VAL)) return "BHP limit must be finite and >= 0 (0 = none)";
  return nullptr;
}

extern "C" sim_status sim_create(sim_t *out, const sim_grid *g, const sim_rock *r, const sim_fluid *f,
                                 const sim_well *wells, int n_wells, const sim_options *o) {
  ABI_BEGIN
  if (!out || !g || !r || !f || !o || (n_wells > 0 && !wells) || n_wells < 0) RS_FAIL(SIM_ERR_ARG, "sim_create: NULL argument");
  *out = nullptr;
  if (g->nx < 1 || g->ny < 1 || g->nz < 1 || !(g->dx > 0) || !(g->dy > 0) || !(g->dz > 0))
    RS_FAIL(SIM_ERR_ARG, "sim_create: bad grid");
  // counts inside the setup are 32-bit: the largest, the Galerkin products of
  // one AMG level, reach ~30 per cell on the channelised 1M-cell case, so
  // 2^31 would be crossed near 70M cells; the limit keeps a margin below that
  if ((long long)g->nx * g->ny * g->nz > 50000000LL)
    RS_FAIL(SIM_ERR_ARG, "sim_create: grid too large (at most 50M cells: 32-bit counts in the solver setup)");
  if (!r->kx || !r->ky || !r->kz || !r->phi) RS_FAIL(SIM_ERR_ARG, "sim_create: NULL rock array");
  if (const char *e = rs_opts_invalid(o)) RS_FAIL(SIM_ERR_ARG, "sim_create: %s", e);
  if (!(o->dt > 0.0 && o->dt < HUGE_VAL)) RS_FAIL(SIM_ERR_ARG, "sim_create: dt must be finite and > 0");
  if (f->pc_n < 0 || f->pc_n > PC_MAX) RS_FAIL(SIM_ERR_ARG, "sim_create: a capillary pressure table holds 0 to %d points", PC_MAX);
  if (f->pc_n > 0) {
    if (!f->pc_sw || !f->pc_val) RS_FAIL(SIM_ERR_ARG, "sim_create: NULL capillary pressure table");
    for (int k = 0; k < f->pc_n; k++) {
      if (!std::isfinite(f->pc_sw[k]) || !std::isfinite(f->pc_val[k]))
        RS_FAIL(SIM_ERR_ARG, "sim_create: capillary pressure table entry %d is not finite", k);
      if (k > 0 && !(f->pc_sw[k] > f->pc_sw[k - 1]))
        RS_FAIL(SIM_ERR_ARG, "sim_create: capillary pressure table saturations must increase");
    }
  }
  for (int w = 0; w < n_wells; w++) {           // host-side well checks before any device work
    const sim_well &W = wells[w];
    if (const char *e = well_control_invalid(W.kind, W.control, W.target, W.bhp_limit)) RS_FAIL(SIM_ERR_ARG, "well %d: %s", w, e);
    if (W.n_perf < 1 || !W.perf_cell) RS_FAIL(SIM_ERR_ARG, "well %d: no perforations", w);
    for (int q = 0; q < W.n_perf; q++)
      if (W.perf_cell[q] < 0 || W.perf_cell[q] >= g->nx * g->ny * g->nz)
        RS_FAIL(SIM_ERR_ARG, "well %d: perforation outside the grid", w);
  }
  sim_s *h = new sim_s();
  std::unique_ptr<sim_s> guard(h);
  h->nx = g->nx; h->ny = g->ny; h->nz = g->nz; h->n = g->nx * g->ny * g->nz; h->nw = n_wells;
  h->dx = g->dx; h->dy = g->dy; h->dz = g->dz; h->top = g->top_depth;
  {
    fluid_c &F = h->fl;
    memset(&F, 0, sizeof(F));
    for (int a = 0; a < 2; a++) { F.rho_ref[a] = f->rho_ref[a]; F.c_f[a] = f->c_f[a]; F.mu_ref[a] = f->mu_ref[a]; F.c_mu[a] = f->c_mu[a]; }
    F.p_ref = f->p_ref; F.c_r = f->c_r; F.swc = f->swc; F.sor = f->sor; F.nw = f->nw; F.no = f->no;
    F.krw_max = f->krw_max; F.kro_max = f->kro_max; F.g = f->g;
    F.span = (1.0 - F.swc) - F.sor;                   // the same IEEE operations as on the device
    F.inv_span = 1.0 / F.span;
    F.pc_n = f->pc_n;
    for (int k = 0; k < f->pc_n; k++) { F.pc_sw[k] = f->pc_sw[k]; F.pc_val[k] = f->pc_val[k]; }
  }
  h->o = rs_opts_from(o);
  h->st = (cudaStream_t)o->cuda_stream;
  h->dt = h->o.dt;
  memset(&h->stats, 0, sizeof(h->stats));
  int n = h->n, nw = n_wells;
  cudaStream_t s = h->st;
  copy_in(h->kx, r->kx, n, s); copy_in(h->ky, r->ky, n, s); copy_in(h->kz, r->kz, n, s); copy_in(h->phi, r->phi, n, s);
  // wells, perforations and the block pattern
  h->pptr.assign(nw + 1, 0);
  std::vector<int> pcell, pwell;
  std::vector<double> pwi, rw(nw), skin(nw);
  std::vector<std::vector<int>> cellwells(n);
  for (int w = 0; w < nw; w++) {
    const sim_well &W = wells[w];
    if (const char *e = well_control_invalid(W.kind, W.control, W.target, W.bhp_limit)) RS_FAIL(SIM_ERR_ARG, "well %d: %s", w, e);
    if (W.n_perf < 1 || !W.perf_cell) RS_FAIL(SIM_ERR_ARG, "well %d: no perforations", w);
    h->wkind.push_back(W.kind); h->wctrl.push_back(W.control);
    h->wtarget.push_back(W.target); h->wzref.push_back(W.z_ref);
    h->wctrl0.push_back(W.control); h->wtarget0.push_back(W.target); h->wlimit.push_back(W.bhp_limit);
    h->wswitched.push_back(0);
    if (W.bhp_limit > 0.0) h->any_limit = true;
    rw[w] = W.r_w; skin[w] = W.skin;
    for (int q = 0; q < W.n_perf; q++) {
      int c = W.perf_cell[q];
      if (c < 0 || c >= n) RS_FAIL(SIM_ERR_ARG, "well %d: perforation outside the grid", w);
      for (int w2 : cellwells[c]) if (w2 == w) RS_FAIL(SIM_ERR_ARG, "well %d perforates cell %d twice", w, c);
      cellwells[c].push_back(w);
      pcell.push_back(c); pwell.push_back(w);
      pwi.push_back(W.wi ? W.wi[q] : -1.0);
    }
    h->pptr[w + 1] = (int)pcell.size();
  }
  h->np_ = (int)pcell.size();
  int nb = n + nw, nx = h->nx, ny = h->ny, nz = h->nz, nxy = nx * ny;
  std::vector<int> rp(nb + 1, 0), ci;
  ci.reserve((size_t)7 * n + 2 * h->np_ + nw);
  for (int c = 0; c < n; c++) {
    int i = c % nx, j = (c / nx) % ny, k = c / nxy;
    if (k > 0) ci.push_back(c - nxy);
    if (j > 0) ci.push_back(c - nx);
    if (i > 0) ci.push_back(c - 1);
    ci.push_back(c);
    if (i + 1 < nx) ci.push_back(c + 1);
    if (j + 1 < ny) ci.push_back(c + nx);
    if (k + 1 < nz) ci.push_back(c + nxy);
    std::vector<int> ws = cellwells[c];
    std::sort(ws.begin(), ws.end());
    for (int w : ws) ci.push_back(n + w);
    rp[c + 1] = (int)ci.size();
  }
  for (int w = 0; w < nw; w++) {
    std::vector<int> cs(pcell.begin() + h->pptr[w], pcell.begin() + h->pptr[w + 1]);
    std::sort(cs.begin(), cs.end());
    for (int c : cs) ci.push_back(c);
    ci.push_back(n + w);
    rp[n + w + 1] = (int)ci.size();
  }
  auto find = [&](int row, int col) {
    for (int q = rp[row]; q < rp[row + 1]; q++) if (ci[q] == col) return q;
    return -1;
  };
  std::vector<int> ppos_cw(h->np_), ppos_wc(h->np_), wdiag(nw), cpp(n + 1, 0), cpi(h->np_), wc0(nw);
  for (int q = 0; q < h->np_; q++) {
    ppos_cw[q] = find(pcell[q], n + pwell[q]);
    ppos_wc[q] = find(n + pwell[q], pcell[q]);
    cpp[pcell[q] + 1]++;
  }
  for (int c = 0; c < n; c++) cpp[c + 1] += cpp[c];
  {
    std::vector<int> fill(n, 0);
    for (int q = 0; q < h->np_; q++) cpi[cpp[pcell[q]] + fill[pcell[q]]++] = q;
  }
  for (int w = 0; w < nw; w++) { wdiag[w] = find(n + w, n + w); wc0[w] = pcell[h->pptr[w]]; }
  h2d(h->pcell, pcell, s); h2d(h->pwell, pwell, s); h2d(h->pwi, pwi, s);
  h2d(h->ppos_cw, ppos_cw, s); h2d(h->ppos_wc, ppos_wc, s); h2d(h->cpp, cpp, s); h2d(h->cpi, cpi, s);
  h2d(h->wpptr, h->pptr, s); h2d(h->wdiag, wdiag, s);
  h2d(h->wkind_d, h->wkind, s); h2d(h->wctrl_d, h->wctrl, s); h2d(h->wtarget_d, h->wtarget, s); h2d(h->wzref_d, h->wzref, s);
  dbuf<double> rw_d, skin_d;
  h2d(rw_d, rw, s); h2d(skin_d, skin, s);
  h->tx.alloc(n); h->ty.alloc(n); h->tz.alloc(n);
  k_trans<<<grid_for(n, 256), 256, 0, s>>>(nx, ny, nz, h->dx, h->dy, h->dz, h->kx.p, h->ky.p, h->kz.p, h->tx.p, h->ty.p, h->tz.p);
  RS_LAUNCHED(1);
  if (h->np_) {
    k_peaceman<<<grid_for(h->np_, 128), 128, 0, s>>>(h->np_, h->dx, h->dy, h->dz, h->pcell.p, h->pwell.p, rw_d.p, skin_d.p,
                                                     h->kx.p, h->ky.p, h->pwi.p);
    RS_LAUNCHED(1);
  }
  h->p.alloc(n); h->s.alloc(n); h->pb.alloc(nw ? nw : 1); h->acc0.alloc(2 * (size_t)n);
  h->props.alloc(15 * (size_t)n); h->p0.alloc(n); h->s0.alloc(n); h->pb0.alloc(nw ? nw : 1);
  rs_fill_d(h->p.p, h->fl.p_ref, n, s); rs_fill_d(h->s.p, h->fl.swc, n, s); rs_fill_d(h->pb.p, 0.0, nw ? nw : 1, s);
  h->ls = new sim_ls_s();
  ls_init(h->ls, nx, ny, nz, nw, rp.data(), ci.data(), wc0.data(), h->o, s);
  RS_CUDA(cudaEventCreate(&h->e0)); RS_CUDA(cudaEventCreate(&h->e1));
  s_store_old(h);
  RS_CUDA(cudaStreamSynchronize(s));
  *out = guard.release();
  ABI_END
}

extern "C" void sim_destroy(sim_t h) { if (h) { cudaStreamSynchronize(h->st); delete h; } }

extern "C" sim_status sim_init_hydrostatic(sim_t h, double p_datum, double sw0) {
  ABI_BEGIN
  if (!h) RS_FAIL(SIM_ERR_ARG, "NULL handle");
  int nxy = h->nx * h->ny;
  k_hydrostatic<<<grid_for(h->n, 256), 256, 0, h->st>>>(h->n, nxy, h->fl, h->top, h->dz, p_datum, sw0, h->p.p, h->s.p);
  RS_LAUNCHED(1);
  if (h->nw) {
    s_controls_reset(h);
    k_init_pb<<<grid_for(h->nw, 32), 32, 0, h->st>>>(h->nw, h->wkind_d.p, h->wctrl_d.p, h->wtarget_d.p, h->wpptr.p,
                                                     h->pcell.p, h->p.p, h->pb.p);
    RS_LAUNCHED(1);
  }
  h->t = 0.0;
  h->have_prev = h->have_first = false;
  s_store_old(h);
  RS_CHECK_LAUNCH();
  RS_CUDA(cudaStreamSynchronize(h->st));
  ABI_END
}

extern "C" sim_status sim_set_state(sim_t h, const double *p, const double *sw, const double *pb, double t) {
  ABI_BEGIN
  if (!h || !p || !sw || (h->nw && !pb)) RS_FAIL(SIM_ERR_ARG, "sim_set_state: NULL argument");
  RS_CUDA(cudaMemcpyAsync(h->p.p, p, h->n * sizeof(double), cudaMemcpyDefault, h->st));
  RS_CUDA(cudaMemcpyAsync(h->s.p, sw, h->n * sizeof(double), cudaMemcpyDefault, h->st));
  if (h->nw) RS_CUDA(cudaMemcpyAsync(h->pb.p, pb, h->nw * sizeof(double), cudaMemcpyDefault, h->st));
  h->t = t;
  RS_CUDA(cudaStreamSynchronize(h->st));
  ABI_END
}

extern "C" sim_status sim_get_state(sim_t h, double *p, double *sw, double *pb, double *t) {
  ABI_BEGIN
  if (!h) RS_FAIL(SIM_ERR_ARG, "NULL handle");
  if (p) RS_CUDA(cudaMemcpyAsync(p, h->p.p, h->n * sizeof(double), cudaMemcpyDefault, h->st));
  if (sw) RS_CUDA(cudaMemcpyAsync(sw, h->s.p, h->n * sizeof(double), cudaMemcpyDefault, h->st));
  if (pb && h->nw) RS_CUDA(cudaMemcpyAsync(pb, h->pb.p, h->nw * sizeof(double), cudaMemcpyDefault, h->st));
  if (t) *t = h->t;
  RS_CUDA(cudaStreamSynchronize(h->st));
  ABI_END
}

extern "C" sim_status sim_begin_step(sim_t h, double dt) {
  ABI_BEGIN
  if (!h || !(dt > 0)) RS_FAIL(SIM_ERR_ARG, "sim_begin_step: bad argument");
  h->dt = dt;
  h->first_pending = true;
  s_store_old(h);
  RS_CHECK_LAUNCH();
  ABI_END
}

extern "C" sim_status sim_assemble(sim_t h, double *scaled_norm) {
  ABI_BEGIN
  if (!h) RS_FAIL(SIM_ERR_ARG, "NULL handle");
  s_props_assemble(h);
  double nr = s_norm(h);
  if (scaled_norm) *scaled_norm = nr;
  ABI_END
}

extern "C" sim_status sim_linear_solve(sim_t h, double tol, int *iters, double *relres) {
  ABI_BEGIN
  if (!(tol >= 0.0 && tol < HUGE_VAL)) RS_FAIL(SIM_ERR_ARG, "sim_linear_solve: tol must be finite and >= 0");
  if (!h) RS_FAIL(SIM_ERR_ARG, "NULL handle");
  ls_setup(h->ls);
  int its; double rel;
  double bn = rs_norm2(h->ls->b.p, 2 * h->ls->nb, h->st);
  int rc = s_solve(h, tol, bn, &its, &rel);
  if (iters) *iters = its;
  if (relres) *relres = rel;
  if (rc == 2) RS_FAIL(SIM_ERR_NAN, "linear solve produced a non-finite value");
  ABI_END
}

extern "C" sim_status sim_newton_step(sim_t h, int *converged, sim_stats *st) {
  ABI_BEGIN
  if (!h) RS_FAIL(SIM_ERR_ARG, "NULL handle");
  s_props_assemble(h);
  double nr = s_norm(h);
  h->stats.last_norm = nr;
  if (!std::isfinite(nr)) RS_FAIL(SIM_ERR_NAN, "non-finite residual");
  if (converged) *converged = nr <= h->o.newton_tol;
  if (nr > h->o.newton_tol) {
    ls_setup(h->ls);
    int its; double rel;
    double bn = rs_norm2(h->ls->b.p, 2 * h->ls->nb, h->st);
    int rc = s_solve(h, h->o.lin_tol, bn, &its, &rel);
    h->stats.linear_its += its; h->stats.linear_solves++; h->stats.last_its = its; h->stats.last_relres = rel;
    if (rc == 2) RS_FAIL(SIM_ERR_NAN, "linear solve produced a non-finite value");
    k_update<<<grid_for(h->n + h->nw, 256), 256, 0, h->st>>>(h->n, h->nw, h->o.sat_chop, h->ls->y.p, h->p.p, h->s.p, h->pb.p);
    RS_LAUNCHED(1);
    h->stats.newton++;
    h->stats.switches += s_limits_rate_to_bhp(h);
  }
  if (st) *st = h->stats;
  ABI_END
}

extern "C" sim_status sim_advance(sim_t h, int n_steps, sim_stats *st) {
  ABI_BEGIN
  if (!h || n_steps < 0) RS_FAIL(SIM_ERR_ARG, "sim_advance: bad argument");
  cudaStream_t s = h->st;
  int n = h->n, nw = h->nw;
  sim_status bad = SIM_OK;
  std::vector<int> c0(nw), w0(nw);
  std::vector<double> t0(nw);
  for (int stp = 0; stp < n_steps && bad == SIM_OK; stp++) {
    double rem = h->o.dt, hh = h->o.dt;
    int cuts = 0;
    while (rem > 0.0) {
      double dt = hh < rem ? hh : rem;
      RS_CUDA(cudaMemcpyAsync(h->p0.p, h->p.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      RS_CUDA(cudaMemcpyAsync(h->s0.p, h->s.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      if (nw) RS_CUDA(cudaMemcpyAsync(h->pb0.p, h->pb.p, nw * sizeof(double), cudaMemcpyDeviceToDevice, s));
      s_store_old(h);
      h->dt = dt;
      h->first_pending = true;
      s_limits_bhp_to_rate(h);
      c0 = h->wctrl; t0 = h->wtarget; w0 = h->wswitched;
      int its;
      int r = s_newton(h, &its);
      h->stats.last_newton = its;
      if (r == 0) { h->t += dt; rem -= dt; h->stats.steps++; continue; }
      RS_CUDA(cudaMemcpyAsync(h->p.p, h->p0.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      RS_CUDA(cudaMemcpyAsync(h->s.p, h->s0.p, n * sizeof(double), cudaMemcpyDeviceToDevice, s));
      if (nw) RS_CUDA(cudaMemcpyAsync(h->pb.p, h->pb0.p, nw * sizeof(double), cudaMemcpyDeviceToDevice, s));
      if (h->wctrl != c0 || h->wtarget != t0 || h->wswitched != w0) {
        h->wctrl = c0; h->wtarget = t0; h->wswitched = w0;
        s_controls_upload(h);
      }
      h->stats.cuts++; cuts++;
      if (cuts > h->o.max_cuts) { bad = r == 2 ? SIM_ERR_NAN : SIM_ERR_NOT_CONVERGED; break; }
      hh = 0.5 * hh;
    }
  }
  h->stats.t = h->t;
  if (st) *st = h->stats;
  RS_CUDA(cudaStreamSynchronize(s));
  if (bad != SIM_OK) RS_FAIL(bad, "time step did not converge after %d cuts", h->o.max_cuts);
  ABI_END
}

extern "C" sim_status sim_get_stats(sim_t h, sim_stats *st) {
  ABI_BEGIN
  if (!h || !st) RS_FAIL(SIM_ERR_ARG, "NULL argument");
  h->stats.t = h->t;
  *st = h->stats;
  ABI_END
}

extern "C" sim_status sim_set_well(sim_t h, int w, int control, double target, double bhp_limit) {
  ABI_BEGIN
  if (!h) RS_FAIL(SIM_ERR_ARG, "NULL handle");
  if (w < 0 || w >= h->nw) RS_FAIL(SIM_ERR_ARG, "sim_set_well: no well %d", w);
  if (const char *e = well_control_invalid(h->wkind[w], control, target, bhp_limit))
    RS_FAIL(SIM_ERR_ARG, "sim_set_well: well %d: %s", w, e);
  h->wctrl[w] = h->wctrl0[w] = control;
  h->wtarget[w] = h->wtarget0[w] = target;
  h->wlimit[w] = bhp_limit; h->wswitched[w] = 0;
  h->any_limit = false;
  for (int k = 0; k < h->nw; k++) if (h->wlimit[k] > 0.0) h->any_limit = true;
  s_controls_upload(h);
  double pbw = 0.0;
  if (control == SIM_BHP) pbw = target;
  else if (control != SIM_SHUT) {
    double p0 = d2h(h->p.p + d2h(h->pcell.p + h->pptr[w], 1, h->st)[0], 1, h->st)[0];
    pbw = h->wkind[w] == SIM_PROD ? p0 - 10.0 : p0 + 10.0;
  }
  if (control != SIM_SHUT) RS_CUDA(cudaMemcpyAsync(h->pb.p + w, &pbw, sizeof(double), cudaMemcpyHostToDevice, h->st));
  RS_CUDA(cudaStreamSynchronize(h->st));
  ABI_END
}

extern "C" sim_status sim_get_well_controls(sim_t h, int *control, double *target) {
  ABI_BEGIN
  if (!h) RS_FAIL(SIM_ERR_ARG, "NULL handle");
  for (int w = 0; w < h->nw; w++) {
    if (control) control[w] = h->wctrl[w];
    if (target) target[w] = h->wtarget[w];
  }
  ABI_END
}

void sim_dims(sim_t h, int *n, int *n_wells) { *n = h->n; *n_wells = h->nw; }
void sim_put_stats(sim_t h, const sim_stats *st) { h->stats = *st; }
// warm-start history (previous update and scales): save into / restore from
// caller-owned device buffers of 2 nb and 8 doubles
int sim_history(sim_t h, double *y, double *sc, int have, bool save) {
  size_t nu = 2 * (size_t)h->ls->nb;
  if (save) {
    if (h->have_prev) {
      RS_CUDA(cudaMemcpyAsync(y, h->yprev.p, nu * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
      RS_CUDA(cudaMemcpyAsync(sc, h->wsc.p, 8 * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    }
    if (h->have_first) RS_CUDA(cudaMemcpyAsync(y + nu, h->yfirst.p, nu * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    RS_CUDA(cudaStreamSynchronize(h->st));
    return (h->have_prev ? 1 : 0) | (h->have_first ? 2 : 0);
  }
  if (have & 1) {
    RS_CUDA(cudaMemcpyAsync(h->yprev.p, y, nu * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
    RS_CUDA(cudaMemcpyAsync(h->wsc.p, sc, 8 * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  }
  if (have & 2) {
    h->yfirst.ensure(nu);
    RS_CUDA(cudaMemcpyAsync(h->yfirst.p, y + nu, nu * sizeof(double), cudaMemcpyDeviceToDevice, h->st));
  }
  RS_CUDA(cudaStreamSynchronize(h->st));
  h->have_prev = (have & 1) != 0;
  h->have_first = (have & 2) != 0;
  return have;
}

extern "C" sim_status sim_ws_attach(sim_t h, sim_ws_t ws) {
  ABI_BEGIN
  if (!h) RS_FAIL(SIM_ERR_ARG, "NULL handle");
  if (ws) { h->yprev.ensure(2 * (size_t)h->ls->nb); h->wsc.ensure(8); }
  h->ws = ws;
  ABI_END
}

extern "C" sim_status sim_ws_record(sim_t h, sim_ws_t ws) {
  ABI_BEGIN
  if (!h) RS_FAIL(SIM_ERR_ARG, "NULL handle");
  if (ws) { h->yprev.ensure(2 * (size_t)h->ls->nb); h->wsc.ensure(8); }
  h->rec = ws;
  ABI_END
}

extern "C" sim_ls_t sim_linear_system(sim_t h) { return h ? h->ls : nullptr; }

// ---------------------------------------------------- linear-system ABI --
extern "C" sim_status sim_ls_create(sim_ls_t *out, int nx, int ny, int nz, int n_wells, const int *rowptr,
                                    const int *cols, const int *well_cell0, const sim_options *o) {
  ABI_BEGIN
  if (!out || !rowptr || !cols || !o || nx < 1 || ny < 1 || nz < 1 || n_wells < 0 || (n_wells && !well_cell0))
    RS_FAIL(SIM_ERR_ARG, "sim_ls_create: bad argument");
  *out = nullptr;
  if (const char *e = rs_opts_invalid(o)) RS_FAIL(SIM_ERR_ARG, "sim_ls_create: %s", e);
  if ((long long)nx * ny * nz > 50000000LL)                 // as in sim_create
    RS_FAIL(SIM_ERR_ARG, "sim_ls_create: grid too large (at most 50M cells: 32-bit counts in the solver setup)");
  std::unique_ptr<sim_ls_s> ls(new sim_ls_s());
  ls_init(ls.get(), nx, ny, nz, n_wells, rowptr, cols, well_cell0, rs_opts_from(o), (cudaStream_t)o->cuda_stream);
  *out = ls.release();
  ABI_END
}

extern "C" void sim_ls_destroy(sim_ls_t ls) { if (ls) { cudaStreamSynchronize(ls->st); delete ls; } }

extern "C" sim_status sim_ls_set(sim_ls_t ls, const double *vals, const double *b, const double *key) {
  ABI_BEGIN
  if (!ls || !vals || !b || !key) RS_FAIL(SIM_ERR_ARG, "sim_ls_set: NULL argument");
  RS_CUDA(cudaMemcpyAsync(ls->val.p, vals, 4 * (size_t)ls->nnzb * sizeof(double), cudaMemcpyDefault, ls->st));
  RS_CUDA(cudaMemcpyAsync(ls->b.p, b, 2 * (size_t)ls->nb * sizeof(double), cudaMemcpyDefault, ls->st));
  RS_CUDA(cudaMemcpyAsync(ls->key.p, key, (size_t)ls->n * sizeof(double), cudaMemcpyDefault, ls->st));
  RS_CUDA(cudaStreamSynchronize(ls->st));
  ls->have_setup = false;
  ABI_END
}

extern "C" sim_status sim_ls_setup(sim_ls_t ls) {
  ABI_BEGIN
  if (!ls) RS_FAIL(SIM_ERR_ARG, "NULL handle");
  ls_setup(ls);
  RS_CUDA(cudaStreamSynchronize(ls->st));
  ABI_END
}

extern "C" sim_status sim_ls_solve(sim_ls_t ls, double tol, double *y, int *iters, double *relres) {
  ABI_BEGIN
  if (!(tol >= 0.0 && tol < HUGE_VAL)) RS_FAIL(SIM_ERR_ARG, "sim_ls_solve: tol must be finite and >= 0");
  if (!ls) RS_FAIL(SIM_ERR_ARG, "NULL handle");
  if (!ls->have_setup) RS_FAIL(SIM_ERR_STATE, "sim_ls_solve before sim_ls_setup");
  int its; double rel;
  int rc = ls_solve(ls, tol, &its, &rel);
  if (iters) *iters = its;
  if (relres) *relres = rel;
  if (y) RS_CUDA(cudaMemcpyAsync(y, ls->y.p, 2 * (size_t)ls->nb * sizeof(double), cudaMemcpyDefault, ls->st));
  RS_CUDA(cudaStreamSynchronize(ls->st));
  if (rc == 2) RS_FAIL(SIM_ERR_NAN, "non-finite value in the linear solve");
  ABI_END
}

__global__ void k_cast_f2d(size_t m, const float *a, double *b) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < m) b[i] = a[i];
}
__global__ void k_cast_d2f_(size_t m, const double *a, float *b) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (i < m) b[i] = (float)a[i];
}

extern "C" sim_status sim_ls_apply(sim_ls_t ls, int op, const double *x, double *y) {
  ABI_BEGIN
  if (!ls || !x || !y) RS_FAIL(SIM_ERR_ARG, "sim_ls_apply: NULL argument");
  if (op != SIM_OP_SPMV && !ls->have_setup) RS_FAIL(SIM_ERR_STATE, "sim_ls_apply before sim_ls_setup");
  cudaStream_t s = ls->st;
  size_t nu = 2 * (size_t)ls->nb, m = op == SIM_OP_VCYCLE ? (size_t)ls->n : nu;
  dbuf<double> xin, yout;
  xin.alloc(m); yout.alloc(m);
  RS_CUDA(cudaMemcpyAsync(xin.p, x, m * sizeof(double), cudaMemcpyDefault, s));
  bool mixed = ls->o.precision != SIM_PREC_FP64;
  if (op == SIM_OP_SPMV) ls_spmv64(ls, xin.p, yout.p);
  else if (op == SIM_OP_RAS) {
    if (mixed) {
      dbuf<float> a, b2; a.alloc(nu); b2.alloc(nu);
      k_cast_d2f_<<<grid_for(nu, 256), 256, 0, s>>>(nu, xin.p, a.p);
      ls_ras_apply<float, float>(ls, a.p, b2.p, false);
      k_cast_f2d<<<grid_for(nu, 256), 256, 0, s>>>(nu, b2.p, yout.p);
      RS_LAUNCHED(2);
      RS_CUDA(cudaStreamSynchronize(s));
    } else ls_ras_apply<double, double>(ls, xin.p, yout.p, false);
  } else if (op == SIM_OP_VCYCLE) {
    amg_level &L0 = ls->amg.lev[0];
    if (mixed) {
      k_cast_d2f_<<<grid_for(m, 256), 256, 0, s>>>(m, xin.p, L0.f32.p);
      amg_vcycle<float>(ls->amg, 0, s);
      k_cast_f2d<<<grid_for(m, 256), 256, 0, s>>>(m, L0.x32.p, yout.p);
      RS_LAUNCHED(2);
    } else {
      RS_CUDA(cudaMemcpyAsync(L0.f.p, xin.p, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
      amg_vcycle<double>(ls->amg, 0, s);
      RS_CUDA(cudaMemcpyAsync(yout.p, L0.x.p, m * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
  } else if (op == SIM_OP_CPR) {
    if (mixed) {
      dbuf<float> z; z.alloc(nu);
      ls_cpr(ls, xin.p, nullptr, z.p);
      k_cast_f2d<<<grid_for(nu, 256), 256, 0, s>>>(nu, z.p, yout.p);
      RS_LAUNCHED(1);
      RS_CUDA(cudaStreamSynchronize(s));
    } else ls_cpr(ls, xin.p, yout.p, nullptr);
  } else RS_FAIL(SIM_ERR_ARG, "sim_ls_apply: unknown operator %d", op);
  RS_CHECK_LAUNCH();
  RS_CUDA(cudaMemcpyAsync(y, yout.p, m * sizeof(double), cudaMemcpyDefault, s));
  RS_CUDA(cudaStreamSynchronize(s));
  ABI_END
}

extern "C" sim_status sim_ls_residual_norm(sim_ls_t ls, const double *x, double *norm) {
  ABI_BEGIN
  if (!ls || !x || !norm) RS_FAIL(SIM_ERR_ARG, "sim_ls_residual_norm: NULL argument");
  size_t nu = 2 * (size_t)ls->nb;
  dbuf<double> xd;
  xd.alloc(nu);
  RS_CUDA(cudaMemcpyAsync(xd.p, x, nu * sizeof(double), cudaMemcpyDefault, ls->st));
  *norm = ls_residual_norm(ls, xd.p);
  ABI_END
}

template <class T>
static void put(void *dst, size_t bytes, size_t *needed, const T *src_dev, size_t count, cudaStream_t s) {
  size_t need = count * sizeof(T);
  if (needed) *needed = need;
  if (!dst) return;
  if (bytes < need) RS_FAIL(SIM_ERR_ARG, "sim_ls_export: buffer of %zu bytes, %zu needed", bytes, need);
  if (count) RS_CUDA(cudaMemcpyAsync(dst, src_dev, need, cudaMemcpyDefault, s));
  RS_CUDA(cudaStreamSynchronize(s));
}
static void put_host(void *dst, size_t bytes, size_t *needed, const void *src, size_t need) {
  if (needed) *needed = need;
  if (!dst) return;
  if (bytes < need) RS_FAIL(SIM_ERR_ARG, "sim_ls_export: buffer of %zu bytes, %zu needed", bytes, need);
  memcpy(dst, src, need);
}

extern "C" sim_status sim_ls_export(sim_ls_t ls, int what, int index, void *dst, size_t bytes, size_t *needed) {
  ABI_BEGIN
  if (!ls) RS_FAIL(SIM_ERR_ARG, "NULL handle");
  cudaStream_t s = ls->st;
  RS_CUDA(cudaStreamSynchronize(s));
  amg_hier &H = ls->amg;
  auto lev = [&](int l) -> amg_level & {
    if (l < 0 || l >= H.nlev) RS_FAIL(SIM_ERR_ARG, "sim_ls_export: no AMG level %d", l);
    return H.lev[l];
  };
  switch (what) {
    case SIM_X_VALS: put(dst, bytes, needed, ls->val.p, 4 * (size_t)ls->nnzb, s); break;
    case SIM_X_RHS: put(dst, bytes, needed, ls->b.p, 2 * (size_t)ls->nb, s); break;
    case SIM_X_SOLUTION: put(dst, bytes, needed, ls->y.p, 2 * (size_t)ls->nb, s); break;
    case SIM_X_ROWPTR: put_host(dst, bytes, needed, ls->h_rp.data(), ls->h_rp.size() * sizeof(int)); break;
    case SIM_X_COLS: put_host(dst, bytes, needed, ls->h_ci.data(), ls->h_ci.size() * sizeof(int)); break;
    case SIM_X_KEY: put(dst, bytes, needed, ls->key.p, (size_t)ls->n, s); break;
    case SIM_X_AMG_SIZES: {
      if (index < 0) { int v = H.nlev; put_host(dst, bytes, needed, &v, sizeof(int)); break; }
      amg_level &L = lev(index);
      bool last = index == H.nlev - 1;
      int v[6] = {L.A.n, L.A.nnz, last ? 0 : L.P.nnz, last ? 0 : L.nc, L.rounds, H.coarse_dense};
      put_host(dst, bytes, needed, v, sizeof(v));
      break;
    }
    case SIM_X_AMG_RP: { amg_level &L = lev(index); put(dst, bytes, needed, L.A.rp.p, L.A.n + 1, s); break; }
    case SIM_X_AMG_CI: { amg_level &L = lev(index); put(dst, bytes, needed, L.A.ci.p, L.A.nnz, s); break; }
    case SIM_X_AMG_V: { amg_level &L = lev(index); put(dst, bytes, needed, L.A.v.p, L.A.nnz, s); break; }
    case SIM_X_AMG_CF: { amg_level &L = lev(index); put(dst, bytes, needed, L.cf.p, L.A.n, s); break; }
    case SIM_X_AMG_PRP: case SIM_X_AMG_PCI: case SIM_X_AMG_PV: {
      amg_level &L = lev(index);
      if (index == H.nlev - 1) RS_FAIL(SIM_ERR_ARG, "sim_ls_export: the coarsest level has no P");
      if (what == SIM_X_AMG_PRP) put(dst, bytes, needed, L.P.rp.p, L.P.n + 1, s);
      else if (what == SIM_X_AMG_PCI) put(dst, bytes, needed, L.P.ci.p, L.P.nnz, s);
      else put(dst, bytes, needed, L.P.v.p, L.P.nnz, s);
      break;
    }
    case SIM_X_RAS_SIZES: {
      if (index < 0) { int v = ls->ras.nsub; put_host(dst, bytes, needed, &v, sizeof(int)); break; }
      if (index >= ls->ras.nsub) RS_FAIL(SIM_ERR_ARG, "sim_ls_export: no subdomain %d", index);
      std::vector<int> sp = d2h(ls->ras.sub_ptr.p + index, 2, s), lp = d2h(ls->ras.lrp_ptr.p + index, 2, s);
      int m = sp[1] - sp[0];
      std::vector<uint8_t> ow = d2h(ls->ras.owned.p + sp[0], m, s);
      int nown = 0; for (auto o : ow) nown += o;
      int v[3] = {nown, m, lp[1] - lp[0]};
      put_host(dst, bytes, needed, v, sizeof(v));
      break;
    }
    case SIM_X_RAS_EXT: case SIM_X_RAS_LEVELS: {
      if (index < 0 || index >= ls->ras.nsub) RS_FAIL(SIM_ERR_ARG, "sim_ls_export: no subdomain %d", index);
      if (!ls->ras.built) RS_FAIL(SIM_ERR_STATE, "sim_ls_export: no setup yet");
      std::vector<int> sp = d2h(ls->ras.sub_ptr.p + index, 2, s);
      int base = sp[0], m = sp[1] - sp[0];
      if (what == SIM_X_RAS_EXT) {
        std::vector<int> perm = d2h(ls->ras.perm.p + base, m, s), ext = d2h(ls->ras.ext.p + base, m, s), out(m);
        for (int a = 0; a < m; a++) out[a] = ext[perm[a]];
        put_host(dst, bytes, needed, out.data(), m * sizeof(int));
      } else {
        std::vector<int> nl = d2h(ls->ras.nlev.p + 2 * index, 2, s), lv = d2h(ls->ras.lvl.p + 2 * base, 2 * m, s);
        std::vector<int> out(2 + 2 * m);
        out[0] = nl[0]; out[1] = nl[1];
        for (int a = 0; a < m; a++) { out[2 + 2 * a] = lv[a]; out[3 + 2 * a] = lv[m + a]; }
        put_host(dst, bytes, needed, out.data(), out.size() * sizeof(int));
      }
      break;
    }
    default: RS_FAIL(SIM_ERR_ARG, "sim_ls_export: unknown item %d", what);
  }
  ABI_END
}

extern "C" sim_status sim_kernel_timer(sim_ls_t ls, unsigned mask) {
  ABI_BEGIN
  if (!ls) RS_FAIL(SIM_ERR_ARG, "NULL handle");
  ls->timer_flush();
  ls->timer_mask = mask;
  for (int k = 0; k < SIM_T_NFAMILIES; k++) { ls->timer_launches[k] = 0; ls->timer_ms[k] = 0; }
  ABI_END
}
extern "C" sim_status sim_ls_graph_mode(sim_ls_t ls, int *mode) {
  ABI_BEGIN
  if (!ls || !mode) RS_FAIL(SIM_ERR_ARG, "NULL argument");
  *mode = ls->last_mode;
  ABI_END
}
extern "C" sim_status sim_ls_step_graph(sim_ls_t ls, int on) {
  ABI_BEGIN
  if (!ls) RS_FAIL(SIM_ERR_ARG, "NULL handle");
  if (on < 0 || on > 2) RS_FAIL(SIM_ERR_ARG, "sim_ls_step_graph: mode %d (0, 1 or 2)", on);
  ls->graph_mode = on;
  ls->drop_graph();
  ABI_END
}
extern "C" sim_status sim_kernel_time(sim_ls_t ls, int which, long long *launches, double *ms) {
  ABI_BEGIN
  if (!ls || which < 0 || which >= SIM_T_NFAMILIES) RS_FAIL(SIM_ERR_ARG, "sim_kernel_time: bad argument");
  RS_CUDA(cudaStreamSynchronize(ls->st));
  ls->timer_flush();
  if (launches) *launches = ls->timer_launches[which];
  if (ms) *ms = ls->timer_ms[which];
  ABI_END
}
