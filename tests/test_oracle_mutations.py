"""The oracle's pins catch plausible mistakes (no GPU needed).

Each case plants one mistake in a private copy of the oracle (a dropped
term, a wrong sign, a transposed operand or index, a reversed comparison, a
wrong constant): the C sources are copied, changed and built into their own
library, or the network module's text is changed and executed as a module
of its own.  The pin that should expose the mistake then runs with the copy
in place of the oracle and must fail.  The real oracle is untouched; the
planted C copies live in pytest's temporary directory.

Mistakes that would make the C code read out of bounds or loop forever are
not planted (they would end the test process rather than fail a pin).
"""
import ctypes
import importlib
import os

import pytest

# (name, source file, text that occurs once, its replacement, pin module, pin name, pin arguments)
MUTATIONS = [
    # model and discretisation, eqs. (3)-(18)
    ("accumulation: dropped d(phi)/dp term", "or_model.c",
     "J[0] += vt * (P[c].dphi * P[c].rho[1] + P[c].phi * P[c].drho[1]) * so;",
     "J[0] += vt * (P[c].phi * P[c].drho[1]) * so;",
     "test_oracle_model", "test_jacobian_matches_finite_differences", dict(seed=5, crossflow=False)),
    ("flux: wrong sign of dF/dp_d", "or_model.c",
     "+ Tm * P[d].dpot[a];", "- Tm * P[d].dpot[a];",
     "test_oracle_model", "test_jacobian_matches_finite_differences", dict(seed=6, crossflow=False)),
    ("flux: oil and water rows swapped", "or_model.c",
     "int e = 1 - a;                       /* equation row: oil 0, water 1 */",
     "int e = a;",
     "test_oracle_model", "test_linear_pressure_profile", {}),
    ("flux: downstream instead of upstream mobility, eq. (18)", "or_model.c",
     "int upc = P[c].pot[a] >= P[d].pot[a];", "int upc = P[c].pot[a] < P[d].pot[a];",
     "test_oracle_model", "test_buckley_leverett_front", {}),
    ("potential: gravity term with the wrong sign, eq. (5)", "or_model.c",
     "P->pot[a] = pa - P->rho[a] * gz5;", "P->pot[a] = pa + P->rho[a] * gz5;",
     "test_oracle_model", "test_hydrostatic_initial_state_is_at_rest", {}),
    ("transmissibility: arithmetic instead of harmonic mean", "or_model.c",
     "S->ft[nf++] = OR_CDARCY * (g->dy * g->dz) / (g->dx / (2.0 * kx[c]) + g->dx / (2.0 * kx[d]));",
     "S->ft[nf++] = OR_CDARCY * (g->dy * g->dz) * (kx[c] + kx[d]) / (2.0 * g->dx);",
     "test_oracle_model", "test_series_flow_through_heterogeneous_cells", dict(axis="x")),
    ("transmissibility: y faces with the x permeability", "or_model.c",
     "(g->dy / (2.0 * ky[c]) + g->dy / (2.0 * ky[d]))", "(g->dy / (2.0 * kx[c]) + g->dy / (2.0 * kx[d]))",
     "test_oracle_model", "test_series_flow_through_heterogeneous_cells", dict(axis="y")),
    ("transmissibility: z faces with the arithmetic mean", "or_model.c",
     "OR_CDARCY * (g->dx * g->dy) / (g->dz / (2.0 * kz[c]) + g->dz / (2.0 * kz[d]))",
     "OR_CDARCY * (g->dx * g->dy) * (kz[c] + kz[d]) / (2.0 * g->dz)",
     "test_oracle_model", "test_series_flow_through_heterogeneous_cells", dict(axis="z")),
    ("well index: Peaceman radius constant halved", "or_model.c",
     "double ro = 0.28 *", "double ro = 0.14 *",
     "test_oracle_model", "test_peaceman_isotropic_square", {}),
    ("well index: permeability ratio inverted in one term", "or_model.c",
     "double ro = 0.28 * sqrt(sqrt(b / a) * g->dx * g->dx", "double ro = 0.28 * sqrt(sqrt(a / b) * g->dx * g->dx",
     "test_oracle_model", "test_peaceman_anisotropic_invariances", {}),
    ("well: drawdown with the wrong sign, eq. (10)", "or_model.c",
     "double dd = (S->pb[w] - pa) + P->rho[a] * dz5;",
     "double dd = (pa - S->pb[w]) + P->rho[a] * dz5;",
     "test_oracle_model", "test_linear_pressure_profile", {}),
    ("viscosity: pressure term with the wrong sign, eq. (7)", "or_model.c",
     "P->mu[a] = f->mu_ref[a] + f->c_mu[a] * (pa - f->p_ref);", "P->mu[a] = f->mu_ref[a] - f->c_mu[a] * (pa - f->p_ref);",
     "test_oracle_model", "test_pressure_dependent_viscosity", {}),
    ("relative permeability: water exponent taken from oil", "or_model.c",
     "P->kr[0] = f->krw_max * pow(sh, f->nw);", "P->kr[0] = f->krw_max * pow(sh, f->no);",
     "test_oracle_model", "test_buckley_leverett_front_unequal_exponents", {}),
    ("geometry: cell depth at the top face instead of the centre", "or_model.c",
     "S->z[c] = g->top + ((double)k + 0.5) * g->dz;", "S->z[c] = g->top + ((double)k) * g->dz;",
     "test_oracle_model", "test_hydrostatic_initial_state_is_at_rest", {}),
    ("well: a producer also injects", "or_model.c",
     "if (dd <= 0.0) {            /* at dd = 0", "if (1) {            /* at dd = 0",
     "test_oracle_model", "test_well_flow_directions", {}),
    ("well: injector crossflow with the total mobility", "or_model.c",
     "} else if (dd < 0.0) {        /* injector crossflow", "} else if (0) {        /* injector crossflow",
     "test_oracle_model", "test_well_flow_directions", {}),
    ("old accumulation: oil stored with the water density", "or_model.c",
     "S->acc0[2 * c + 0] = P.phi * P.rho[1] * (1.0 - S->s[c]);",
     "S->acc0[2 * c + 0] = P.phi * P.rho[0] * (1.0 - S->s[c]);",
     "test_oracle_model", "test_mass_balance_identity", dict(seed=3)),
    ("inexact Newton: the fixed tolerance instead of the forcing term", "or_model.c",
     "double eta = (S->o.newton == OR_INEXACT) ? or_forcing(l, bn, rprev, bprev) : S->o.lin_tol;",
     "double eta = S->o.lin_tol;",
     "test_oracle_model", "test_inexact_newton_solves_loosely", {}),
    ("forcing term: divided by the new residual norm, eq. (26)", "or_model.c",
     "double eta = (bn - rprev) / bprev;", "double eta = (bn - rprev) / bn;",
     "test_oracle_model", "test_forcing_term_choice_two", {}),
    ("Newton: saturation chop never applied", "or_model.c",
     "if (S->o.sat_chop > 0.0) {                 /* optional saturation chop */",
     "if (0) {",
     "test_oracle_model", "test_saturation_chop_bounds_each_update", {}),
    ("time loop: a cut step advances the clock by the full step", "or_model.c",
     "if (r == 0) { S->t += dt; rem -= dt;", "if (r == 0) { S->t += S->o.dt; rem -= dt;",
     "test_oracle_model", "test_time_step_cuts_cover_the_interval", {}),
    ("Newton measure: not scaled by the step length", "or_model.c",
     "fabs(S->ls.b[2 * c + e]) * S->dt / (S->f.rho_ref[1 - e]", "fabs(S->ls.b[2 * c + e]) / (S->f.rho_ref[1 - e]",
     "test_oracle_model", "test_newton_measure_closed_cell", dict(c_w=0.0, c_o=0.0, expect=0.05)),
    ("Newton measure: each row scaled by the other phase's density", "or_model.c",
     "S->dt / (S->f.rho_ref[1 - e] * S->vol[c]", "S->dt / (S->f.rho_ref[e] * S->vol[c]",
     "test_oracle_model", "test_newton_measure_closed_cell", dict(c_w=0.0, c_o=0.0, expect=0.05)),
    ("Newton measure: well rows left out", "or_model.c",
     "    double rr = fabs(S->ls.b[2 * (S->n + w)]);\n    if (!(rr <= mx)) mx = rr;",
     "    double rr = 0.0 * fabs(S->ls.b[2 * (S->n + w)]);\n    if (!(rr <= mx)) mx = rr;",
     "test_oracle_model", "test_newton_measure_bhp_well_row", {}),
    ("BHP well row: not scaled by its target, eq. (11)", "or_model.c",
     "R[2 * wr] = (S->pb[w] - S->wtarget[w]) / S->wtarget[w];", "R[2 * wr] = (S->pb[w] - S->wtarget[w]);",
     "test_oracle_model", "test_newton_measure_bhp_well_row", {}),
    ("water-rate row: target in reservoir instead of mass units, eq. (12)", "or_model.c",
     "*cw = sgn / (S->f.rho_ref[0] * T);", "*cw = sgn / T;",
     "test_oracle_model", "test_newton_measure_water_rate_row", {}),
    # capillary pressure (eq. 9) and rate controls (eqs. 12-14, limits)
    ("capillary pressure: p_w = p_o + p_c, eq. (9)", "or_model.c",
     "double pa = a == 0 ? p - P->pc : p;", "double pa = a == 0 ? p + P->pc : p;",
     "test_oracle_wells_capillary", "test_capillary_gravity_equilibrium_is_at_rest", {}),
    ("capillary pressure: applied to the oil phase", "or_model.c",
     "double pa = a == 0 ? p - P->pc : p;", "double pa = a == 1 ? p - P->pc : p;",
     "test_oracle_wells_capillary", "test_capillary_gravity_equilibrium_is_at_rest", {}),
    ("capillary pressure: table segment one too far", "or_model.c",
     "  while (s >= f->pc_sw[k + 1]) k++;\n", "  while (s >= f->pc_sw[k + 1]) k++;\n  if (k + 2 < n) k++;\n",
     "test_oracle_wells_capillary", "test_capillary_gravity_equilibrium_is_at_rest", {}),
    ("capillary pressure: face derivative d(Pot_w)/ds_w dropped", "or_model.c",
     "double dFdsc = T * ((upc ? P[c].dms[a] : 0.0) * dpot) - Tm * P[c].dpots[a];",
     "double dFdsc = T * ((upc ? P[c].dms[a] : 0.0) * dpot);",
     "test_oracle_wells_capillary", "test_jacobian_with_capillary_pressure_and_rate_controls", dict(seed=41)),
    ("capillary pressure: water density at the oil pressure", "or_model.c",
     "P->drhos[a] = P->drho[a] * dpa_s;", "P->drhos[a] = 0.0;",
     "test_oracle_wells_capillary", "test_jacobian_with_capillary_pressure_and_rate_controls", dict(seed=42)),
    ("oil rate: target taken in water surface volumes, eq. (13)", "or_model.c",
     "*co = sgn / (S->f.rho_ref[1] * T);", "*co = sgn / (S->f.rho_ref[0] * T);",
     "test_oracle_wells_capillary", "test_rate_producer_withdraws_its_target", dict(control=2, target=40.0)),
    ("liquid rate: water left out, eq. (14)", "or_model.c",
     "if (S->wctrl[w] == OR_WRATE || S->wctrl[w] == OR_LRATE) *cw", "if (S->wctrl[w] == OR_WRATE) *cw",
     "test_oracle_wells_capillary", "test_rate_producer_withdraws_its_target", dict(control=3, target=60.0)),
    ("rate producer: production counted negative", "or_model.c",
     "double sgn = S->wkind[w] == OR_PROD ? -1.0 : 1.0", "double sgn = 1.0",
     "test_oracle_wells_capillary", "test_rate_producer_withdraws_its_target", dict(control=2, target=40.0)),
    ("BHP limit: never checked", "or_model.c",
     "    S->n_switch += limits_rate_to_bhp(S);\n", "\n",
     "test_oracle_wells_capillary", "test_injector_switches_to_its_bhp_limit_and_back", {}),
    ("BHP limit: switched back whatever the rate", "or_model.c",
     "if (r > 0.0) S->wswitched[w] = 0;", "if (1) S->wswitched[w] = 0;",
     "test_oracle_wells_capillary", "test_held_well_stays_on_its_limit_when_the_rate_is_out_of_reach", {}),
    ("BHP limit: never switched back", "or_model.c",
     "if (r > 0.0) S->wswitched[w] = 0;", "if (0) S->wswitched[w] = 0;",
     "test_oracle_wells_capillary", "test_held_producer_returns_to_its_rate_once_the_limit_delivers_it", {}),
    ("shut well: perforations still flow", "or_model.c",
     "    if (S->wctrl[w] == OR_SHUT) continue;\n", "\n",
     "test_oracle_wells_capillary", "test_shut_well_carries_no_flow", {}),
    # processing, eqs. (29)-(32)
    ("reordering key: water instead of oil potential", "or_model.c",
     "for (int c = 0; c < n; c++) ls->key[c] = P[c].pot[1];", "for (int c = 0; c < n; c++) ls->key[c] = P[c].pot[0];",
     "test_oracle_solver", "test_reordering_key_is_the_oil_potential", {}),
    ("ABF: inverse of the diagonal block transposed", "or_solve.c",
     "double i00 = d / det, i01 = -b / det, i10 = -c / det, i11 = a / det;",
     "double i00 = d / det, i01 = -c / det, i10 = -b / det, i11 = a / det;",
     "test_oracle_solver", "test_decoupling_keeps_solution", dict(dec=1)),
    ("Quasi-IMPES: ratio inverted", "or_solve.c",
     "double ratio = ls->val[4 * (size_t)qd + 1] / ls->val[4 * (size_t)qd + 3];",
     "double ratio = ls->val[4 * (size_t)qd + 3] / ls->val[4 * (size_t)qd + 1];",
     "test_oracle_solver", "test_decoupling_keeps_solution", dict(dec=2)),
    ("reordering: ascending instead of descending potential, eq. (30)", "or_solve.c",
     "if (ka > kb) return -1;                 /* descending potential */\n  if (ka < kb) return 1;",
     "if (ka < kb) return -1;\n  if (ka > kb) return 1;",
     "test_oracle_solver", "test_potential_reordering_worked_example", {}),
    ("RAS: overlap rows written back (not restricted)", "or_solve.c",
     "    for (int b = 0; b < S->nown; b++) {\n      int g = S->own[b], a = S->opos[b];\n",
     "    for (int a = 0; a < m; a++) {\n      int g = S->ext[a];\n",
     "test_oracle_solver", "test_ras_is_restricted_schwarz_with_exact_local_solves", dict(overlap=1)),
    ("RAS: overlap 2 builds a single ring", "or_solve.c",
     "int m = 0, ov = ls->o.overlap == 2 ? 2 : 1;", "int m = 0, ov = 1;",
     "test_oracle_solver", "test_subdomains_partition_and_overlap", dict(overlap=2)),
    ("GMRES: Givens rotation with the wrong sign", "or_solve.c",
     "h[k + 1] = -sn[k] * h[k] + cs[k] * h[k + 1];", "h[k + 1] = sn[k] * h[k] + cs[k] * h[k + 1];",
     "test_oracle_solver", "test_fgmres_iterations_equal_minimal_residual_gmres", dict(tile=(2, 2), coarse=8)),
    ("GMRES: Hessenberg transposed in the back substitution", "or_solve.c",
     "s -= H[(size_t)k * m + l] * yy[l];", "s -= H[(size_t)l * m + k] * yy[l];",
     "test_oracle_solver", "test_fgmres_iterations_equal_minimal_residual_gmres", dict(tile=(3, 2), coarse=128)),
    ("FGMRES restart: new basis from b instead of the residual", "or_solve.c",
     "for (int i = 0; i < nu; i++) V[i] = r[i] / beta;", "for (int i = 0; i < nu; i++) V[i] = ls->b[i] / beta;",
     "test_oracle_solver", "test_restarted_fgmres_matches_dense_solve", {}),
    ("FGMRES restart: the cycle's correction replaces the iterate", "or_solve.c",
     "s += yy[k] * Z[(size_t)k * nu + i]; y[i] += s; }", "s += yy[k] * Z[(size_t)k * nu + i]; y[i] = s; }",
     "test_oracle_solver", "test_restarted_fgmres_matches_dense_solve", {}),
    ("BiCGSTAB: search direction without the omega v term", "or_solve.c",
     "p[i] = r[i] + beta * (p[i] - omega * v[i]);", "p[i] = r[i] + beta * p[i];",
     "test_oracle_solver", "test_bicgstab_cpr_matches_dense_solve", dict(tile=(2, 2), coarse=8)),
    ("BiCGSTAB: update without the second preconditioned direction", "or_solve.c",
     "x[i] += alpha * ph[i] + omega * sh[i];", "x[i] += alpha * ph[i];",
     "test_oracle_solver", "test_bicgstab_cpr_matches_dense_solve", dict(tile=(2, 2), coarse=8)),
    ("BiCGSTAB: residual update with the wrong sign", "or_solve.c",
     "r[i] = s[i] - omega * t[i];", "r[i] = s[i] + omega * t[i];",
     "test_oracle_solver", "test_bicgstab_cpr_matches_dense_solve", dict(tile=(2, 2), coarse=8)),
    ("BiCGSTAB: beta without the alpha / omega factor", "or_solve.c",
     "double beta = (rho / rho_prev) * (alpha / omega);", "double beta = (rho / rho_prev);",
     "test_oracle_solver", "test_bicgstab_cpr_matches_dense_solve", dict(tile=(2, 2), coarse=8)),
    # AMG (Algorithm 2, pressure stage)
    ("strength: comparison reversed", "or_amg.c",
     "-A->v[q] >= thr", "-A->v[q] <= thr",
     "test_oracle_solver", "test_strength_hand_example", {}),
    ("strength: threshold from the largest magnitude", "or_amg.c",
     "      double v = -A->v[q];\n", "      double v = fabs(A->v[q]);\n",
     "test_oracle_solver", "test_strength_hand_example", {}),
    ("strength: a zero entry counts as strong", "or_amg.c",
     "have && mx > 0.0 && ", "have && ",
     "test_oracle_solver", "test_strength_hand_example", {}),
    ("interpolation: positive entries not lumped into the diagonal", "or_amg.c",
     "double dg = aii + spos,", "double dg = aii,",
     "test_oracle_solver", "test_interpolation_and_galerkin_product", dict(positive=True)),
    ("interpolation: alpha inverted", "or_amg.c",
     "alpha = sneg / snegc;", "alpha = snegc / sneg;",
     "test_oracle_solver", "test_interpolation_and_galerkin_product", dict(positive=False)),
    ("interpolation: weights with the wrong sign", "or_amg.c",
     "P->v[o++] = -(alpha * A->v[q]) / dg;", "P->v[o++] = (alpha * A->v[q]) / dg;",
     "test_oracle_solver", "test_interpolation_and_galerkin_product", dict(positive=False)),
    ("extended+i: no distance-two points", "or_amg.c",
     "      else for (int r = A->rp[j]; r < A->rp[j + 1]; r++) {\n        int l = A->ci[r];\n        if (S[r] && cf[l] == 1 && stamp[l] != i)",
     "      else for (int r = A->rp[j]; r < A->rp[j]; r++) {\n        int l = A->ci[r];\n        if (S[r] && cf[l] == 1 && stamp[l] != i)",
     "test_oracle_solver", "test_exti_reproduces_linear_interpolation_in_1d", {}),
    ("extended+i: D_k without the coupling back to i", "or_amg.c",
     "if (l == i || in_sorted(cs, m, l)) d = d + hat(akk, A->v[r]);", "if (in_sorted(cs, m, l)) d = d + hat(akk, A->v[r]);",
     "test_oracle_solver", "test_exti_reproduces_linear_interpolation_in_1d", {}),
    ("extended+i: distributes couplings of the diagonal's sign", "or_amg.c",
     "  return akl < 0.0 ? akl : 0.0;\n}", "  return akl > 0.0 ? akl : 0.0;\n}",
     "test_oracle_solver", "test_exti_reproduces_linear_interpolation_in_1d", {}),
    ("extended+i: weak couplings not lumped into the diagonal", "or_amg.c",
     "      } else if (!in_sorted(cs, m, j)) at = at + A->v[q];", "      }",
     "test_oracle_solver", "test_exti_pattern_and_row_sums", dict(seed=1)),
    ("coarsest solve: LU without row exchanges", "or_amg.c",
     "if (fabs(a[(size_t)i * n + k]) > mx) {", "if (0) {",
     "test_oracle_solver", "test_coarsest_only_hierarchy_is_a_dense_solve", dict(permuted=True)),
    ("V-cycle: coarse-grid correction subtracted", "or_amg.c",
     "for (int i = 0; i < n; i++) x[i] += t[i];", "for (int i = 0; i < n; i++) x[i] -= t[i];",
     "test_oracle_solver", "test_vcycle_convergence_on_poisson", {}),
]


@pytest.fixture(scope="module")
def oracle_mod():
    import oracle
    oracle.build()
    return oracle


@pytest.mark.parametrize("name,src,old,new,mod,pin,kw", MUTATIONS, ids=[m[0] for m in MUTATIONS])
def test_pin_catches_planted_mistake(oracle_mod, tmp_path, monkeypatch, name, src, old, new, mod, pin, kw):
    here = os.path.dirname(oracle_mod.__file__)
    for f in oracle_mod._SRC + ["or_internal.h"]:
        text = open(os.path.join(here, f)).read()
        if f == src:
            assert text.count(old) == 1, f"{name}: the text to replace occurs {text.count(old)} times in {src}"
            text = text.replace(old, new)
        (tmp_path / f).write_text(text)
    so = str(tmp_path / "liboracle_planted.so")
    oracle_mod.compile_sources(str(tmp_path), so)
    lib = ctypes.CDLL(so)
    oracle_mod._sig(lib)
    fn = getattr(importlib.import_module(mod), pin)
    fn(oracle_mod, **kw)                                  # the real oracle passes the pin ...
    monkeypatch.setattr(oracle_mod, "_lib", lib)
    with pytest.raises(AssertionError):                   # ... the planted copy fails it
        fn(oracle_mod, **kw)


# the network oracle (numpy): (name, text that occurs once, its replacement, pin name, pin arguments)
NN_MUTATIONS = [
    ("conv: tap order z-fastest instead of x-fastest",
     "OFFSETS = [(dx, dy, dz) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]",
     "OFFSETS = [(dx, dy, dz) for dx in (-1, 0, 1) for dy in (-1, 0, 1) for dz in (-1, 0, 1)]",
     "test_conv_matches_brute_force", {}),
    ("conv backward: gradient shifted the wrong way",
     "dX += _shift(G @ W[t], -dx, -dy, -dz)", "dX += _shift(G @ W[t], dx, dy, dz)",
     "test_conv_backward_is_the_adjoint", {}),
    ("conv backward: weight gradient from the unshifted input",
     "dW[t] = Gf.T @ S.reshape(-1, S.shape[-1])", "dW[t] = Gf.T @ X.reshape(-1, X.shape[-1])",
     "test_conv_backward_is_the_adjoint", {}),
    ("pool: divided by 8 at ragged edges", "    return S / cnt\n", "    return S / 8.0\n",
     "test_pool_and_up_adjoints", dict(shape=(3, 5, 7))),
    ("pool backward: not divided by the child count", "    Gs = G / cnt\n", "    Gs = G\n",
     "test_pool_and_up_adjoints", dict(shape=(4, 6, 8))),
    ("forward: skip concatenated before the up-sampled tensor",
     "np.concatenate([up(b2, s1), e1], axis=-1)", "np.concatenate([e1, up(b2, s1)], axis=-1)",
     "test_network_gradient_matches_finite_differences", {}),
    ("backward: ReLU mask dropped on a skip gradient",
     'de1 = r(masked("c11", dcat1[..., 32:] + pool_backward(s1, dp2)))',
     'de1 = r(dcat1[..., 32:] + pool_backward(s1, dp2))',
     "test_network_gradient_matches_finite_differences", {}),
    ("loss: factor 1/2 dropped", "return 0.5 * float(np.sum(E * E)) / n", "return float(np.sum(E * E)) / n",
     "test_loss_definition", {}),
    ("Adam: second moment without its bias correction", "vh = v / (1.0 - beta2 ** t)", "vh = v / (1.0 - beta2)",
     "test_adam_constant_gradient_every_step", {}),
    ("Adam: first moment not accumulated", "m = beta1 * m + (1.0 - beta1) * g", "m = (1.0 - beta1) * g",
     "test_adam_constant_gradient_every_step", {}),
    ("bf16: ties rounded up instead of to even", "r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16",
     "r = ((u + 0x8000) >> 16) << 16", "test_bf16_round_matches_torch", {}),
]


@pytest.mark.parametrize("name,old,new,pin,kw", NN_MUTATIONS, ids=[m[0] for m in NN_MUTATIONS])
def test_network_pin_catches_planted_mistake(monkeypatch, name, old, new, pin, kw):
    import types
    from oracle import nn
    text = open(nn.__file__).read()
    assert text.count(old) == 1, f"{name}: the text to replace occurs {text.count(old)} times"
    planted = types.ModuleType("planted_nn")
    exec(compile(text.replace(old, new), "planted_nn.py", "exec"), planted.__dict__)
    tests = importlib.import_module("test_oracle_nn")
    fn = getattr(tests, pin)
    fn(**kw)                                              # the real network oracle passes the pin ...
    monkeypatch.setattr(tests, "nn", planted)
    with pytest.raises(AssertionError):                   # ... the planted copy fails it
        fn(**kw)
