"""Pins of the CPU oracle's linear-system processing and CPR-FGMRES solver
(no GPU needed).

Passages: ABF / Quasi-IMPES decoupling and eq. (29); local potential
reordering eqs. (30)-(32) and its worked example; Algorithm 2 (CPR-FPF);
GMRES(m) of arXiv 1701.06254.  AMG and RAS details follow the readings
stated in the oracle sources.
"""
import os

import numpy as np
import pytest

from paper_1701_06254_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _dense_J(rp, ci, val, nb):
    J = np.zeros((2 * nb, 2 * nb))
    for i in range(nb):
        for q in range(rp[i], rp[i + 1]):
            j = ci[q]
            J[2 * i:2 * i + 2, 2 * j:2 * j + 2] = val[4 * q:4 * q + 4].reshape(2, 2)
    return J


def _system(oracle_lib, case, seed, **opts):
    """Assemble the Newton system of `case` at a random state."""
    s = oracle_lib.Sim(case, **opts)
    p0, s0, pb0 = I.random_state(case, seed)
    p1, s1, pb1 = I.random_state(case, seed + 1)
    s.set_state(p0, s0, pb0); s.store_old()
    s.set_state(p1, s1, pb1); s.assemble()
    return s


def _read_kv(path):
    out = {}
    for line in open(path):
        if line.startswith("#") or ":" not in line:
            continue
        k, v = line.split(":", 1)
        out[k.strip()] = v.split()
    return out


def test_potential_reordering_worked_example(oracle_lib):
    g = _read_kv(os.path.join(GOLD, "potential_reordering_example.txt"))
    pot = np.array([float(x) for x in g["potentials"]])
    pm = np.array([int(x) for x in g["pm"]])
    np.testing.assert_array_equal(oracle_lib.pm_mapping(pot), pm)


def test_potential_reordering_ties_and_permutation(oracle_lib):
    key = np.array([1.0, 3.0, 1.0, 3.0, 2.0])
    order = oracle_lib.potential_order(key)
    np.testing.assert_array_equal(order, [1, 3, 4, 0, 2])       # ties keep index order
    rng = np.random.default_rng(0)
    key = rng.integers(0, 5, 200).astype(float)
    order = oracle_lib.potential_order(key)
    assert sorted(order.tolist()) == list(range(200))
    assert np.all(np.diff(key[order]) <= 0)


def test_splitmix64_published_vectors(oracle_lib):
    for line in open(os.path.join(GOLD, "splitmix64_vectors.txt")):
        if line.startswith("#") or not line.strip():
            continue
        x, y = (int(v) for v in line.split())
        assert oracle_lib.splitmix64(x) == y
    h = [oracle_lib.pmis_hash(7, 0, i) for i in range(1000)]
    assert 0.0 <= min(h) and max(h) < 1.0 and len(set(h)) == 1000


@pytest.mark.parametrize("dec", [1, 2])
def test_decoupling_keeps_solution(oracle_lib, dec):
    """D^{-1} A x = D^{-1} b has the solution of A x = b (eq. 29).  ABF
    turns every cell's diagonal block into I; Quasi-IMPES zeroes its (p, s)
    entry; well rows are left unchanged by both."""
    c = I.small_case(4, 3, 2, seed=11)
    s = _system(oracle_lib, c, 40, decoupling=dec)
    rp, ci, val, b, key = s.system()
    nb = c.n + 2
    J = _dense_J(rp, ci, val, nb)
    x = np.linalg.solve(J, b)
    s.ls.setup()
    rp2, ci2, val2, b2, _ = s.ls.get()
    J2 = _dense_J(rp2, ci2, val2, nb)
    x2 = np.linalg.solve(J2, b2)
    np.testing.assert_allclose(x2, x, rtol=1e-9, atol=1e-12 * np.abs(x).max())
    for i in range(c.n):
        D = J2[2 * i:2 * i + 2, 2 * i:2 * i + 2]
        if dec == 1:
            M = J[2 * i:2 * i + 2, 2 * i:2 * i + 2]
            bound = 4 * np.finfo(float).eps * (np.abs(np.linalg.inv(M)) @ np.abs(M))
            assert np.all(np.abs(D - np.eye(2)) <= bound)
        else:
            assert abs(D[0, 1]) <= 1e-12 * abs(J[2 * i, 2 * i + 1])
            # only the pressure row changes, by a multiple of its own
            # cell's saturation row
            np.testing.assert_array_equal(J2[2 * i + 1], J[2 * i + 1])
            assert b2[2 * i + 1] == b[2 * i + 1]
            ratio = J[2 * i, 2 * i + 1] / J[2 * i + 1, 2 * i + 1]
            np.testing.assert_allclose(J2[2 * i], J[2 * i] - ratio * J[2 * i + 1],
                                       rtol=0, atol=1e-13 * np.abs(J[2 * i]).max())
    np.testing.assert_array_equal(J2[2 * c.n:], J[2 * c.n:])


def test_cpr_is_exact_with_exact_stages(oracle_lib):
    """Algorithm 2 with an exact RAS stage (one subdomain, BILU(0) = LU on a
    block-tridiagonal 1D system) returns A^{-1} f: FGMRES converges in one
    iteration."""
    n = 40
    kk = np.exp(np.random.default_rng(2).normal(np.log(100), 1, n))
    c = I.Case("line", n, 1, 1, 10.0, 10.0, 10.0, 1000.0, kk, kk.copy(), kk.copy(),
               np.full(n, 0.2), I.Fluid(g=0.0), [], dt=1.0, n_steps=1)
    s = _system(oracle_lib, c, 50, tile_x=64, tile_y=64, reorder=0)
    rp, ci, val, b, key = s.system()
    J = _dense_J(rp, ci, val, n)
    rc, y, its, rel = s.linear_solve(1e-12)
    assert rc == 0 and its == 1
    np.testing.assert_allclose(y, np.linalg.solve(J, b), rtol=1e-10, atol=1e-14)
    # and RAS alone on the decoupled system is already a direct solve
    _, _, val2, b2, _ = s.ls.get()
    J2 = _dense_J(rp, ci, val2, n)
    np.testing.assert_allclose(s.ls.ras(b2), np.linalg.solve(J2, b2), rtol=1e-10, atol=1e-14)


@pytest.mark.parametrize("tile,coarse", [((2, 2), 8), ((3, 2), 128), ((8, 8), 4)])
def test_fgmres_cpr_matches_dense_solve(oracle_lib, tile, coarse):
    """CPR-FGMRES on small heterogeneous systems with wells, several RAS
    subdomains and a multi-level AMG: the result matches a dense LU solve
    and the reported relative residual is the true one."""
    c = I.small_case(6, 5, 3, seed=12)
    s = _system(oracle_lib, c, 60, tile_x=tile[0], tile_y=tile[1], amg_coarse_max=coarse)
    rp, ci, val, b, key = s.system()
    nb = c.n + 2
    J = _dense_J(rp, ci, val, nb)
    ystar = np.linalg.solve(J, b)
    rc, y, its, rel = s.linear_solve(1e-11)
    assert rc == 0 and 1 <= its <= 60
    _, _, val2, b2, _ = s.ls.get()
    J2 = _dense_J(rp, ci, val2, nb)
    assert np.linalg.norm(b2 - J2 @ y) <= 1.0001e-11 * np.linalg.norm(b2)
    np.testing.assert_allclose(rel, np.linalg.norm(b2 - J2 @ y) / np.linalg.norm(b2), rtol=1e-3)
    cond = np.linalg.cond(J2)
    assert np.linalg.norm(y - ystar) <= 1e-11 * cond * np.linalg.norm(ystar)


def test_restarted_fgmres_matches_dense_solve(oracle_lib):
    """FGMRES(m) with a short restart (m = 3): each cycle starts from the
    true residual of the current iterate and adds its correction, so the
    restarted solver still reaches the tolerance and the dense solution."""
    c = I.small_case(6, 5, 3, seed=12)
    s = _system(oracle_lib, c, 60, tile_x=2, tile_y=2, amg_coarse_max=8, restart=3, max_lin=600)
    rp, ci, val, b, key = s.system()
    nb = c.n + 2
    ystar = np.linalg.solve(_dense_J(rp, ci, val, nb), b)
    rc, y, its, rel = s.linear_solve(1e-10)
    assert rc == 0 and its > 3, (rc, its)                  # converged, after restarts
    _, _, val2, b2, _ = s.ls.get()
    J2 = _dense_J(rp, ci, val2, nb)
    assert np.linalg.norm(b2 - J2 @ y) <= 1.0001e-10 * np.linalg.norm(b2)
    np.testing.assert_allclose(y, ystar, rtol=1e-6, atol=1e-9 * np.abs(ystar).max())


@pytest.mark.parametrize("tile,coarse", [((2, 2), 8), ((3, 2), 128)])
def test_fgmres_iterations_equal_minimal_residual_gmres(oracle_lib, tile, coarse):
    """With a fixed preconditioner M (the CPR of Algorithm 2 is linear once
    set up), FGMRES(m) before its first restart is right-preconditioned
    GMRES: iterate k minimises ||b - A x|| over x in M K_k(A M, b).  So it
    reaches the tolerance at the same iteration as a plain Arnoldi process
    whose small least-squares problem is solved by numpy's lstsq (rounding
    may move the crossing by one)."""
    c = I.small_case(6, 5, 3, seed=12)
    s = _system(oracle_lib, c, 60, tile_x=tile[0], tile_y=tile[1], amg_coarse_max=coarse)
    s.ls.setup()
    rp, ci, val, b, key = s.ls.get()
    nb = c.n + 2
    A = _dense_J(rp, ci, val, nb)
    tol = 1e-10
    rc, y, its, rel = s.ls.solve(tol)
    assert rc == 0 and its < 50                       # converged inside the first cycle
    beta = np.linalg.norm(b)
    V = [b / beta]
    H = np.zeros((52, 51))
    its_ref = None
    for j in range(50):
        w = A @ s.ls.cpr(V[j])
        for k in range(j + 1):                        # modified Gram-Schmidt
            H[k, j] = V[k] @ w
            w = w - H[k, j] * V[k]
        H[j + 1, j] = np.linalg.norm(w)
        V.append(w / H[j + 1, j])
        e1 = np.zeros(j + 2)
        e1[0] = beta
        yk = np.linalg.lstsq(H[:j + 2, :j + 1], e1, rcond=None)[0]
        if np.linalg.norm(e1 - H[:j + 2, :j + 1] @ yk) <= tol * beta:
            its_ref = j + 1
            break
    assert its_ref is not None and abs(its - its_ref) <= 1, (its, its_ref)


def test_reordering_key_is_the_oil_potential(oracle_lib):
    """The key of the local reordering is each cell's oil-phase potential,
    eq. (5) with eq. (6): p - rho_o(p) g z at the cell centre (depth z,
    positive downwards; bar)."""
    c = I.small_case(4, 3, 5, seed=33)
    s = _system(oracle_lib, c, 90)
    key = s.system()[4]
    p = s.get_state()[0]
    f = c.fluid
    z = c.top + (np.arange(c.n) // (c.nx * c.ny) + 0.5) * c.dz
    rho_o = f.rho_ref[1] * (1.0 + f.c_f[1] * (p - f.p_ref))
    np.testing.assert_allclose(key, p - rho_o * f.g * z * 1e-5, rtol=1e-13)
    rho_w = f.rho_ref[0] * (1.0 + f.c_f[0] * (p - f.p_ref))
    assert np.abs(key - (p - rho_w * f.g * z * 1e-5)).max() > 1.0    # the phases differ by bars here


@pytest.mark.parametrize("overlap", [1, 2])
def test_subdomains_partition_and_overlap(oracle_lib, overlap):
    """Owned sets partition the unknowns; the extended set of each
    subdomain is every row within graph distance `overlap` of its owned
    rows (1, or 2 as in the paper's Table 9); cells come in descending
    potential order and wells last (eq. 32)."""
    c = I.small_case(7, 5, 2, seed=13)
    s = _system(oracle_lib, c, 70, tile_x=3, tile_y=2, overlap=overlap)
    s.ls.setup()
    rp, ci, val, b, key = s.ls.get()
    nb = c.n + 2
    owned = []
    for k in range(s.ls.nsub):
        d = s.ls.sub(k)
        owned.extend(d["own"].tolist())
        nbrs = set(d["own"].tolist())
        for _ in range(overlap):                       # breadth-first rings
            nbrs = nbrs | {int(x) for g in nbrs for x in ci[rp[g]:rp[g + 1]]}
        assert set(d["ext"].tolist()) == nbrs
        cells = [g for g in d["ext"] if g < c.n]
        wells = [g for g in d["ext"] if g >= c.n]
        assert list(d["ext"]) == cells + wells
        kk = key[cells]
        assert np.all((np.diff(kk) < 0) | ((np.diff(kk) == 0) & (np.diff(cells) > 0)))
    assert sorted(owned) == list(range(nb))
    assert s.ls.nsub == 3 * 3


@pytest.mark.parametrize("overlap", [1, 2])
def test_ras_is_restricted_schwarz_with_exact_local_solves(oracle_lib, overlap):
    """The RAS stage of Algorithm 2 is sum_s R~_s^T A_s^{-1} R_s: each
    subdomain solves on its extended rows and keeps only the rows it owns.
    On a heterogeneous 1D line in natural order every extended matrix is
    block tridiagonal, so BILU(0) is its exact LU, and the output at a
    subdomain's owned unknowns equals a dense solve of its extended system
    (overlap rows: `overlap` cells on each inner side)."""
    n = 40
    kk = np.exp(np.random.default_rng(3).normal(np.log(100.0), 1.0, n))
    c = I.Case("line", n, 1, 1, 10.0, 10.0, 10.0, 1000.0, kk, kk.copy(), kk.copy(),
               np.full(n, 0.2), I.Fluid(g=0.0), [], dt=1.0, n_steps=1)
    s = _system(oracle_lib, c, 80, tile_x=4, tile_y=1, reorder=0, overlap=overlap)
    s.ls.setup()
    assert s.ls.nsub == 10
    rp, ci, val, b, key = s.ls.get()
    J = _dense_J(rp, ci, val, n)
    f = np.random.default_rng(4).standard_normal(2 * n)
    x = s.ls.ras(f)
    expect = np.full(2 * n, np.nan)
    for k in range(s.ls.nsub):
        d = s.ls.sub(k)
        ext = list(d["ext"])
        assert len(ext) == len(d["own"]) + overlap * ((k > 0) + (k < s.ls.nsub - 1))
        idx = np.array([2 * g + e for g in ext for e in (0, 1)])
        y = np.linalg.solve(J[np.ix_(idx, idx)], f[idx])
        for g in d["own"]:
            a = ext.index(g)
            expect[2 * g:2 * g + 2] = y[2 * a:2 * a + 2]
    assert not np.isnan(expect).any()
    np.testing.assert_allclose(x, expect, rtol=1e-10, atol=1e-12 * np.abs(expect).max())


def test_reordered_saturation_block_is_lower_triangular(oracle_lib):
    """Upstream weighting makes each cell's water equation depend only on
    the saturations of cells with a higher potential, so after the
    descending-potential reordering A_ss is lower triangular (the paper's
    motivation for the reordering).  Flow runs towards cell 0 here, so the
    natural order gives an upper triangular A_ss instead."""
    n = 30
    kk = np.full(n, 100.0)
    c = I.Case("line", n, 1, 1, 10.0, 10.0, 10.0, 1000.0, kk, kk.copy(), kk.copy(),
               np.full(n, 0.2), I.Fluid(g=0.0), [], dt=1.0, n_steps=1)
    c.wells = [I.Well(I.PROD, I.BHP, 150.0, [0]), I.Well(I.INJ, I.WRATE, 50.0, [n - 1])]
    res = {}
    for reorder in (0, 1):
        s = oracle_lib.Sim(c, tile_x=64, reorder=reorder)
        p = 200.0 + np.arange(n, dtype=float)
        sw = np.random.default_rng(1).uniform(0.3, 0.7, n)
        s.set_state(p, sw * 0.9, [170.0, 260.0]); s.store_old()
        s.set_state(p, sw, [170.0, 260.0]); s.assemble()
        rp, ci, val, b, key = s.system()
        s.ls.setup()
        ext = s.ls.sub(0)["ext"]
        pos = {g: a for a, g in enumerate(ext)}
        upper = lower = 0
        for i in range(n):
            for q in range(rp[i], rp[i + 1]):
                j = ci[q]
                if j >= n or j == i or val[4 * q + 3] == 0.0:
                    continue
                if pos[j] > pos[i]:
                    upper += 1
                else:
                    lower += 1
        res[reorder] = (upper, lower)
    assert res[1][0] == 0 and res[1][1] == n - 1
    assert res[0][1] == 0 and res[0][0] == n - 1


# ------------------------------- AMG pins ----------------------------------

def _csr(M):
    rp = [0]; ci = []; v = []
    for i in range(M.shape[0]):
        nz = np.nonzero(M[i])[0]
        ci.extend(nz.tolist()); v.extend(M[i, nz].tolist()); rp.append(len(ci))
    return np.array(rp, np.int32), np.array(ci, np.int32), np.array(v)


def _poisson3d(m):
    n = m ** 3
    M = np.zeros((n, n))
    for k in range(m):
        for j in range(m):
            for i in range(m):
                c = i + m * (j + m * k)
                M[c, c] = 6.0
                for di, dj, dk in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
                    ii, jj, kk = i + di, j + dj, k + dk
                    if 0 <= ii < m and 0 <= jj < m and 0 <= kk < m:
                        M[c, ii + m * (jj + m * kk)] = -1.0
    return M


def _random_mmatrix(n, seed, density=0.12):
    """A random weighted graph Laplacian plus a small diagonal shift:
    structurally symmetric, non-symmetric values, off-diagonals <= 0."""
    rng = np.random.default_rng(seed)
    M = np.zeros((n, n))
    for i in range(n):
        for j in range(i + 1, n):
            if rng.random() < density:
                M[i, j] = -rng.uniform(0.05, 1.0)
                M[j, i] = -rng.uniform(0.05, 1.0)
    np.fill_diagonal(M, -M.sum(axis=1) + 0.01)
    return M


def test_strength_hand_example(oracle_lib):
    """Row [4, -1, -0.2, -1, +0.5]: max(-a_ij) = 1, theta = 0.25 -> the two
    -1 entries are strong; -0.2 and the positive entry are not."""
    M = np.zeros((5, 5))
    M[0] = [4, -1, -0.2, -1, 0.5]
    for i in range(1, 5):
        M[i, i] = 3.0; M[i, 0] = -1.0
    rp, ci, v = _csr(M)
    h = oracle_lib.AMG(rp, ci, v, theta=0.25, coarse_max=1, max_levels=2)
    L = h.level(0)
    s0 = L["strong"][rp[0]:rp[1]]
    np.testing.assert_array_equal(s0, [False, True, False, True, False])
    # a row without negative off-diagonal entries has no strong connection,
    # also when one of its stored entries is an exact zero (Galerkin products
    # keep cancelled entries in the pattern)
    M[4] = [-1.0, 0.0, 0.0, 0.0, 3.0]
    M[3] = [-1.0, 0.0, 0.0, 3.0, 0.5]
    rp, ci, v = _csr(M)
    v[rp[4]] = 0.0                                           # stored zero at (4, 0)
    h = oracle_lib.AMG(rp, ci, v, theta=0.25, coarse_max=1, max_levels=2)
    st = h.level(0)["strong"]
    assert not st[rp[4]:rp[5]].any()
    np.testing.assert_array_equal(st[rp[3]:rp[4]], [True, False, False])
    # the threshold follows the most negative entry, not the largest in
    # magnitude: next to a +2 entry, -0.3 is still strong (0.3 >= 0.25 * 1)
    M[2] = [-1.0, 0.0, 4.0, -0.3, 2.0]
    rp, ci, v = _csr(M)
    h = oracle_lib.AMG(rp, ci, v, theta=0.25, coarse_max=1, max_levels=2)
    np.testing.assert_array_equal(h.level(0)["strong"][rp[2]:rp[3]], [True, False, True, False])


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("symmetric", [False, True])
def test_pmis_invariants(oracle_lib, seed, symmetric):
    """What the PMIS rounds guarantee: every point is decided; a C point
    influences someone; an F point that influences someone strongly depends
    on a C point; two C points are never mutually dependent, and when C
    point i depends on C point j then i was picked first, i.e. it has the
    larger weight |S^T_i| + h(i).  With a symmetric strength graph the C
    points are an independent set of it."""
    n = 30 + 5 * seed
    M = _random_mmatrix(n, seed)
    if symmetric:                      # unweighted symmetric graph: every edge is strong both ways
        M = -((M != 0) | (M.T != 0)).astype(float)
        np.fill_diagonal(M, 0.0)
        np.fill_diagonal(M, -M.sum(axis=1) + 0.01)
    rp, ci, v = _csr(M)
    h = oracle_lib.AMG(rp, ci, v, theta=0.25, seed=seed, coarse_max=1, max_levels=2)
    L = h.level(0)
    cf, S = L["cf"], L["strong"]
    assert set(np.unique(cf).tolist()) <= {-1, 1}
    Smat = np.zeros((n, n), bool)
    for i in range(n):
        for q in range(rp[i], rp[i + 1]):
            Smat[i, ci[q]] = S[q]
    stcount = Smat.sum(axis=0)                                   # |S^T_i|
    w = stcount + np.array([oracle_lib.pmis_hash(seed, 0, i) for i in range(n)])
    C = np.nonzero(cf == 1)[0]
    assert (stcount[C] > 0).all()
    for i in np.nonzero(cf == -1)[0]:
        if stcount[i] > 0:
            assert (Smat[i] & (cf == 1)).any()
    for i in C:
        for j in C:
            if Smat[i, j]:
                assert not Smat[j, i]
                assert w[i] > w[j]
    if symmetric:
        assert (Smat == Smat.T).all()
        assert not Smat[np.ix_(C, C)].any()
    assert 0 < len(C) < n


@pytest.mark.parametrize("positive", [False, True])
def test_interpolation_and_galerkin_product(oracle_lib, positive):
    """Direct interpolation: C rows of P are unit rows; an F row of a
    zero-row-sum matrix row sums to 1, also when the row has positive
    off-diagonal entries (they are lumped into the diagonal, so the
    weights still reproduce constants).  The coarse matrix equals the dense
    product P^T A P."""
    M = _poisson3d(6)
    if positive:                                 # weak positive couplings two cells apart along x
        for c in range(M.shape[0]):
            if c % 6 < 4:
                M[c, c + 2] = M[c + 2, c] = 0.3
    # zero row sums in the interior: remove the Dirichlet-like excess on the boundary
    np.fill_diagonal(M, 0.0)
    np.fill_diagonal(M, -M.sum(axis=1))
    M[0, 0] += 1.0                                               # one anchor keeps A nonsingular
    rp, ci, v = _csr(M)
    h = oracle_lib.AMG(rp, ci, v, theta=0.25, coarse_max=10, max_levels=3)
    assert h.nlev >= 2
    L = h.level(0)
    n, nc = L["n"], L["nc"]
    P = np.zeros((n, nc))
    for i in range(n):
        for q in range(L["prp"][i], L["prp"][i + 1]):
            P[i, L["pci"][q]] = L["pv"][q]
    cf = L["cf"]
    Crows = np.nonzero(cf == 1)[0]
    np.testing.assert_array_equal(P[Crows], np.eye(nc)[np.arange(nc)])
    zero_sum = np.abs(M.sum(axis=1)) < 1e-14
    checked = 0
    for i in np.nonzero((cf == -1) & zero_sum)[0]:
        if P[i].any():
            assert abs(P[i].sum() - 1.0) < 1e-14
            checked += (M[i] > 0).sum() > 1 if positive else 1
    assert checked > 10
    L1 = h.level(1)
    Ac = np.zeros((nc, nc))
    for i in range(nc):
        for q in range(L1["rp"][i], L1["rp"][i + 1]):
            Ac[i, L1["ci"][q]] = L1["v"][q]
    np.testing.assert_allclose(Ac, P.T @ M @ P, rtol=1e-12, atol=1e-12 * np.abs(M).max())


def test_vcycle_convergence_on_poisson(oracle_lib):
    """One V(1,1) per iteration of x <- x + M(f - A x) on the 3D Poisson
    matrix reduces the error by a factor well below 1 (divergence or a slow
    factor would expose a wrong sign, transpose or weight in P, R, A_c or
    the smoother)."""
    A = _poisson3d(12)
    rp, ci, v = _csr(A)
    h = oracle_lib.AMG(rp, ci, v, theta=0.25, coarse_max=64, max_levels=10)
    assert h.nlev >= 3
    rng = np.random.default_rng(3)
    xs = rng.standard_normal(A.shape[0])
    f = A @ xs
    x = np.zeros_like(f)
    errs = []
    for it in range(12):
        x = x + h.apply(f - A @ x)
        errs.append(np.sqrt((x - xs) @ A @ (x - xs)))
    rho = (errs[-1] / errs[-6]) ** (1 / 5)
    assert rho < 0.7, rho         # measured 0.60 (PMIS + direct interpolation, one l1-Jacobi sweep)


@pytest.mark.parametrize("permuted", [False, True])
def test_coarsest_only_hierarchy_is_a_dense_solve(oracle_lib, permuted):
    """The coarsest level is solved exactly (LU with partial pivoting); the
    row-permuted matrix has zeros on its diagonal, so the factorisation must
    exchange rows."""
    A = _random_mmatrix(40, 9)
    if permuted:
        A = A[np.roll(np.arange(40), 7)]
        assert (np.diag(A) == 0).sum() > 20
    rp, ci, v = _csr(A)
    h = oracle_lib.AMG(rp, ci, v, coarse_max=128)
    assert h.nlev == 1
    f = np.random.default_rng(4).standard_normal(40)
    np.testing.assert_allclose(h.apply(f), np.linalg.solve(A, f), rtol=1e-10)


# ---- BiCGSTAB, the paper's other Krylov method (Examples 3, 6, 7) ----
def test_bicgstab_with_an_exact_preconditioner_takes_one_iteration(oracle_lib):
    """With exact CPR stages (one subdomain, BILU(0) = LU on a 1D block-
    tridiagonal system) M^-1 = A^-1, so the first BiCGSTAB half step already
    gives s = r - alpha A M^-1 p = 0 (p = r, alpha = 1): one iteration, and
    the dense solution."""
    n = 40
    kk = np.exp(np.random.default_rng(2).normal(np.log(100), 1, n))
    c = I.Case("line", n, 1, 1, 10.0, 10.0, 10.0, 1000.0, kk, kk.copy(), kk.copy(),
               np.full(n, 0.2), I.Fluid(g=0.0), [], dt=1.0, n_steps=1)
    s = _system(oracle_lib, c, 50, tile_x=64, tile_y=64, reorder=0, krylov=1)
    rp, ci, val, b, key = s.system()
    rc, y, its, rel = s.linear_solve(1e-12)
    assert rc == 0 and its == 1, (rc, its)
    np.testing.assert_allclose(y, np.linalg.solve(_dense_J(rp, ci, val, n), b), rtol=1e-10, atol=1e-14)


@pytest.mark.parametrize("tile,coarse", [((2, 2), 8), ((3, 2), 128)])
def test_bicgstab_cpr_matches_dense_solve(oracle_lib, tile, coarse):
    """CPR-BiCGSTAB on small heterogeneous systems with wells, several RAS
    subdomains and a multi-level AMG: the reported relative residual is the
    true one, below the tolerance, the result matches a dense LU solve, and
    it takes no more iterations than CPR-FGMRES takes Arnoldi steps (each
    BiCGSTAB iteration applies the preconditioner twice)."""
    c = I.small_case(6, 5, 3, seed=12)
    s = _system(oracle_lib, c, 60, tile_x=tile[0], tile_y=tile[1], amg_coarse_max=coarse, krylov=1)
    rp, ci, val, b, key = s.system()
    nb = c.n + 2
    ystar = np.linalg.solve(_dense_J(rp, ci, val, nb), b)
    rc, y, its, rel = s.linear_solve(1e-11)
    assert rc == 0 and 1 <= its, (rc, its)
    _, _, val2, b2, _ = s.ls.get()
    J2 = _dense_J(rp, ci, val2, nb)
    res = np.linalg.norm(b2 - J2 @ y) / np.linalg.norm(b2)
    assert res <= 1.0001e-11
    np.testing.assert_allclose(rel, res, rtol=1e-3)
    assert np.linalg.norm(y - ystar) <= 1e-11 * np.linalg.cond(J2) * np.linalg.norm(ystar)
    s2 = _system(oracle_lib, c, 60, tile_x=tile[0], tile_y=tile[1], amg_coarse_max=coarse, krylov=0)
    rc2, y2, its2, rel2 = s2.linear_solve(1e-11)
    assert rc2 == 0 and its <= its2, (its, its2)


def test_bicgstab_newton_run_matches_fgmres_run(oracle_lib):
    """Newton steps with CPR-BiCGSTAB reach the same converged states as with
    CPR-FGMRES (Algorithm 1 only needs ||A y - b|| <= eta ||b||): 3 steps of
    the 2,000-cell case, per-cell agreement far inside the 1e-6 bar."""
    c = I.case0()
    out = []
    for kry in (0, 1):
        s = oracle_lib.Sim(c, krylov=kry, max_lin=300)
        s.init_hydrostatic()
        assert s.advance(3) == 0
        out.append(s.get_state())
    assert np.max(np.abs(out[1][0] - out[0][0]) / out[0][0]) < 1e-8
    assert np.max(np.abs(out[1][1] - out[0][1])) < 1e-8


# ---- extended+i interpolation (the survey's stronger AMG option) ----
def _lap1d(n):
    """[-1 2 -1] with zero-row-sum (Neumann) ends, CSR."""
    M = np.zeros((n, n))
    for i in range(n):
        if i > 0: M[i, i - 1] = -1.0
        if i + 1 < n: M[i, i + 1] = -1.0
        M[i, i] = -M[i].sum()
    return M


def test_exti_reproduces_linear_interpolation_in_1d(oracle_lib):
    """On the 1D Laplacian with two F points between C points (C F F C F F C),
    direct interpolation can only copy the one strong C neighbour, while
    extended+i reaches the C point behind the strong F neighbour: the first
    F point gets 2/3 and 1/3, the second 1/3 and 2/3 -- linear
    interpolation, exact for the discrete harmonic functions of this
    operator."""
    M = _lap1d(7)
    rp, ci, v = _csr(M)
    cf = np.array([1, -1, -1, 1, -1, -1, 1], np.int8)
    prp, pci, pv = oracle_lib.interpolation(rp, ci, v, cf, interp=1)
    rows = {i: dict(zip(pci[prp[i]:prp[i + 1]].tolist(), pv[prp[i]:prp[i + 1]].tolist())) for i in range(7)}
    assert rows[0] == {0: 1.0} and rows[3] == {1: 1.0} and rows[6] == {2: 1.0}
    for i, (a, b) in ((1, (0, 1)), (2, (0, 1)), (4, (1, 2)), (5, (1, 2))):
        near, far = (2 / 3, 1 / 3) if i in (1, 4) else (1 / 3, 2 / 3)
        assert rows[i].keys() == {a, b}
        assert rows[i][a] == pytest.approx(near, rel=1e-14) and rows[i][b] == pytest.approx(far, rel=1e-14)
    # direct interpolation for comparison: one C point per F row
    prp, pci, pv = oracle_lib.interpolation(rp, ci, v, cf, interp=0)
    assert np.all(np.diff(prp)[[1, 2, 4, 5]] == 1)


@pytest.mark.parametrize("seed", range(4))
def test_exti_pattern_and_row_sums(oracle_lib, seed):
    """For the C/F split PMIS gives on a zero-row-sum M-matrix with weak and
    strong couplings: the pattern of each F row of P is exactly its strong C
    neighbours plus the strong C neighbours of its strong F neighbours, and
    every such row sums to 1 (the interpolation preserves constants, the
    near null space of the operator)."""
    M = _random_mmatrix(60, seed)
    M[np.diag_indices(60)] = 0.0
    M[np.diag_indices(60)] = -M.sum(axis=1)
    rp, ci, v = _csr(M)
    amg = oracle_lib.AMG(rp, ci, v, coarse_max=4, interp=1)
    lv = amg.level(0)
    cf, S = lv["cf"], lv["strong"]
    prp, pci, pv = oracle_lib.interpolation(rp, ci, v, cf, interp=1)
    np.testing.assert_array_equal(prp, lv["prp"])
    np.testing.assert_array_equal(pci, lv["pci"])
    cidx = np.cumsum(cf == 1) - 1
    n = 60
    strong = [set() for _ in range(n)]
    for i in range(n):
        for q in range(rp[i], rp[i + 1]):
            if S[q]:
                strong[i].add(int(ci[q]))
    for i in range(n):
        got = set(pci[prp[i]:prp[i + 1]].tolist())
        if cf[i] == 1:
            assert got == {int(cidx[i])}
            continue
        want = {j for j in strong[i] if cf[j] == 1}
        for k in strong[i]:
            if cf[k] == -1:
                want |= {j for j in strong[k] if cf[j] == 1}
        assert got == {int(cidx[j]) for j in want}, i
        if want:
            assert pv[prp[i]:prp[i + 1]].sum() == pytest.approx(1.0, rel=1e-12)
    assert any(len(set(pci[prp[i]:prp[i + 1]])) > sum(cf[j] == 1 for j in strong[i]) for i in range(n) if cf[i] == -1)


def test_exti_vcycle_converges_faster_than_direct(oracle_lib):
    """On the 3D Poisson problem the extended+i hierarchy's V-cycle reduces
    the error faster than direct interpolation's (the reason the survey
    lists it as the stronger option)."""
    rates = {}
    for interp in (0, 1):
        M = _poisson3d(12)
        rp, ci, v = _csr(M)
        amg = oracle_lib.AMG(rp, ci, v, coarse_max=32, interp=interp)
        n = M.shape[0]
        x = np.random.default_rng(5).standard_normal(n)
        e = x.copy()
        for _ in range(8):
            e_new = e - amg.apply(M @ e)
            rate = np.linalg.norm(e_new) / np.linalg.norm(e)
            e = e_new
        rates[interp] = rate
    assert rates[1] < rates[0] < 0.7, rates
