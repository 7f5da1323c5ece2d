"""The ensemble driver (sim_batch_*): many independent models on one GPU.

Members share nothing, so (1) every member's run matches the CPU oracle's
run of the same model with the whole-run tolerances (per-cell |dp|/p and
|ds_w| <= 1e-6, Newton counts within +-1 per step), and (2) the GPU results do
not depend on how members are scheduled: a batch run is bit-identical to
running each member alone, for any worker count, and before or after the
worker-count autotuner (which must restore every state it touches).
"""
import numpy as np
import pytest

import oracle
import paper_1701_06254_gb300 as R
from paper_1701_06254_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TINY = dict(size_lo=(5, 4, 2), size_hi=(13, 11, 4))


def _members(m, seed0=4100, **kw):
    return I.ensemble(m, seed0=seed0, **{**TINY, **kw})


def _states(sims):
    return [s.get_state() for s in sims]


def test_batch_members_match_oracle():
    """Five members of different sizes (ragged RAS tiles), three workers,
    two 10-day steps: each member against the oracle's run of that model."""
    cases = _members(5)
    b = R.Batch(cases, workers=3)
    b.init_hydrostatic()
    for step in range(2):
        n_before = [m.stats()["newton"] for m in b.members]
        b.advance(1)
        for k, (case, mem) in enumerate(zip(cases, b.members)):
            o = _oracles[k] if step else None
            if step == 0:
                o = oracle.Sim(case)
                o.init_hydrostatic()
                _oracles[k] = o
            n0 = o.stats()["newton"]
            assert o.advance(1) == 0
            po, so, pbo, to = o.get_state()
            pg, sg, pbg, tg = mem.get_state()
            assert tg == to
            assert np.max(np.abs(pg - po) / np.abs(po)) <= 1e-6, (k, step)
            assert np.max(np.abs(sg - so)) <= 1e-6, (k, step)
            dn_g = mem.stats()["newton"] - n_before[k]
            dn_o = o.stats()["newton"] - n0
            assert abs(dn_g - dn_o) <= 1, (k, step, dn_g, dn_o)


_oracles = {}


def test_batch_is_bit_identical_to_single_runs_for_any_worker_count():
    cases = _members(6, seed0=4200)
    ref = []
    for c in cases:
        s = R.Sim(c, precision=R.PREC_MIXED_BF16)
        s.init_hydrostatic()
        s.advance(2)
        ref.append(s.get_state())
    for workers in (1, 4):
        b = R.Batch(cases, workers=workers, precision=R.PREC_MIXED_BF16)
        b.init_hydrostatic()
        stats = b.advance(2)
        for k, (mem, r) in enumerate(zip(b.members, ref)):
            got = mem.get_state()
            for a, e in zip(got[:3], r[:3]):
                np.testing.assert_array_equal(a, e, err_msg=f"member {k}, {workers} workers")
            assert got[3] == r[3]
            assert stats[k]["steps"] == 2


def test_autotune_restores_states_exactly():
    cases = _members(6, seed0=4300)
    plain = R.Batch(cases, workers=2)
    plain.init_hydrostatic()
    plain.advance(1)
    expect = _states(plain.members)
    tuned = R.Batch(cases, workers=2)
    tuned.init_hydrostatic()
    before = _states(tuned.members)
    chosen, secs = tuned.autotune(candidates=(1, 2, 3), sample=4)
    assert chosen in (1, 2, 3) and tuned.workers == chosen
    assert all(v > 0 for v in secs.values())
    for k, (st0, mem) in enumerate(zip(before, tuned.members)):
        now = mem.get_state()
        for a, e in zip(now[:3], st0[:3]):
            np.testing.assert_array_equal(a, e, err_msg=f"member {k}")
        assert mem.stats()["steps"] == 0 and mem.stats()["newton"] == 0
    tuned.advance(1)
    for k, (mem, e) in enumerate(zip(tuned.members, expect)):
        for a, b in zip(mem.get_state()[:3], e[:3]):
            np.testing.assert_array_equal(a, b, err_msg=f"member {k}")


def test_batch_create_reports_the_failing_member():
    cases = _members(3, seed0=4400)
    bad = cases[1]
    bad.wells[0].perf_cells = [bad.n + 5]           # perforation outside the grid
    with pytest.raises(R.SimError) as e:
        R.Batch(cases)
    assert e.value.code == 1 and "member 1" in str(e.value)
