"""The device-side scheduler of the task graph (one persistent launch per
solve of an FP64 plan, Section 3 and Section 5.3) against the stage walk it
replaces, through the C ABI.

The updates land in each tile in the same (descending source) order and the
kernels' arithmetic is the same, so the two walks must agree bit for bit, and
two walks of the scheduler must agree with each other however its CTAs were
scheduled.  Both are also held to the oracle.  The scheduler's bounded
dependence wait is exercised with its counter withheld (it gives up and
reports ERR_TIMEOUT) and with the counter set, and a solve follows on the
same context.
"""
import os

import numpy as np
import pytest

import oracle
import pencilgen
from oracle import check

pytestmark = pytest.mark.gpu


def _solve(pevc, p, tile, sched, select=None, monkeypatch=None):
    monkeypatch.setenv("PEVC_SCHED", sched)
    plan = pevc.Plan(p.n, prec="fp64", tile=tile)
    try:
        V, sc, st = plan.solve(p.S, p.T, select=select, check=False)
        used = plan.stats[7]
    finally:
        plan.close()
    assert st == 0
    assert used == (1.0 if sched == "dag" else 0.0)
    return V, sc


@pytest.mark.parametrize("n,tile,stress", [(257, 32, False), (300, 64, True), (700, 128, False),
                                           (1030, 128, True), (2000, 64, False)])
def test_dag_matches_stage_walk_bitwise_and_oracle(pevc_lib, monkeypatch, n, tile, stress):
    p = pencilgen.make_pencil(n, 8100 + n + tile, stress=stress)
    Vd, scd = _solve(pevc_lib, p, tile, "dag", monkeypatch=monkeypatch)
    Vd2, scd2 = _solve(pevc_lib, p, tile, "dag", monkeypatch=monkeypatch)
    Vs, scs = _solve(pevc_lib, p, tile, "stage", monkeypatch=monkeypatch)
    assert np.isfinite(Vd).all()
    assert np.array_equal(Vd, Vd2) and np.array_equal(scd, scd2), "the scheduler is not deterministic"
    assert np.array_equal(Vd, Vs) and np.array_equal(scd, scs), "scheduler and stage walk differ"
    ost, Vo, sco, m = oracle.evc(p.S, p.T, nthreads=os.cpu_count() or 1)
    kinds, pos = check.column_kinds(p.block)
    err, _ = check.compare_normalised(Vo, Vd, kinds)
    _, blk, a, b, beta, _ = oracle.eigpairs(p.S, p.T)
    res = check.residuals(p.S, p.T, Vd, kinds, pos, a, b, beta).max() / (n * check.U)
    print(f"dag n={n} tile={tile} stress={stress}: err {err:.3e} resid/(nu) {res:.3e}")
    assert res <= 100.0
    assert err <= (1e-6 if stress else 1e-10)


def test_dag_selection_and_empty_column_tiles(pevc_lib, monkeypatch):
    """A selection that leaves whole column tiles without eigenvectors (no
    tasks for them) and pairs on sub-chunk edges."""
    n = 600
    p = pencilgen.make_pencil(n, 8201)
    sel = np.zeros(n, dtype=np.int32)
    sel[40:90] = 1
    sel[300:310] = 1
    sel[590:] = 1
    Vd, scd = _solve(pevc_lib, p, 64, "dag", select=sel, monkeypatch=monkeypatch)
    Vs, scs = _solve(pevc_lib, p, 64, "stage", select=sel, monkeypatch=monkeypatch)
    assert np.array_equal(Vd, Vs) and np.array_equal(scd, scs)
    ost, Vo, sco, m = oracle.evc(p.S, p.T, select=sel)
    kinds, _ = check.column_kinds(p.block, sel)
    assert Vd.shape == Vo.shape
    assert check.compare_normalised(Vo, Vd, kinds)[0] <= 1e-10


def test_scheduler_wait_runs_out_and_context_survives(pevc_lib):
    plan = pevc_lib.Plan(200, prec="fp64", device_walk=True)
    try:
        h = plan.h
        assert pevc_lib.pevc_scheduler_selftest(h, 0, 2_000_000) == 0
        assert pevc_lib.pevc_scheduler_selftest(h, 1, 2_000_000) == pevc_lib.ERR_TIMEOUT
        assert pevc_lib.pevc_scheduler_selftest(h, 0, 2_000_000) == 0
        assert pevc_lib.pevc_scheduler_selftest(h, 1, 0) == -3
        assert pevc_lib.pevc_scheduler_selftest(h, 2, 1000) == -2
        p = pencilgen.make_pencil(200, 8301)
        V, sc, st = plan.solve(p.S, p.T)
        assert st == 0 and np.isfinite(V).all()
        assert plan.stats[7] == 1.0
    finally:
        plan.close()
