"""pevc_solve_batched: pencils of uneven orders (plain and stress, with and
without a selection, an empty one and an invalid one) in one call.  FP64
plans run the whole batch on the device-side scheduler (the task graphs of
all pencils in one persistent launch per wave); split plans run the pencils
concurrently on child workspaces.  Every pencil must give exactly what a
single pevc_solve gives on the same plan settings (the kernels are
deterministic, and the scheduler applies the updates in the stage walk's
order), and match the oracle within the parity tolerance."""
import os

import numpy as np
import pytest

import oracle
import pencilgen
from oracle import check

pytestmark = pytest.mark.gpu


def _bad_pencil(n=20, seed=7):
    p = pencilgen.make_pencil(n, seed)
    S = p.S.copy()
    S[5, 4] = 0.5      # subdiagonal entries at rows 4 and 5: adjacent 2x2 blocks
    S[6, 5] = 0.25
    return S, p.T.copy()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("bf16x5", 1e-8), ("fp8x4", 1e-8)])
def test_batched_matches_single_solves_and_oracle(pevc_lib, prec, tol):
    orders = [1, 7, 40, 100, 0, 257, 300, 129, 64, 513, 33, 200]
    pencils, selects, metas = [], [], []
    for q, n in enumerate(orders):
        stress = (q % 3 == 2)
        p = pencilgen.make_pencil(n, 6000 + q, stress=stress) if n > 0 else None
        if p is None:
            pencils.append((np.zeros((0, 0)), np.zeros((0, 0))))
            metas.append(None)
            selects.append(None)
            continue
        pencils.append((p.S, p.T))
        metas.append(p)
        sel = None
        if q % 4 == 1:
            sel = (np.arange(n) % 3 == 0).astype(np.int32)
        selects.append(sel)
    bad_S, bad_T = _bad_pencil()
    pencils.append((bad_S, bad_T))
    metas.append("bad")
    selects.append(None)
    nmax = max(orders + [20])
    plan = pevc_lib.Plan(nmax, prec=prec, batch_max=len(pencils))
    single = pevc_lib.Plan(nmax, prec=prec)
    try:
        st, out = plan.solve_batched(pencils, selects)
        assert st == 0
        for b, (meta, (V, sc, stb)) in enumerate(zip(metas, out)):
            if meta is None:
                assert stb == 0 and V.shape[1] == 0
                continue
            if meta == "bad":
                assert stb == pevc_lib.ERR_NOT_SCHUR
                continue
            assert stb == 0, (b, stb)
            V1, sc1, st1 = single.solve(meta.S, meta.T, select=selects[b], check=False)
            assert st1 == 0
            assert np.array_equal(V, V1), b
            assert np.array_equal(sc, sc1), b
            ost, Vo, sco, m = oracle.evc(meta.S, meta.T, select=selects[b], nthreads=os.cpu_count() or 1)
            kinds, pos = check.column_kinds(meta.block, selects[b])
            err, _ = check.compare_normalised(Vo, V, kinds)
            assert np.isfinite(V).all()
            if not meta.stress:
                assert err <= tol, (b, err)
            st_, blk, a, bb, beta, _ = oracle.eigpairs(meta.S, meta.T)
            res = check.residuals(meta.S, meta.T, V, kinds, pos, a, bb, beta)
            assert res.max() <= 100 * max(meta.n, 1) * check.U, b
    finally:
        plan.close()
        single.close()


_ORACLE_CACHE = {}


def _config4_oracle(pencils):
    """The oracle's eigenvectors of the plain (even-index) pencils of the
    batched workload, computed once per session."""
    if not _ORACLE_CACHE:
        threads = os.cpu_count() or 1
        for b in range(0, len(pencils), 2):
            st, Vo, sco, m = oracle.evc(pencils[b].S, pencils[b].T, nthreads=threads)
            assert st == 0
            _ORACLE_CACHE[b] = (Vo, sco)
    return _ORACLE_CACHE


_SENS_CACHE = {}


def _sensitivity(p, b):
    """Per eigenvector: check.perturbation_sensitivity of the oracle's vectors
    (cached per pencil)."""
    if b not in _SENS_CACHE:
        kinds, _ = check.column_kinds(p.block)
        evc = lambda S, T: oracle.evc(S, T, nthreads=os.cpu_count() or 1)
        _SENS_CACHE[b] = check.perturbation_sensitivity(p.S, p.T, _ORACLE_CACHE[b][0], kinds, evc, 7700 + b)
    return _SENS_CACHE[b]


# per eigenvector: err <= max(flat bar, 16 * digits factor * sensitivity); the
# split path's operands carry 40 bits instead of 53 (factor 2^13)
_BARS = {"fp64": (1e-10, 1.0), "bf16x5": (1e-8, 2.0 ** 13)}


@pytest.mark.parametrize("prec", ["fp64", "bf16x5"])
def test_batched_config4_workload(pevc_lib, prec):
    """The batched workload at its stated size: 1024 pencils, n log-uniform in
    [32, 2048], odd indices stress pencils, all eigenvectors, one call.  Every
    pencil: finite, residual <= 100 n u over every column (also per 64-row
    block with the block's own norms); every eigenvector of the plain pencils
    against the oracle componentwise, within the flat bar or, for the few
    ill-conditioned ones, within 16x its measured sensitivity (times 2^13 for
    the 40-bit slices).  The per-pencil error distribution is printed."""
    import sys
    import torch
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    orders = pencilgen.batch_orders()
    assert orders.size == 1024 and orders.min() >= 32 and orders.max() <= 2048
    pencils = [pencilgen.batch_pencil(b, int(n)) for b, n in enumerate(orders)]
    assert all(p.stress == bool(b % 2) for b, p in enumerate(pencils))
    batch = bench.Batch(pencils, pevc_lib)
    plan = pevc_lib.Plan(int(orders.max()), prec=prec, batch_max=len(pencils))
    try:
        m_out = batch.solve(plan)
    finally:
        plan.close()
    torch.cuda.synchronize()
    assert m_out == [int(n) for n in orders]
    res, res_rb, finite = bench.batch_accuracy(batch)
    assert finite.all()
    ref = _config4_oracle(pencils)
    flat, digits = _BARS[prec]
    errs, dsc, over, worst_ratio = [], 0, 0, 0.0
    for b, (Vo, sco) in ref.items():
        Vg = batch.view(batch.V, b).cpu().numpy().T
        kinds, _ = check.column_kinds(pencils[b].block)
        err, per = check.compare_normalised(Vo, Vg, kinds)
        errs.append(err)
        if err > flat:
            over += 1
            bound = np.maximum(flat, 16.0 * digits * _sensitivity(pencils[b], b))
            worst_ratio = max(worst_ratio, float((per / bound).max()))
            assert np.all(per <= bound), (b, float(per.max()), float(bound[np.argmax(per / bound)]))
        sc = batch.scale[int(batch.soff[b]):int(batch.soff[b + 1])].cpu().numpy()
        dsc = max(dsc, int(np.abs(sc.astype(np.int64) - sco.astype(np.int64)).max()))
    errs = np.asarray(errs)
    q = lambda a: ", ".join(f"{x:.2e}" for x in np.percentile(a, [50, 90, 99, 100]))
    print(f"config4 {prec}: residual/(n u) p50/p90/p99/max {q(res)}; per-block {q(res_rb)}; "
          f"plain pencils' error vs oracle {q(errs)}; {over} pencils above {flat:.0e}, each within its "
          f"conditioning bound (largest error / bound {worst_ratio:.2f}); scale exponents within {dsc}")
    assert res.max() <= 100.0 and res_rb.max() <= 100.0
    assert dsc <= 1


def test_batched_fp64_waves_match_single_solves(pevc_lib, monkeypatch):
    """A workspace budget that holds only a few pencils at a time: the batch
    runs as several waves of the scheduler, and every pencil still equals its
    single solve (which walks stage by stage from the host) bit for bit."""
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    orders = [300, 64, 500, 1, 257, 400, 129, 450]
    pencils = [pencilgen.make_pencil(n, 6600 + q, stress=bool(q % 2)) for q, n in enumerate(orders)]
    monkeypatch.setenv("PEVC_BATCH_BYTES", "4000000")          # two pencils of order 500 per wave
    plan = pevc_lib.Plan(500, prec="fp64", tile=64, batch_max=len(pencils))
    single = pevc_lib.Plan(500, prec="fp64", tile=64)
    try:
        st, out = plan.solve_batched([(p.S, p.T) for p in pencils])
        assert st == 0
        for p, (V, sc, stb) in zip(pencils, out):
            assert stb == 0
            V1, sc1, st1 = single.solve(p.S, p.T, check=False)
            assert st1 == 0 and single.stats[7] == 0.0        # a single pencil: the stage walk
            assert np.array_equal(V, V1) and np.array_equal(sc, sc1)
    finally:
        plan.close()
        single.close()
