"""pevc_solve_batched: pencils of uneven orders (plain and stress, with and
without a selection, an empty one and an invalid one) in one call, run
concurrently on the plan's child workspaces.  Every pencil must give exactly
what a single pevc_solve gives on the same plan settings (the kernels are
deterministic), and match the oracle within the parity tolerance."""
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


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("bf16x5", 1e-8)])
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
