"""The entry point without device allocation (pevc_solve_static) against the
plan-based one (pevc_solve), both through the C ABI.

Two calls in a row on pencils of different orders (and a selection on the
second), each compared with an FP64 plan's output on the same input:
componentwise within the FP64 parity tolerance after normalisation, equal
column counts and scale exponents; the second is also held to the FP64 oracle
directly.  The second call also checks that nothing
of the first call's contents in the shared scratch array leaks into it.
"""
import numpy as np
import pytest

import oracle
import pencilgen
from oracle import check

pytestmark = pytest.mark.gpu

TOL = 1e-10


def _plan_solve(pevc, S, T, select=None):
    plan = pevc.Plan(S.shape[0], prec="fp64")
    try:
        V, sc, st = plan.solve(S, T, select=select, check=False)
    finally:
        plan.close()
    return V, sc, st


def _static_solve(pevc, S, T, select=None):
    import torch
    n = S.shape[0]
    St = pevc.to_device_colmajor(S)
    Tt = pevc.to_device_colmajor(T)
    V = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")   # column-major storage
    scale = torch.full((n,), -7, dtype=torch.int32, device="cuda")
    sel = None
    if select is not None:
        sel = torch.as_tensor(np.asarray(select, dtype=np.int32)).to("cuda")
    stream = torch.cuda.current_stream()
    st, m = pevc.pevc_solve_static(St.data_ptr(), n, Tt.data_ptr(), n, n,
                                   sel.data_ptr() if sel is not None else 0,
                                   V.data_ptr(), n, scale.data_ptr(), 0, stream.cuda_stream)
    torch.cuda.synchronize()
    Vh = V[:m].cpu().numpy().T if m else np.zeros((n, 0))
    return np.asfortranarray(Vh[:n, :m]), scale[:m].cpu().numpy(), st


def _agree(Vp, scp, Vs, scs, block, select=None):
    assert Vs.shape == Vp.shape
    assert np.isfinite(Vs).all()
    kinds, _ = check.column_kinds(block, select)
    err, _ = check.compare_normalised(Vp, Vs, kinds)
    assert err <= TOL, f"max componentwise difference {err:.3e}"
    assert np.array_equal(scs, scp)
    return err


def test_static_entry_matches_plan_on_two_calls(pevc_lib):
    p1 = pencilgen.make_pencil(300, 9301)
    p2 = pencilgen.make_pencil(200, 9302)
    rng = np.random.default_rng(9303)
    sel2 = (rng.random(200) < 0.5).astype(np.int32)

    Vs1, scs1, sts1 = _static_solve(pevc_lib, p1.S, p1.T)
    Vs2, scs2, sts2 = _static_solve(pevc_lib, p2.S, p2.T, select=sel2)
    assert sts1 == 0 and sts2 == 0

    Vp1, scp1, stp1 = _plan_solve(pevc_lib, p1.S, p1.T)
    Vp2, scp2, stp2 = _plan_solve(pevc_lib, p2.S, p2.T, select=sel2)
    assert stp1 == 0 and stp2 == 0

    e1 = _agree(Vp1, scp1, Vs1, scs1, p1.block)
    e2 = _agree(Vp2, scp2, Vs2, scs2, p2.block, sel2)
    # and directly against the FP64 oracle
    ost, Vo, sco, mo = oracle.evc(p2.S, p2.T, select=sel2)
    assert ost == 0
    eo, _ = check.compare_normalised(Vo, Vs2, check.column_kinds(p2.block, sel2)[0])
    assert eo <= TOL and np.all(np.abs(scs2.astype(np.int64) - sco.astype(np.int64)) <= 1)
    print(f"static vs plan: {e1:.3e}, {e2:.3e}; vs oracle {eo:.3e}")


def test_static_entry_rejects_orders_above_its_maximum(pevc_lib):
    n = pevc_lib.STATIC_N_MAX + 1
    st, m = pevc_lib.pevc_solve_static(0, n, 0, n, n, 0, 0, n, 0)
    assert st == pevc_lib.ERR_TOO_LARGE and m == 0
    assert "PEVC_STATIC_N_MAX" in pevc_lib.pevc_strerror(st)
