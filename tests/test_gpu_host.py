"""pevc_solve_host: the solve on host arrays, with S and T streamed to the
device by column blocks behind the bottom-up walk (each block's pre-pass,
slices and tips on its arrival, the lower triangles never copied).

The walk is the one pevc_solve runs on device arrays, so the two entry points
must give the same bits: for FP64 and split BF16x5 plans, ragged and stress
pencils, a selection, pinned torch tensors and plain numpy arrays.  The
eigenvalues' pre-scale is taken from the blocks seen so far; a pencil whose
largest entry sits in the first column block (the last to arrive) at 2^1005
changes the pre-scale late, and the solve that the call then runs again
must still match.  The result is also held to the oracle and the residual
bar, every entry of the host output is written (it starts as NaN; the zeros
below each column tile come from host threads), and the bytes copied each
way are checked against the upper tiles.
"""
import os

import numpy as np
import pytest

import oracle
import pencilgen
from oracle import check

pytestmark = pytest.mark.gpu


def _device_solve(pevc, p, prec, tile, sel=None):
    plan = pevc.Plan(p.n, prec=prec, tile=tile)
    try:
        V, sc, st = plan.solve(p.S, p.T, select=sel, check=False)
    finally:
        plan.close()
    return V, sc, st


def _host_solve(pevc, p, prec, tile, sel=None, pinned=True):
    import torch
    n = p.n
    plan = pevc.Plan(n, prec=prec, tile=tile)
    try:
        if pinned:
            Sh = torch.from_numpy(np.ascontiguousarray(p.S.T)).pin_memory()
            Th = torch.from_numpy(np.ascontiguousarray(p.T.T)).pin_memory()
            Vh = torch.full((n, n), float("nan"), dtype=torch.float64).pin_memory()   # every entry must be written
            sch = torch.zeros(n, dtype=torch.int32).pin_memory()
        else:
            Sh, Th = np.asfortranarray(p.S), np.asfortranarray(p.T)
            Vh, sch = np.full((n, n), np.nan, order="F"), np.zeros(n, dtype=np.int32)
        st, m = plan.solve_host(Sh, Th, Vh, sch, select=sel)
        nbytes = plan.host_bytes
    finally:
        plan.close()
    if pinned:
        V = Vh.numpy().T[:, :m].copy()      # row-major storage of V^T
        sc = sch.numpy()[:m].copy()
    else:
        V, sc = Vh[:, :m].copy(), sch[:m].copy()
    return V, sc, st, nbytes


@pytest.mark.parametrize("prec,tile,n,stress,every,pinned", [
    ("fp64", 64, 1030, False, 1, True),
    ("fp64", 96, 700, True, 3, False),
    ("bf16x5", 128, 1030, False, 1, True),
    ("bf16x5", 128, 2000, True, 1, True),
    ("bf16x5", 128, 513, False, 4, False),
    ("fp8x4", 128, 700, False, 1, True),       # the correction sweep: copied whole, then solved
])
def test_host_solve_matches_device_solve_bitwise(pevc_lib, prec, tile, n, stress, every, pinned):
    p = pencilgen.make_pencil(n, 9900 + n + tile, stress=stress)
    sel = None if every == 1 else (np.arange(n) % every != 1).astype(np.int32)
    Vd, scd, std = _device_solve(pevc_lib, p, prec, tile, sel)
    Vh, sch, sth, (h2d, d2h) = _host_solve(pevc_lib, p, prec, tile, sel, pinned)
    assert std == 0 and sth == 0
    assert Vh.shape == Vd.shape
    assert np.array_equal(Vh, Vd) and np.array_equal(sch, scd), "host and device entry points differ"
    m = Vd.shape[1]
    # the upper tiles of S and T only, and V with its scales back
    assert n * (n + 1) * 8 <= h2d < 2 * n * n * 8
    assert m * 8 <= d2h - m * 4 < m * n * 8    # the rows above each column tile's end
    ost, Vo, sco, mo = oracle.evc(p.S, p.T, select=sel, nthreads=os.cpu_count() or 1)
    kinds, pos = check.column_kinds(p.block, sel)
    err, _ = check.compare_normalised(Vo, Vh, kinds)
    _, blk, a, b, beta, _ = oracle.eigpairs(p.S, p.T)
    res = check.residuals(p.S, p.T, Vh, kinds, pos, a, b, beta).max() / (n * check.U)
    print(f"host solve {prec} n={n} stress={stress}: err {err:.3e} resid/(nu) {res:.3e} h2d {h2d / 1e6:.1f} MB")
    assert res <= 100.0
    assert err <= (1e-6 if stress else (1e-10 if prec == "fp64" else 1e-8))


@pytest.mark.parametrize("prec,tile", [("fp64", 64), ("bf16x5", 128)])
def test_host_solve_late_prescale_is_redone(pevc_lib, prec, tile):
    """The largest entry (2^1005) in column block 0, which arrives last: the
    blocks before it take their pre-scale from a smaller maximum, so the call
    must detect the change and solve again on the copied data."""
    n = 600
    p = pencilgen.make_pencil(n, 9950)
    p.S[0, 5] = 2.0 ** 1005
    Vd, scd, std = _device_solve(pevc_lib, p, prec, tile)
    Vh, sch, sth, _ = _host_solve(pevc_lib, p, prec, tile)
    assert std == sth
    if std == 0:
        assert np.array_equal(Vh, Vd) and np.array_equal(sch, scd)
