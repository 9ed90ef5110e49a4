"""Failure detection without a GPU fault: the library's bounded device wait
(an mbarrier wait limited in SM clock cycles, the primitive every wait of the
tcgen05 update uses) gives up when its arrival is
withheld, reports ERR_TIMEOUT through the status word, and leaves the context
usable for the next solve."""
import numpy as np
import pytest

import pencilgen

pytestmark = pytest.mark.gpu


def test_watchdog_wait_runs_out_and_context_survives(pevc_lib):
    """A bounded device wait whose arrival is withheld gives up and reports
    ERR_TIMEOUT; the context stays usable for a solve afterwards."""
    plan = pevc_lib.Plan(64, prec="fp64")
    try:
        h = plan.h
        assert pevc_lib.pevc_watchdog_selftest(h, 0, 2_000_000) == 0
        assert pevc_lib.pevc_watchdog_selftest(h, 1, 2_000_000) == pevc_lib.ERR_TIMEOUT
        assert pevc_lib.pevc_watchdog_selftest(h, 1, 0) == -3
        assert pevc_lib.pevc_watchdog_selftest(h, 2, 1000) == -2
        p = pencilgen.make_pencil(64, 7700)
        V, sc, st = plan.solve(p.S, p.T)
        assert st == 0 and np.isfinite(V).all()
    finally:
        plan.close()
