"""Properties of the seeded input generator (CPU): the structure both the
oracle and the GPU path rely on, and the workload recipe's statistics."""
import numpy as np
import pytest

import pencilgen


@pytest.mark.parametrize("stress", [False, True])
def test_real_schur_structure(stress):
    p = pencilgen.make_pencil(300, 4242, stress=stress)
    n = p.n
    S, T, blk = p.S, p.T, p.block
    assert S.shape == T.shape == (n, n)
    assert np.isfinite(S).all() and np.isfinite(T).all()
    # nothing below the quasi-diagonal of S, nothing below the diagonal of T
    for i in range(n):
        for j in range(i - 1):
            assert S[i, j] == 0.0
        assert np.all(T[i, :i] == 0.0)
    for c in range(n):
        if blk[c] == 1:                       # first row of a 2x2 block
            assert blk[c + 1] == 2
            assert S[c + 1, c] != 0.0
            assert T[c, c + 1] == 0.0 and T[c + 1, c] == 0.0
            assert T[c, c] > 0 and T[c + 1, c + 1] > 0
            # a complex pair: the discriminant of det(S_jj - lambda T_jj) is negative
            t1, t2 = T[c, c], T[c + 1, c + 1]
            s11, s12, s21, s22 = S[c, c], S[c, c + 1], S[c + 1, c], S[c + 1, c + 1]
            half = 0.5 * (s11 / t1 - s22 / t2)
            assert half * half + s12 * s21 / (t1 * t2) < 0.0
        elif blk[c] == 0:
            assert c == n - 1 or S[c + 1, c] == 0.0


def test_block_pattern_statistics():
    p = pencilgen.make_pencil(20000 // 4, 99, stress=False)
    frac = np.mean(p.block != 0)              # rows inside 2x2 blocks
    assert 0.45 < frac < 0.55


def test_seeded_and_reproducible():
    a = pencilgen.make_pencil(120, 7)
    b = pencilgen.make_pencil(120, 7)
    c = pencilgen.make_pencil(120, 8)
    assert np.array_equal(a.S, b.S) and np.array_equal(a.T, b.T)
    assert not np.array_equal(a.S, c.S)
    assert pencilgen.config_seed(3) == pencilgen.config_seed(3, 0)
    assert pencilgen.config_seed(3, 1) != pencilgen.config_seed(3, 0)


def test_stress_variant_scales():
    # n = 1024: 120 strictly upper tiles on the 64 x 64 generator grid, 5 % of them scaled
    p = pencilgen.make_pencil(1024, 11, stress=True)
    q = pencilgen.make_pencil(1024, 11, stress=False)
    # T's diagonal scaled by 2^-40, and some off-diagonal tiles carry entries near 1e100
    assert np.max(np.abs(np.diag(p.T))) < 2.0 ** -38
    assert np.max(np.abs(np.diag(q.T))) > 0.4
    assert np.max(np.abs(np.triu(p.S, 2))) > 1e90


def test_batch_orders_range():
    orders = pencilgen.batch_orders()
    assert len(orders) == pencilgen.BATCH_COUNT
    assert orders.min() >= pencilgen.BATCH_NMIN and orders.max() <= pencilgen.BATCH_NMAX
