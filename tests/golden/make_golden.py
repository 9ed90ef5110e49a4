"""Write the exact-eigenvector fixtures of tests/golden/.

Each fixture is a tiny pencil with dyadic-rational entries (exact in
binary64) together with its eigenvectors computed in exact Gaussian-rational
arithmetic by ``oracle.exact`` (kernel of beta*S - alpha*T, Section 2 of the
paper: the tall equation and its Lemma), normalised at the first entry of
largest modulus.  Only ``oracle/`` and ``pencilgen`` are used.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys
from fractions import Fraction

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import pencilgen  # noqa: E402
from oracle import exact  # noqa: E402

# (name, order, seed, rows whose 1x1 eigenvalue is made infinite)
CASES = [
    ("exact_n4_s11", 4, 11, []),
    ("exact_n6_s5", 6, 5, []),
    ("exact_n8_s3", 8, 3, []),
    ("exact_n8_s21_inf", 8, 21, ["first1x1"]),
    ("exact_n7_s8_real", 7, 8, None),
]


def make(name, n, seed, infinite):
    ep = pencilgen.exact_pencil(n, seed, two_by_two=infinite is not None)
    if infinite:
        r = ep.block.index(0)
        ep.T[r][r] = Fraction(0)
        ep.S[r][r] = Fraction(3, 2)
    V, dims = exact.exact_eigenvectors(ep)
    assert all(d == 1 for d in dims), dims
    lines = [f"# {name}: pencil order {n}, generator seed {seed}; exact eigenvectors",
             "# (kernel of beta*S - alpha*T over Q(i), normalised at the first entry of",
             "# largest modulus; paper Section 2, tall equation and Lemma)",
             f"n {n}", "block " + " ".join(str(b) for b in ep.block)]
    for nm, M in (("S", ep.S), ("T", ep.T)):
        for i in range(n):
            lines.append(f"{nm} {i} " + " ".join(str(x) for x in M[i]))
    for c in range(n):
        col = V[:, c]
        lines.append(f"V {c} " + " ".join(f"{float(z.real)!r},{float(z.imag)!r}" for z in col))
    with open(os.path.join(HERE, name + ".txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


# Complex triangular pencils (the extension to complex data, Section 7):
# (name, order, seed, last eigenvalue infinite)
CPLX_CASES = [
    ("cexact_n5_s7", 5, 7, False),
    ("cexact_n8_s13", 8, 13, False),
    ("cexact_n6_s29_inf", 6, 29, True),
]


def make_cplx(name, n, seed, infinite):
    ep = pencilgen.exact_complex_pencil(n, seed, infinite=infinite)
    V, dims = exact.exact_complex_eigenvectors(ep)
    assert all(d == 1 for d in dims), dims
    lines = [f"# {name}: complex triangular pencil of order {n}, generator seed {seed};",
             "# exact eigenvectors (kernel of beta*S - alpha*T, (alpha, beta) = (S_cc, T_cc),",
             "# over Q(i), normalised at the first entry of largest modulus; paper Section 2,",
             "# tall equation and Lemma, for complex data as in Section 7)",
             f"n {n}"]
    for nm, M in (("S", ep.S), ("T", ep.T)):
        for i in range(n):
            lines.append(f"{nm} {i} " + " ".join(f"{re},{im}" for re, im in M[i]))
    for c in range(n):
        col = V[:, c]
        lines.append(f"V {c} " + " ".join(f"{float(z.real)!r},{float(z.imag)!r}" for z in col))
    with open(os.path.join(HERE, name + ".txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


def load_cplx(path):
    """Parse a complex fixture: returns (S, T, V), all complex n x n."""
    import numpy as np
    S = T = V = None
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            tok = line.split()
            if tok[0] == "n":
                n = int(tok[1])
                S = np.zeros((n, n), dtype=complex, order="F")
                T = np.zeros((n, n), dtype=complex, order="F")
                V = np.zeros((n, n), dtype=complex)
            elif tok[0] in ("S", "T"):
                i = int(tok[1])
                M = S if tok[0] == "S" else T
                M[i, :] = [complex(float(Fraction(p.split(",")[0])), float(Fraction(p.split(",")[1])))
                           for p in tok[2:]]
            elif tok[0] == "V":
                c = int(tok[1])
                V[:, c] = [complex(float(p.split(",")[0]), float(p.split(",")[1])) for p in tok[2:]]
    return S, T, V


def load(path):
    """Parse a fixture: returns (S, T, block, V) with V complex n x n."""
    import numpy as np
    S = T = V = None
    block = None
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            tok = line.split()
            if tok[0] == "n":
                n = int(tok[1])
                S = np.zeros((n, n), order="F")
                T = np.zeros((n, n), order="F")
                V = np.zeros((n, n), dtype=complex)
            elif tok[0] == "block":
                block = [int(x) for x in tok[1:]]
            elif tok[0] in ("S", "T"):
                i = int(tok[1])
                M = S if tok[0] == "S" else T
                M[i, :] = [float(Fraction(x)) for x in tok[2:]]
            elif tok[0] == "V":
                c = int(tok[1])
                V[:, c] = [complex(float(p.split(",")[0]), float(p.split(",")[1])) for p in tok[2:]]
    return S, T, block, V


if __name__ == "__main__":
    for case in CASES:
        make(*case)
    for case in CPLX_CASES:
        make_cplx(*case)
    print("wrote", len(CASES) + len(CPLX_CASES), "fixtures")
