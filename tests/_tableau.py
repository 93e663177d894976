"""Exact rational Butcher tableau of RK4(3)5[2R+]C, read from the golden fixture.

Test helper: builds A, b, bhat, c as Fractions from the published coefficients so
that stability polynomials and order conditions can be evaluated exactly, with no
code from the oracle or the GPU path.
"""
from fractions import Fraction as Fr
import os

_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lsrk_rk4_3_5_2Rplus_C.txt")


def load():
    vals = {}
    with open(_GOLDEN) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            name, num, den = line.split()
            vals[name] = Fr(int(num), int(den))
    sub = [vals["a21"], vals["a32"], vals["a43"], vals["a54"]]
    b = [vals[f"b{i}"] for i in range(1, 6)]
    bh = [vals[f"bh{i}"] for i in range(1, 6)]
    s = 5
    A = [[Fr(0)] * s for _ in range(s)]
    for i in range(1, s):
        for j in range(i - 1):
            A[i][j] = b[j]
        A[i][i - 1] = sub[i - 1]
    c = [sum(A[i]) for i in range(s)]
    return {"sub": sub, "b": b, "bh": bh, "A": A, "c": c}


def stability(z, w, A):
    """R(z) = 1 + z w^T (I - z A)^{-1} 1 for the explicit tableau, exactly in Fractions
    (z may be a Fraction or a complex pair handled by the caller)."""
    s = len(w)
    # stage amplification g = (I - zA)^{-1} 1 by forward substitution (A strictly lower)
    g = []
    for i in range(s):
        gi = 1 + z * sum(A[i][j] * g[j] for j in range(i))
        g.append(gi)
    return 1 + z * sum(w[i] * g[i] for i in range(s))


def order_residuals(w, A, c):
    s = len(w)
    r = {}
    r["1"] = sum(w) - 1
    r["c"] = sum(w[i] * c[i] for i in range(s)) - Fr(1, 2)
    r["c2"] = sum(w[i] * c[i] ** 2 for i in range(s)) - Fr(1, 3)
    r["Ac"] = sum(w[i] * A[i][j] * c[j] for i in range(s) for j in range(s)) - Fr(1, 6)
    r["c3"] = sum(w[i] * c[i] ** 3 for i in range(s)) - Fr(1, 4)
    r["cAc"] = sum(w[i] * c[i] * A[i][j] * c[j] for i in range(s) for j in range(s)) - Fr(1, 8)
    r["Ac2"] = sum(w[i] * A[i][j] * c[j] ** 2 for i in range(s) for j in range(s)) - Fr(1, 12)
    r["AAc"] = sum(w[i] * A[i][j] * A[j][k] * c[k]
                   for i in range(s) for j in range(s) for k in range(s)) - Fr(1, 24)
    return r
