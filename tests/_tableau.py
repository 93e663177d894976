"""Exact rational Butcher tableaux of RK4(3)5[2R+]C and of Fehlberg's RKF45, read from the
golden fixtures.

Test helper: builds A, b, bhat, c as Fractions from the published coefficients so
that stability polynomials and order conditions can be evaluated exactly, with no
code from the oracle or the GPU path.
"""
from fractions import Fraction as Fr
import os

_GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "lsrk_rk4_3_5_2Rplus_C.txt")
_GOLDEN_RKF = os.path.join(os.path.dirname(__file__), "golden", "rkf45_fehlberg.txt")


def _read(path):
    vals = {}
    with open(path) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            name, num, den = line.split()
            vals[name] = Fr(int(num), int(den))
    return vals


def load_rkf45():
    """Fehlberg's RKF45: A (6 x 6), b (fourth order, propagated), bh (fifth order), c."""
    v = _read(_GOLDEN_RKF)
    s = 6
    A = [[Fr(0)] * s for _ in range(s)]
    for i in range(1, s):
        for j in range(i):
            A[i][j] = v[f"a{i + 1}{j + 1}"]
    b = [v[f"b4_{i}"] for i in range(1, 7)]
    bh = [v[f"b5_{i}"] for i in range(1, 7)]
    c = [sum(A[i]) for i in range(s)]
    return {"b": b, "bh": bh, "A": A, "c": c}


def load():
    vals = _read(_GOLDEN)
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


def order5_residuals(w, A, c):
    """The nine order-5 conditions (one per rooted tree with five vertices)."""
    s = len(w)
    R = range(s)
    Ac = [sum(A[i][j] * c[j] for j in R) for i in R]
    Ac2 = [sum(A[i][j] * c[j] ** 2 for j in R) for i in R]
    Ac3 = [sum(A[i][j] * c[j] ** 3 for j in R) for i in R]
    AAc = [sum(A[i][j] * Ac[j] for j in R) for i in R]
    AcAc = [sum(A[i][j] * c[j] * Ac[j] for j in R) for i in R]
    AAc2 = [sum(A[i][j] * Ac2[j] for j in R) for i in R]
    AAAc = [sum(A[i][j] * AAc[j] for j in R) for i in R]
    r = {}
    r["c4"] = sum(w[i] * c[i] ** 4 for i in R) - Fr(1, 5)
    r["c2Ac"] = sum(w[i] * c[i] ** 2 * Ac[i] for i in R) - Fr(1, 10)
    r["cAc2"] = sum(w[i] * c[i] * Ac2[i] for i in R) - Fr(1, 15)
    r["cAAc"] = sum(w[i] * c[i] * AAc[i] for i in R) - Fr(1, 30)
    r["(Ac)2"] = sum(w[i] * Ac[i] ** 2 for i in R) - Fr(1, 20)
    r["Ac3"] = sum(w[i] * Ac3[i] for i in R) - Fr(1, 20)
    r["AcAc"] = sum(w[i] * AcAc[i] for i in R) - Fr(1, 40)
    r["AAc2"] = sum(w[i] * AAc2[i] for i in R) - Fr(1, 60)
    r["AAAc"] = sum(w[i] * AAAc[i] for i in R) - Fr(1, 120)
    return r
