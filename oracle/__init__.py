"""Python access to the plain FP64 CPU oracle (``oracle.c``).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by the
benchmark's CPU-baseline leg.  The GPU product path never imports it.

``build()`` compiles ``liboracle.so`` with gcc (OpenMP over cells, no FMA contraction,
so x86 and Arm hosts round alike).  The wrappers take the mechanism dict of
``chem_inputs.mechanism`` and numpy arrays; species data are laid out as planes
Y[k, i].
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

MAXSP = 16
MAXRX = 64
NEL = 3


class OMech(C.Structure):
    _fields_ = [
        ("nsp", C.c_int32), ("nrx", C.c_int32),
        ("W", C.c_double * MAXSP),
        ("ncomp", (C.c_int32 * NEL) * MAXSP),
        ("Tmid", C.c_double * MAXSP),
        ("alo", (C.c_double * 7) * MAXSP),
        ("ahi", (C.c_double * 7) * MAXSP),
        ("rtype", C.c_int32 * MAXRX),
        ("nuf", (C.c_int32 * MAXSP) * MAXRX),
        ("nur", (C.c_int32 * MAXSP) * MAXRX),
        ("A", C.c_double * MAXRX), ("b", C.c_double * MAXRX), ("Ea", C.c_double * MAXRX),
        ("A0", C.c_double * MAXRX), ("b0", C.c_double * MAXRX), ("Ea0", C.c_double * MAXRX),
        ("troe", (C.c_double * 4) * MAXRX),
        ("troe_n", C.c_int32 * MAXRX),
        ("eff", (C.c_double * MAXSP) * MAXRX),
        ("reversible", C.c_int32 * MAXRX),
    ]


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (skipped when up to date)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-Wall", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int32)
        mp = C.POINTER(OMech)
        sig = {
            "oracle_cp_R": (C.c_double, [mp, C.c_int, C.c_double]),
            "oracle_h_RT": (C.c_double, [mp, C.c_int, C.c_double]),
            "oracle_s_R": (C.c_double, [mp, C.c_int, C.c_double]),
            "oracle_e_mix": (C.c_double, [mp, dp, C.c_double]),
            "oracle_cv_mix": (C.c_double, [mp, dp, C.c_double]),
            "oracle_T_from_e": (C.c_int, [mp, dp, C.c_double, C.c_double, dp, ip]),
            "oracle_T_from_e_bisect": (C.c_int, [mp, dp, C.c_double, dp]),
            "oracle_troe_F": (C.c_double, [mp, C.c_int, C.c_double, C.c_double]),
            "oracle_rate_constants": (None, [mp, C.c_double, dp, dp, dp]),
            "oracle_progress": (None, [mp, C.c_double, C.c_double, dp, dp, dp]),
            "oracle_wdot": (None, [mp, C.c_double, C.c_double, dp, dp]),
            "oracle_state_from_TPY": (None, [mp, C.c_int64, dp, dp, dp, C.c_int64, dp, dp]),
            "oracle_lsrk_coefficients": (None, [dp, dp, dp]),
            "oracle_linear_step": (None, [C.c_int32, dp, C.c_double, dp, dp]),
            "oracle_linear_integrate": (C.c_int32, [C.c_int32, dp, dp, C.c_double, C.c_double,
                                                    C.c_double, C.c_double, C.c_int32, dp, dp, ip,
                                                    C.c_int32, ip]),
            "oracle_quadratic_fixed": (C.c_double, [C.c_double, C.c_double, C.c_int32, C.c_int32]),
            "oracle_chem_rhs": (C.c_double, [mp, C.c_double, C.c_double, dp, C.c_double, dp]),
            "oracle_integrate": (C.c_int32, [mp, C.c_int64, dp, dp, dp, C.c_int64, dp, C.c_double,
                                             C.c_double, C.c_double, dp, C.c_int32, ip, ip, ip, dp,
                                             dp, C.c_int32]),
            "oracle_chem_fixed": (C.c_int32, [mp, C.c_double, C.c_double, dp, C.c_double,
                                              C.c_double, C.c_int32, dp]),
            "oracle_struct_size": (C.c_int32, []),
            "oracle_butcher": (None, [C.c_int32, ip, dp, dp, dp, dp]),
            "oracle_euler1d_step": (C.c_int32, [mp, C.c_int64, C.c_double, C.c_double, C.c_int32, C.c_int32,
                                                dp, dp, dp, dp, C.c_int64, dp]),
            "oracle_euler1d_max_speed": (C.c_double, [mp, C.c_int64, dp, dp, dp, dp, C.c_int64, dp]),
            "oracle_strang_step": (C.c_int32, [mp, C.c_int64, C.c_double, C.c_double, C.c_int32, C.c_int32,
                                               C.c_double, C.c_double, dp, dp, dp, dp, C.c_int64, dp, C.c_int32]),
            "oracle_linear_step_scheme": (None, [C.c_int32, C.c_int32, dp, C.c_double, dp, dp]),
            "oracle_quadratic_fixed_scheme": (C.c_double, [C.c_int32, C.c_double, C.c_double,
                                                           C.c_int32, C.c_int32]),
            "oracle_integrate_scheme": (C.c_int32, [C.c_int32, mp, C.c_int64, dp, dp, dp, C.c_int64, dp,
                                                    C.c_double, C.c_double, C.c_double, dp, C.c_int32,
                                                    ip, ip, ip, dp, dp, C.c_int32]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        assert L.oracle_struct_size() == C.sizeof(OMech), "oracle struct layout mismatch"
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def make_mech(m: dict) -> OMech:
    """Marshal a chem_inputs mechanism dict into the oracle's struct."""
    S, R = len(m["W"]), len(m["A"])
    assert S <= MAXSP and R <= MAXRX
    o = OMech()
    o.nsp, o.nrx = S, R
    for k in range(S):
        o.W[k] = m["W"][k]
        o.Tmid[k] = m["T_mid"][k]
        for e in range(NEL):
            o.ncomp[k][e] = int(m["ncomp"][k][e])
        for i in range(7):
            o.alo[k][i] = m["nasa_lo"][k][i]
            o.ahi[k][i] = m["nasa_hi"][k][i]
    for j in range(R):
        o.rtype[j] = int(m["rtype"][j])
        o.A[j], o.b[j], o.Ea[j] = m["A"][j], m["b"][j], m["Ea"][j]
        o.A0[j], o.b0[j], o.Ea0[j] = m["A0"][j], m["b0"][j], m["Ea0"][j]
        o.troe_n[j] = int(m["troe_n"][j])
        for i in range(4):
            o.troe[j][i] = m["troe"][j][i]
        o.reversible[j] = int(m["reversible"][j])
        for k in range(S):
            o.nuf[j][k] = int(m["nu_f"][j][k])
            o.nur[j][k] = int(m["nu_r"][j][k])
            o.eff[j][k] = m["eff"][j][k]
    return o


class Oracle:
    """The oracle bound to one mechanism."""

    def __init__(self, mech: dict):
        self.mech = mech
        self.S = len(mech["W"])
        self.R = len(mech["A"])
        self._m = make_mech(mech)
        self._mp = C.pointer(self._m)
        self.L = lib()

    # thermo ---------------------------------------------------------------
    def cp_R(self, k, T):
        return self.L.oracle_cp_R(self._mp, k, T)

    def h_RT(self, k, T):
        return self.L.oracle_h_RT(self._mp, k, T)

    def s_R(self, k, T):
        return self.L.oracle_s_R(self._mp, k, T)

    def e_mix(self, Y, T):
        Y = _f64(Y)
        return self.L.oracle_e_mix(self._mp, _dp(Y), T)

    def cv_mix(self, Y, T):
        Y = _f64(Y)
        return self.L.oracle_cv_mix(self._mp, _dp(Y), T)

    def T_from_e(self, Y, e, Tguess=float("nan")):
        Y = _f64(Y)
        T = C.c_double(0.0)
        it = C.c_int32(0)
        rc = self.L.oracle_T_from_e(self._mp, _dp(Y), e, Tguess, C.byref(T), C.byref(it))
        return rc, T.value, it.value

    def T_from_e_bisect(self, Y, e):
        Y = _f64(Y)
        T = C.c_double(0.0)
        rc = self.L.oracle_T_from_e_bisect(self._mp, _dp(Y), e, C.byref(T))
        return rc, T.value

    # kinetics -------------------------------------------------------------
    def troe_F(self, j, T, Pr):
        return self.L.oracle_troe_F(self._mp, j, T, Pr)

    def rate_constants(self, T, c):
        c = _f64(c)
        kf = np.zeros(self.R)
        kr = np.zeros(self.R)
        self.L.oracle_rate_constants(self._mp, T, _dp(c), _dp(kf), _dp(kr))
        return kf, kr

    def progress(self, rho, T, Y):
        Y = _f64(Y)
        qf = np.zeros(self.R)
        qr = np.zeros(self.R)
        self.L.oracle_progress(self._mp, rho, T, _dp(Y), _dp(qf), _dp(qr))
        return qf, qr

    def wdot(self, rho, T, Y):
        Y = _f64(Y)
        w = np.zeros(self.S)
        self.L.oracle_wdot(self._mp, rho, T, _dp(Y), _dp(w))
        return w

    def chem_rhs(self, rho, e, Y, Tguess=float("nan")):
        Y = _f64(Y)
        F = np.zeros(self.S)
        T = self.L.oracle_chem_rhs(self._mp, rho, e, _dp(Y), Tguess, _dp(F))
        return T, F

    def state_from_TPY(self, T, p, Y):
        T, p, Y = _f64(T), _f64(p), _f64(Y)
        n = T.size
        rho = np.zeros(n)
        e = np.zeros(n)
        self.L.oracle_state_from_TPY(self._mp, n, _dp(T), _dp(p), _dp(Y), Y.shape[1], _dp(rho), _dp(e))
        return rho, e

    # integrator -----------------------------------------------------------
    def integrate(self, rho, e, Y, T, dt, rtol=1e-6, atol=1e-10, h0=None, max_steps=100000,
                  nthreads=0, scheme=0):
        """Integrate every cell over dt.  Returns a dict with Y [S, n], T, status,
        nsteps (attempted), naccept, margin (min |err - 1|) and h (next step).
        scheme: 0 the two-register method of Eq. 21, 1 its tableau with full k-storage,
        2 RKF45 (SCHEMES)."""
        rho, e = _f64(rho), _f64(e)
        Y = np.array(Y, dtype=np.float64, order="C", copy=True)
        T = np.array(T, dtype=np.float64, copy=True)
        n = rho.size
        status = np.zeros(n, dtype=np.int32)
        nsteps = np.zeros(n, dtype=np.int32)
        nacc = np.zeros(n, dtype=np.int32)
        margin = np.zeros(n)
        hout = np.zeros(n)
        h0a = _f64(h0) if h0 is not None else None
        h0p = _dp(h0a) if h0 is not None else None
        self.L.oracle_integrate_scheme(int(scheme), self._mp, n, _dp(rho), _dp(e), _dp(Y), Y.shape[1],
                                       _dp(T), dt, rtol, atol, h0p, max_steps, _ip(status), _ip(nsteps),
                                       _ip(nacc), _dp(margin), _dp(hout), nthreads)
        return {"Y": Y, "T": T, "status": status, "nsteps": nsteps, "naccept": nacc,
                "margin": margin, "h": hout}

    # 1D reactive Euler (the operator either side of the chemistry) -----------
    def euler1d_step(self, U, dx, dt, bc=(0, 0)):
        """One SSP-RK2 MUSCL-HLL step of the 1D Euler equations on the conserved state
        U = dict(rho, rhou, rhoE [n], rhoY [S, n], T [n]) (copied; returns (rc, new U))."""
        V = {k: np.array(v, dtype=np.float64, order="C", copy=True) for k, v in U.items()}
        n = V["rho"].size
        rc = self.L.oracle_euler1d_step(self._mp, n, dx, dt, int(bc[0]), int(bc[1]), _dp(V["rho"]),
                                        _dp(V["rhou"]), _dp(V["rhoE"]), _dp(V["rhoY"]), V["rhoY"].shape[1],
                                        _dp(V["T"]))
        return rc, V

    def euler1d_max_speed(self, U):
        V = {k: _f64(v) for k, v in U.items()}
        return self.L.oracle_euler1d_max_speed(self._mp, V["rho"].size, _dp(V["rho"]), _dp(V["rhou"]),
                                               _dp(V["rhoE"]), _dp(V["rhoY"]), V["rhoY"].shape[1], _dp(V["T"]))

    def strang_step(self, U, dx, dt, bc=(0, 0), rtol=1e-6, atol=1e-10, nthreads=0):
        """Chemistry dt/2, Euler dt, chemistry dt/2 (returns (rc, new U))."""
        V = {k: np.array(v, dtype=np.float64, order="C", copy=True) for k, v in U.items()}
        n = V["rho"].size
        rc = self.L.oracle_strang_step(self._mp, n, dx, dt, int(bc[0]), int(bc[1]), rtol, atol, _dp(V["rho"]),
                                       _dp(V["rhou"]), _dp(V["rhoE"]), _dp(V["rhoY"]), V["rhoY"].shape[1],
                                       _dp(V["T"]), nthreads)
        return rc, V

    def conserved_from_prim(self, rho, u, T, Y):
        """U dict from primitive (rho, u, T, Y [S, n]) with the oracle's thermo."""
        rho, u, T, Y = _f64(rho), _f64(u), _f64(T), _f64(Y)
        e = np.array([self.e_mix(Y[:, i], T[i]) for i in range(rho.size)])
        return {"rho": rho.copy(), "rhou": rho * u, "rhoE": rho * (e + 0.5 * u * u), "rhoY": rho[None, :] * Y,
                "T": T.copy()}

    def chem_fixed(self, rho, e, Y, T, h, nsteps):
        Y = np.array(Y, dtype=np.float64, copy=True)
        trace = np.zeros(nsteps)
        rc = self.L.oracle_chem_fixed(self._mp, rho, e, _dp(Y), T, h, nsteps, _dp(trace))
        return rc, Y, trace


def lsrk_coefficients():
    a = np.zeros(4)
    b = np.zeros(5)
    bh = np.zeros(5)
    lib().oracle_lsrk_coefficients(_dp(a), _dp(b), _dp(bh))
    return a, b, bh


def linear_step(M, h, y):
    M = _f64(M)
    y = np.array(y, dtype=np.float64, copy=True)
    E = np.zeros_like(y)
    lib().oracle_linear_step(y.size, _dp(M), h, _dp(y), _dp(E))
    return y, E


def linear_integrate(M, y, dt, rtol, atol, h0=0.0, max_steps=100000, max_log=100000):
    M = _f64(M)
    y = np.array(y, dtype=np.float64, copy=True)
    lh = np.zeros(max_log)
    le = np.zeros(max_log)
    la = np.zeros(max_log, dtype=np.int32)
    out = np.zeros(3, dtype=np.int32)
    k = lib().oracle_linear_integrate(y.size, _dp(M), _dp(y), dt, rtol, atol, h0, max_steps, _dp(lh),
                                      _dp(le), _ip(la), max_log, _ip(out))
    k = min(k, max_log)
    return {"y": y, "h": lh[:k], "err": le[:k], "acc": la[:k].astype(bool), "status": int(out[0]),
            "nacc": int(out[1]), "nrej": int(out[2])}


def quadratic_fixed(y0, h, nsteps, embedded=False):
    return lib().oracle_quadratic_fixed(y0, h, nsteps, int(embedded))


SCHEMES = {"lsrk2r": 0, "full": 1, "rkf45": 2}
MAXSTAGE = 6


def butcher(scheme):
    """Butcher tableau of scheme 1 or 2 (scheme 0 has the same tableau as 1): returns
    (stages, A [6, 6], b, bhat, controller exponent)."""
    s = C.c_int32(0)
    a = np.zeros(MAXSTAGE * MAXSTAGE)
    b = np.zeros(MAXSTAGE)
    bh = np.zeros(MAXSTAGE)
    ex = C.c_double(0.0)
    lib().oracle_butcher(int(scheme), C.byref(s), _dp(a), _dp(b), _dp(bh), C.byref(ex))
    k = s.value
    return k, a.reshape(MAXSTAGE, MAXSTAGE)[:k, :k].copy(), b[:k].copy(), bh[:k].copy(), ex.value


def linear_step_scheme(scheme, M, h, y):
    M = _f64(M)
    y = np.array(y, dtype=np.float64, copy=True)
    E = np.zeros_like(y)
    lib().oracle_linear_step_scheme(int(scheme), y.size, _dp(M), h, _dp(y), _dp(E))
    return y, E


def quadratic_fixed_scheme(scheme, y0, h, nsteps, embedded=False):
    return lib().oracle_quadratic_fixed_scheme(int(scheme), y0, h, nsteps, int(embedded))
