"""Thin Python binding of libchem.so (include/chem.h): argument marshalling only.

Every step of the integration runs in the library's CUDA kernels.  PyTorch provides
device memory and streams: the functions here take torch CUDA tensors and pass their
data pointers and the current stream to the C ABI.  There is no CPU fallback: if
libchem.so is missing or no GPU is present the calls raise.

Names follow the C ABI: ``Context`` wraps chem_setup / chem_teardown, and its methods
``integrate``, ``integrate_host`` and ``state_from_TPY`` wrap chem_integrate,
chem_integrate_host and chem_state_from_TPY.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libchem.so")
# one library per compiled mechanism structure (species count -> library)
LIB_PATHS = {9: LIB_PATH, 13: os.path.join(PKG, "libchem_h2o2_13.so")}

MAX_SPECIES = 16
MAX_REACTIONS = 32
NUM_ELEMENTS = 3

OK, ERR_INVALID, ERR_CUDA, ERR_UNSUPPORTED, ERR_NOMEM, ERR_TIMEOUT, ERR_STATE = 0, -1, -2, -3, -4, -5, -6
CELL_OK, CELL_MAX_STEPS, CELL_H_UNDERFLOW, CELL_NEWTON_FAIL, CELL_NONFINITE, CELL_SURROGATE = range(6)
VARIANTS = {"fp64": 0, "mixed": 1}
SCHEMES = {"lsrk": 0, "full": 1, "rkf45": 2}


class ChemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"libchem error {code}: {msg}")
        self.code = code


class Mechanism(C.Structure):
    _fields_ = [
        ("n_species", C.c_int32), ("n_reactions", C.c_int32),
        ("W", C.c_double * MAX_SPECIES),
        ("ncomp", (C.c_int32 * NUM_ELEMENTS) * MAX_SPECIES),
        ("T_mid", C.c_double * MAX_SPECIES),
        ("nasa_lo", (C.c_double * 7) * MAX_SPECIES),
        ("nasa_hi", (C.c_double * 7) * MAX_SPECIES),
        ("rtype", C.c_int32 * MAX_REACTIONS),
        ("nu_f", (C.c_int32 * MAX_SPECIES) * MAX_REACTIONS),
        ("nu_r", (C.c_int32 * MAX_SPECIES) * MAX_REACTIONS),
        ("A", C.c_double * MAX_REACTIONS), ("b", C.c_double * MAX_REACTIONS),
        ("Ea", C.c_double * MAX_REACTIONS),
        ("A0", C.c_double * MAX_REACTIONS), ("b0", C.c_double * MAX_REACTIONS),
        ("Ea0", C.c_double * MAX_REACTIONS),
        ("troe", (C.c_double * 4) * MAX_REACTIONS),
        ("troe_n", C.c_int32 * MAX_REACTIONS),
        ("eff", (C.c_double * MAX_SPECIES) * MAX_REACTIONS),
        ("reversible", C.c_int32 * MAX_REACTIONS),
    ]


class Options(C.Structure):
    _fields_ = [("variant", C.c_int32), ("max_steps", C.c_int32), ("block_size", C.c_int32),
                ("scheme", C.c_int32), ("reserved", C.c_int32 * 4)]


class State(C.Structure):
    _fields_ = [("d_rho", C.c_void_p), ("d_e", C.c_void_p), ("d_Y", C.c_void_p),
                ("ldY", C.c_int64), ("d_T", C.c_void_p), ("d_h", C.c_void_p),
                ("d_status", C.c_void_p), ("d_nsteps", C.c_void_p)]


class Flow1D(C.Structure):
    _fields_ = [("d_rho", C.c_void_p), ("d_rhou", C.c_void_p), ("d_rhoE", C.c_void_p), ("d_rhoY", C.c_void_p),
                ("ldY", C.c_int64), ("d_T", C.c_void_p), ("d_status", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [("cells", C.c_int64), ("accepted", C.c_int64), ("rejected", C.c_int64),
                ("rhs_evals", C.c_int64), ("max_steps_cell", C.c_int64),
                ("status_count", C.c_int64 * 8)]


class Batch(C.Structure):
    _fields_ = [("nboxes", C.c_int32), ("d_box_offset", C.c_void_p), ("d_box_dt", C.c_void_p),
                ("d_box_nsub", C.c_void_p)]


class BatchOptions(C.Structure):
    _fields_ = [("order", C.c_int32), ("ctas_per_sm", C.c_int32), ("use_graph", C.c_int32),
                ("shape", C.c_int32), ("d_cost_hint", C.c_void_p)]


class TuneResult(C.Structure):
    _fields_ = [("opt", BatchOptions), ("ms", C.c_float), ("block", C.c_int32), ("regs", C.c_int32),
                ("ctas_per_sm", C.c_int32)]


BATCH_SHAPES = 6


class Pairs(C.Structure):
    _fields_ = [("d_rho", C.c_void_p), ("d_e", C.c_void_p), ("d_Y0", C.c_void_p), ("ldY0", C.c_int64),
                ("d_T0", C.c_void_p), ("d_dt", C.c_void_p), ("d_Y1", C.c_void_p), ("ldY1", C.c_int64)]


class TrainCfg(C.Structure):
    _fields_ = [("epochs", C.c_int32), ("batch", C.c_int32), ("lr", C.c_float), ("lr_final", C.c_float),
                ("boxcox_lambda", C.c_float), ("dt_power", C.c_float), ("seed", C.c_uint64)]


class Gate(C.Structure):
    _fields_ = [("ood_margin", C.c_float), ("resid_max", C.c_float), ("neg_tol", C.c_float),
                ("max_dT", C.c_float), ("err_tol", C.c_float),
                ("rate_max", C.c_float)]


ORDER_STIFFNESS, ORDER_NATURAL = 0, 1
STATS_WORDS = C.sizeof(Stats) // 8

_libs = {}


def load(n_species: int = 9) -> C.CDLL:
    """Load the library compiled for the mechanism structure with n_species species
    (libchem.so for 9, libchem_h2o2_13.so for 13; built in-tree by
    paper_2506_02602_gb300.build)."""
    if n_species in _libs:
        return _libs[n_species]
    path = LIB_PATHS.get(n_species)
    if path is None:
        raise ChemError(ERR_UNSUPPORTED, f"no library is compiled for {n_species} species "
                                         f"(structures: {sorted(LIB_PATHS)})")
    if not os.path.exists(path):
        raise ChemError(ERR_CUDA, f"{path} is not built; run paper_2506_02602_gb300.build.build()")
    L = C.CDLL(path)
    vp, i64, dbl = C.c_void_p, C.c_int64, C.c_double
    sig = {
        "chem_version": (C.c_int, []),
        "chem_last_error": (C.c_char_p, [vp]),
        "chem_setup": (C.c_int, [C.POINTER(Mechanism), C.POINTER(Options), C.POINTER(vp)]),
        "chem_teardown": (C.c_int, [vp]),
        "chem_state_from_TPY": (C.c_int, [vp, i64, vp, vp, vp, i64, vp, vp, vp]),
        "chem_integrate": (C.c_int, [vp, C.POINTER(State), i64, dbl, dbl, dbl, vp, vp]),
        "chem_integrate_host": (C.c_int, [vp, i64, vp, vp, vp, i64, vp, vp, vp, vp, dbl, dbl, dbl, vp]),
        "chem_diag_math": (C.c_int, [C.c_int, i64, vp, vp, vp]),
        "chem_diag_fma_peak": (C.c_int, [C.c_int, C.c_int32, C.c_int32, i64, vp, vp]),
        "chem_diag_ln_inv_kc": (C.c_int, [vp, C.c_int, i64, vp, vp, vp]),
        "chem_integrate_batched": (C.c_int, [vp, C.POINTER(State), i64, C.POINTER(Batch), dbl, dbl,
                                             C.POINTER(BatchOptions), vp, vp]),
        "chem_batch_shape_info": (C.c_int, [vp, C.c_int32, vp, vp, vp]),
        "chem_autotune_batched": (C.c_int, [vp, C.POINTER(State), i64, C.POINTER(Batch), dbl, dbl,
                                            C.POINTER(BatchOptions), C.c_char_p, vp, C.POINTER(BatchOptions),
                                            vp, C.c_int32, vp]),
        "chem_surrogate_param_count": (C.c_int64, []),
        "chem_surrogate_train": (C.c_int, [vp, C.POINTER(Pairs), i64, C.POINTER(TrainCfg), vp, vp]),
        "chem_surrogate_infer": (C.c_int, [vp, C.POINTER(State), i64, dbl, dbl, dbl, C.POINTER(Gate),
                                           vp, vp, vp]),
        "chem_surrogate_infer_batched": (C.c_int, [vp, C.POINTER(State), i64, C.POINTER(Batch), dbl, dbl,
                                                   C.POINTER(Gate), vp, vp, vp]),
        "chem_surrogate_save": (C.c_int, [vp, C.c_char_p]),
        "chem_surrogate_load": (C.c_int, [vp, C.c_char_p]),
        "chem_surrogate_params": (C.c_int, [vp, vp, vp, i64]),
        "chem_surrogate_grad": (C.c_int, [vp, vp, vp, i64, vp, vp, vp, vp]),
        "chem_surrogate_forward": (C.c_int, [vp, vp, i64, vp, C.c_int32, vp, vp]),
        "chem_surrogate_adam": (C.c_int, [vp, vp, i64, C.c_float]),
        "chem_euler1d_step": (C.c_int, [vp, C.POINTER(Flow1D), i64, dbl, dbl, C.c_int32, C.c_int32, vp]),
        "chem_euler1d_max_speed": (C.c_int, [vp, C.POINTER(Flow1D), i64, vp, vp]),
        "chem_strang_step": (C.c_int, [vp, C.POINTER(Flow1D), i64, dbl, dbl, C.c_int32, C.c_int32, dbl, dbl,
                                       vp, vp]),
        "chem_surrogate_trace": (C.c_int, [vp, vp, vp, i64, vp, vp, vp, vp, vp, vp, vp, vp]),
        "chem_surrogate_project": (C.c_int, [vp, i64, vp, vp, i64, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _libs[n_species] = L
    return L


def diag_math(op: int, x, stream=None):
    """chem_diag_math on a float64 CUDA tensor; returns a new tensor.  op: 0 table exp,
    1 table log, 2 library exp, 3 library log, 4 / 5 reciprocal with one / two
    Newton-Raphson steps, 6 hardware reciprocal approximation, 7 integer-pipe fp64 ->
    fp32, 8 integer-pipe fp32 -> fp64 of fp32(x), 9 / 10 hi / lo of the 2^-12 split."""
    import torch
    _check_f64_cuda("x", x)
    y = torch.empty_like(x)
    rc = load().chem_diag_math(op, x.numel(), _ptr(x), _ptr(y), _stream(stream))
    if rc != OK:
        raise ChemError(rc, "chem_diag_math failed")
    return y


def fma_peak(op: int, blocks: int, threads: int, iters: int, reps: int = 5, stream=None):
    """chem_diag_fma_peak timed with CUDA events: returns (best GFLOP/s over reps launches,
    flops per launch).  op 0: fp64, 1: fp32."""
    import torch
    sink = torch.empty(blocks * threads + 2, dtype=torch.float64 if op == 0 else torch.float32, device="cuda")
    st = torch.cuda.current_stream() if stream is None else stream
    flops = float(blocks) * threads * iters * 64
    best = float("inf")
    for r in range(reps + 1):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(st)
        rc = load().chem_diag_fma_peak(op, blocks, threads, iters, _ptr(sink), _stream(st))
        b.record(st)
        if rc != OK:
            raise ChemError(rc, "chem_diag_fma_peak failed")
        torch.cuda.synchronize()
        if r:  # the first launch warms up
            best = min(best, a.elapsed_time(b) * 1e-3)
    return flops / best / 1e9, flops


def make_mechanism(m: dict) -> Mechanism:
    """Marshal a mechanism dict (chem_inputs.mechanism layout) into chem_mechanism."""
    S, R = len(m["W"]), len(m["A"])
    if S > MAX_SPECIES or R > MAX_REACTIONS:
        raise ChemError(ERR_INVALID, "mechanism exceeds CHEM_MAX_SPECIES / CHEM_MAX_REACTIONS")
    c = Mechanism()
    c.n_species, c.n_reactions = S, R
    for k in range(S):
        c.W[k] = float(m["W"][k])
        c.T_mid[k] = float(m["T_mid"][k])
        for e in range(NUM_ELEMENTS):
            c.ncomp[k][e] = int(m["ncomp"][k][e])
        for i in range(7):
            c.nasa_lo[k][i] = float(m["nasa_lo"][k][i])
            c.nasa_hi[k][i] = float(m["nasa_hi"][k][i])
    for j in range(R):
        c.rtype[j] = int(m["rtype"][j])
        c.A[j], c.b[j], c.Ea[j] = float(m["A"][j]), float(m["b"][j]), float(m["Ea"][j])
        c.A0[j], c.b0[j], c.Ea0[j] = float(m["A0"][j]), float(m["b0"][j]), float(m["Ea0"][j])
        c.troe_n[j] = int(m["troe_n"][j])
        for i in range(4):
            c.troe[j][i] = float(m["troe"][j][i])
        c.reversible[j] = int(m["reversible"][j])
        for k in range(S):
            c.nu_f[j][k] = int(m["nu_f"][j][k])
            c.nu_r[j][k] = int(m["nu_r"][j][k])
            c.eff[j][k] = float(m["eff"][j][k])
    return c


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _check_f64_cuda(name, t, n=None):
    import torch
    if t.device.type != "cuda" or t.dtype != torch.float64:
        raise ChemError(ERR_INVALID, f"{name} must be a float64 CUDA tensor")
    if n is not None and t.shape[-1] < n:
        raise ChemError(ERR_INVALID, f"{name} has fewer than {n} cells")


def _check_cells(n, rho, e, Y, T, h=None, status=None, nsteps=None, cost_hint=None):
    """The state tensors of one call hold at least n cells, with the dtypes of chem.h:
    rho, e, T (and h) float64 CUDA vectors, Y float64 [S, ld] planes with ld >= n and
    contiguous rows, status / nsteps / cost_hint int32 CUDA vectors."""
    import torch
    if n < 0:
        raise ChemError(ERR_INVALID, "ncells < 0")
    for nm, t in (("rho", rho), ("e", e), ("T", T), ("h", h)):
        if t is not None:
            _check_f64_cuda(nm, t)
            if t.numel() < n:
                raise ChemError(ERR_INVALID, f"{nm} has {t.numel()} < {n} cells")
    _check_f64_cuda("Y", Y)
    if Y.dim() != 2 or Y.stride(1) != 1 or Y.shape[1] < n or Y.stride(0) < n:
        raise ChemError(ERR_INVALID, "Y must be [S, ld] planes with contiguous rows and ld >= ncells")
    for nm, t in (("status", status), ("nsteps", nsteps), ("cost_hint", cost_hint)):
        if t is not None and (t.device.type != "cuda" or t.dtype != torch.int32 or t.numel() < n):
            raise ChemError(ERR_INVALID, f"{nm} must be an int32 CUDA tensor of >= {n} cells")


class Context:
    """A chem_ctx bound to one mechanism and precision variant."""

    def __init__(self, mech: dict, variant: str = "fp64", max_steps: int = 0, block_size: int = 0,
                 scheme: str = "lsrk"):
        self.L = load(len(mech["W"]))
        self._mech = make_mechanism(mech)
        opt = Options()
        opt.variant = VARIANTS[variant]
        opt.max_steps = max_steps
        opt.block_size = block_size
        opt.scheme = SCHEMES[scheme]
        h = C.c_void_p()
        rc = self.L.chem_setup(C.byref(self._mech), C.byref(opt), C.byref(h))
        if rc != OK:
            raise ChemError(rc, self.L.chem_last_error(None).decode())
        self.h = h
        self.variant = variant
        self.scheme = scheme
        self.n_species = len(mech["W"])

    def close(self):
        if getattr(self, "h", None):
            self.L.chem_teardown(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _raise(self, rc):
        if rc != OK:
            raise ChemError(rc, self.L.chem_last_error(self.h).decode())

    def state_from_TPY(self, T, p, Y, rho=None, e=None, stream=None):
        """rho, e from (T, p, Y) on the device (float64 CUDA tensors; Y is [S, ld])."""
        import torch
        n = T.numel()
        for nm, t in (("T", T), ("p", p), ("Y", Y)):
            _check_f64_cuda(nm, t)
        rho = torch.empty_like(T) if rho is None else rho
        e = torch.empty_like(T) if e is None else e
        self._raise(self.L.chem_state_from_TPY(self.h, n, _ptr(T), _ptr(p), _ptr(Y), Y.stride(0),
                                               _ptr(rho), _ptr(e), _stream(stream)))
        return rho, e

    def integrate(self, rho, e, Y, T, dt, rtol=1e-6, atol=1e-10, h=None, status=None, nsteps=None,
                  stats=None, stream=None, ncells=None):
        """Advance Y [S, ld] and T in place over dt (chem_integrate).  status / nsteps
        (int32 CUDA tensors), h (float64) and stats (int64 tensor of STATS_WORDS) are
        optional outputs."""
        n = rho.numel() if ncells is None else ncells
        for nm, t in (("rho", rho), ("e", e), ("Y", Y), ("T", T)):
            _check_f64_cuda(nm, t, n)
        if Y.stride(1) != 1:
            raise ChemError(ERR_INVALID, "Y planes must be contiguous")
        st = State(_ptr(rho).value, _ptr(e).value, _ptr(Y).value, Y.stride(0), _ptr(T).value,
                   None if h is None else h.data_ptr(),
                   None if status is None else status.data_ptr(),
                   None if nsteps is None else nsteps.data_ptr())
        self._raise(self.L.chem_integrate(self.h, C.byref(st), n, float(dt), float(rtol), float(atol),
                                          _stream(stream), _ptr(stats)))

    def integrate_batched(self, rho, e, Y, T, box_offset, box_dt, box_nsub, rtol=1e-6, atol=1e-10,
                          h=None, status=None, nsteps=None, stats=None, order=ORDER_STIFFNESS,
                          ctas_per_sm=0, use_graph=False, cost_hint=None, stream=None, shape=0):
        """chem_integrate_batched: box_offset (int64 [nb+1]), box_dt (float64 [nb]) and
        box_nsub (int32 [nb]) are CUDA tensors; the state tensors are as in integrate."""
        import torch
        n = rho.numel()
        _check_cells(n, rho, e, Y, T, h, status, nsteps, cost_hint)
        if box_offset.dtype != torch.int64 or box_nsub.dtype != torch.int32 or box_dt.dtype != torch.float64:
            raise ChemError(ERR_INVALID, "box_offset int64, box_dt float64, box_nsub int32 expected")
        st = State(_ptr(rho).value, _ptr(e).value, _ptr(Y).value, Y.stride(0), _ptr(T).value,
                   None if h is None else h.data_ptr(),
                   None if status is None else status.data_ptr(),
                   None if nsteps is None else nsteps.data_ptr())
        b = Batch(box_dt.numel(), box_offset.data_ptr(), box_dt.data_ptr(), box_nsub.data_ptr())
        o = BatchOptions(order, ctas_per_sm, int(bool(use_graph)), shape,
                         None if cost_hint is None else cost_hint.data_ptr())
        self._raise(self.L.chem_integrate_batched(self.h, C.byref(st), n, C.byref(b), float(rtol),
                                                  float(atol), C.byref(o), _stream(stream), _ptr(stats)))

    def batch_shape_info(self, shape):
        """chem_batch_shape_info: (threads per CTA, registers per thread, CTAs per SM)."""
        blk, regs, per = C.c_int32(), C.c_int32(), C.c_int32()
        self._raise(self.L.chem_batch_shape_info(self.h, shape, C.byref(blk), C.byref(regs), C.byref(per)))
        return blk.value, regs.value, per.value

    def autotune_batched(self, rho, e, Y, T, box_offset, box_dt, box_nsub, rtol=1e-6, atol=1e-10,
                         h=None, cache_path=None, cost_hint=None, stream=None, max_results=64):
        """chem_autotune_batched on the caller's batch (state untouched).  Returns (best
        options as a dict usable as integrate_batched keywords, list of timed candidates)."""
        n = rho.numel()
        st = State(_ptr(rho).value, _ptr(e).value, _ptr(Y).value, Y.stride(0), _ptr(T).value,
                   None if h is None else h.data_ptr(), None, None)
        b = Batch(box_dt.numel(), box_offset.data_ptr(), box_dt.data_ptr(), box_nsub.data_ptr())
        base = BatchOptions(0, 0, 0, 0, None if cost_hint is None else cost_hint.data_ptr())
        best = BatchOptions()
        res = (TuneResult * max_results)()
        nres = C.c_int32()
        self._raise(self.L.chem_autotune_batched(
            self.h, C.byref(st), n, C.byref(b), float(rtol), float(atol), C.byref(base),
            None if cache_path is None else os.fsencode(cache_path), _stream(stream), C.byref(best),
            res, max_results, C.byref(nres)))
        opts = {"order": best.order, "ctas_per_sm": best.ctas_per_sm, "use_graph": bool(best.use_graph),
                "shape": best.shape}
        table = [{"order": r.opt.order, "ctas_per_sm": r.ctas_per_sm, "use_graph": bool(r.opt.use_graph),
                  "shape": r.opt.shape, "block": r.block, "regs": r.regs, "ms": r.ms}
                 for r in res[: min(nres.value, max_results)]]
        return opts, table

    def integrate_batched_noalloc(self, rho, e, Y, T, box_offset, box_dt, box_nsub, rtol=1e-6,
                                  atol=1e-10, h=None, status=None, nsteps=None, stats=None,
                                  order=ORDER_STIFFNESS, ctas_per_sm=0, cost_hint=None,
                                  stream=None, ncells=None, shape=0):
        """chem_integrate_batched_noalloc: the batched integration for callers that cannot
        allocate device memory during the call (under a memory arena that owns the GPU, in
        latency-bound loops).  The scratch is a fixed array in the library: at most
        1,048,576 cells per call, and calls that overlap on the GPU race on it.  Arguments
        and checks as integrate_batched; ncells (at most the tensors' cell count)
        overrides rho.numel()."""
        import torch
        fn = self.L.chem_integrate_batched_noalloc
        fn.restype = C.c_int
        fn.argtypes = [C.c_void_p, C.POINTER(State), C.c_int64, C.POINTER(Batch), C.c_double,
                       C.c_double, C.POINTER(BatchOptions), C.c_void_p, C.c_void_p]
        n = rho.numel() if ncells is None else int(ncells)
        _check_cells(n, rho, e, Y, T, h, status, nsteps, cost_hint)
        if box_offset.dtype != torch.int64 or box_nsub.dtype != torch.int32 or box_dt.dtype != torch.float64:
            raise ChemError(ERR_INVALID, "box_offset int64, box_dt float64, box_nsub int32 expected")
        st = State(_ptr(rho).value, _ptr(e).value, _ptr(Y).value, Y.stride(0), _ptr(T).value,
                   None if h is None else h.data_ptr(),
                   None if status is None else status.data_ptr(),
                   None if nsteps is None else nsteps.data_ptr())
        b = Batch(box_dt.numel(), box_offset.data_ptr(), box_dt.data_ptr(), box_nsub.data_ptr())
        o = BatchOptions(order, ctas_per_sm, 0, shape, None if cost_hint is None else cost_hint.data_ptr())
        self._raise(fn(self.h, C.byref(st), n, C.byref(b), float(rtol), float(atol), C.byref(o),
                       _stream(stream), _ptr(stats)))

    # learned surrogate ------------------------------------------------------------
    def surrogate_train(self, rho, e, Y0, dt, Y1, T0=None, epochs=20, batch=4096, lr=1e-3,
                        lr_final=0.0, boxcox_lambda=0.1, seed=0, dt_power=0.0, stream=None):
        """chem_surrogate_train on CUDA tensors (Y0, Y1: [S, n] planes; dt: [n]).
        Returns the mean loss of every epoch (numpy)."""
        n = rho.numel()
        for nm, t in (("rho", rho), ("e", e), ("Y0", Y0), ("dt", dt), ("Y1", Y1)):
            _check_f64_cuda(nm, t, n)
        pr = Pairs(rho.data_ptr(), e.data_ptr(), Y0.data_ptr(), Y0.stride(0),
                   None if T0 is None else T0.data_ptr(), dt.data_ptr(), Y1.data_ptr(), Y1.stride(0))
        cfg = TrainCfg(epochs, batch, lr, lr_final, boxcox_lambda, dt_power, seed)
        loss = np.zeros(max(epochs, 1), dtype=np.float32)
        self._raise(self.L.chem_surrogate_train(self.h, C.byref(pr), n, C.byref(cfg), _stream(stream),
                                                loss.ctypes.data_as(C.c_void_p)))
        return loss[:epochs]

    def surrogate_infer(self, rho, e, Y, T, dt, rtol=1e-6, atol=1e-10, status=None, nsteps=None,
                        mask=None, stats=None, gate=None, stream=None):
        """chem_surrogate_infer: advance Y, T in place over dt; gate is a dict of
        ood_margin / resid_max / neg_tol / max_dT / err_tol / rate_max (0 or missing =
        default)."""
        n = rho.numel()
        st = State(_ptr(rho).value, _ptr(e).value, _ptr(Y).value, Y.stride(0), _ptr(T).value, None,
                   None if status is None else status.data_ptr(),
                   None if nsteps is None else nsteps.data_ptr())
        g = Gate(**(gate or {}))
        self._raise(self.L.chem_surrogate_infer(self.h, C.byref(st), n, float(dt), float(rtol),
                                                float(atol), C.byref(g), _stream(stream), _ptr(mask),
                                                _ptr(stats)))

    def surrogate_infer_batched(self, rho, e, Y, T, box_offset, box_dt, box_nsub, rtol=1e-6, atol=1e-10,
                                status=None, nsteps=None, mask=None, stats=None, gate=None, stream=None):
        """chem_surrogate_infer_batched: every box's substeps with the surrogate in one call
        (box arrays as integrate_batched, CUDA tensors); Y, T advanced in place."""
        import torch
        n = rho.numel()
        _check_cells(n, rho, e, Y, T, None, status, nsteps)
        if box_offset.dtype != torch.int64 or box_nsub.dtype != torch.int32 or box_dt.dtype != torch.float64:
            raise ChemError(ERR_INVALID, "box_offset int64, box_dt float64, box_nsub int32 expected")
        st = State(_ptr(rho).value, _ptr(e).value, _ptr(Y).value, Y.stride(0), _ptr(T).value, None,
                   None if status is None else status.data_ptr(),
                   None if nsteps is None else nsteps.data_ptr())
        b = Batch(box_dt.numel(), box_offset.data_ptr(), box_dt.data_ptr(), box_nsub.data_ptr())
        g = Gate(**(gate or {}))
        self._raise(self.L.chem_surrogate_infer_batched(self.h, C.byref(st), n, C.byref(b), float(rtol),
                                                        float(atol), C.byref(g), _stream(stream), _ptr(mask),
                                                        _ptr(stats)))

    def surrogate_save(self, path):
        self._raise(self.L.chem_surrogate_save(self.h, os.fsencode(path)))

    def surrogate_load(self, path):
        self._raise(self.L.chem_surrogate_load(self.h, os.fsencode(path)))

    def surrogate_params(self, new=None):
        """Flat fp32 parameters (numpy); with `new`, upload them first (resets Adam)."""
        n = self.L.chem_surrogate_param_count()
        out = np.zeros(n, dtype=np.float32)
        src = None
        if new is not None:
            src = np.ascontiguousarray(new, dtype=np.float32)
            assert src.size == n
        self._raise(self.L.chem_surrogate_params(self.h, out.ctypes.data_as(C.c_void_p),
                                                 None if src is None else src.ctypes.data_as(C.c_void_p), n))
        return out

    def surrogate_grad(self, X, T, stream=None):
        """chem_surrogate_grad on fp32 CUDA tensors X, T [B, 16]: returns (Y [B, 16] tensor,
        flat gradient numpy, loss)."""
        import torch
        B = X.shape[0]
        Y = torch.empty((B, 16), dtype=torch.float32, device=X.device)
        g = np.zeros(self.L.chem_surrogate_param_count(), dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        self._raise(self.L.chem_surrogate_grad(self.h, _ptr(X), _ptr(T), B, _ptr(Y),
                                               g.ctypes.data_as(C.c_void_p), loss.ctypes.data_as(C.c_void_p),
                                               _stream(stream)))
        return Y, g, float(loss[0])

    def surrogate_trace(self, X, T, stream=None):
        """chem_surrogate_trace on fp32 CUDA tensors X, T [B, 16]: returns a dict of
        numpy arrays Y [B, 16], Z [3, B, 256], H [3, B, 256] (bf16 values as float32),
        G [4, B, 256] (layer 3 in G3 [B, 16]), dH [3, B, 256], grad (flat) and loss."""
        import torch
        B = X.shape[0]
        dev = X.device
        Y = torch.empty((B, 16), dtype=torch.float32, device=dev)
        Z = torch.empty((3, B, 256), dtype=torch.float32, device=dev)
        H = torch.empty((3, B, 256), dtype=torch.bfloat16, device=dev)
        G = torch.zeros((4, B, 256), dtype=torch.bfloat16, device=dev)
        dH = torch.empty((3, B, 256), dtype=torch.float32, device=dev)
        g = np.zeros(self.L.chem_surrogate_param_count(), dtype=np.float32)
        loss = np.zeros(1, dtype=np.float32)
        self._raise(self.L.chem_surrogate_trace(self.h, _ptr(X), _ptr(T), B, _ptr(Y), _ptr(Z), _ptr(H), _ptr(G),
                                                _ptr(dH), g.ctypes.data_as(C.c_void_p),
                                                loss.ctypes.data_as(C.c_void_p), _stream(stream)))
        Gf = G.float()
        return {"Y": Y.cpu().numpy(), "Z": Z.cpu().numpy(), "H": H.float().cpu().numpy(),
                "G": Gf[:3].cpu().numpy(), "G3": Gf[3].reshape(-1)[: B * 16].reshape(B, 16).cpu().numpy(),
                "dH": dH.cpu().numpy(), "grad": g, "loss": float(loss[0])}

    # the split scheme's 1D flow -------------------------------------------------
    @staticmethod
    def _flow(U, status=None):
        """chem_flow1d of a dict of float64 CUDA tensors rho, rhou, rhoE [n], rhoY [S, ld], T [n]."""
        for k in ("rho", "rhou", "rhoE", "rhoY", "T"):
            _check_f64_cuda(k, U[k])
        n = U["rho"].numel()
        for k in ("rhou", "rhoE", "T"):
            if U[k].numel() < n:
                raise ChemError(ERR_INVALID, f"{k} has fewer than {n} cells")
        if U["rhoY"].stride(1) != 1 or U["rhoY"].shape[1] < n:
            raise ChemError(ERR_INVALID, "rhoY must be [S, ld] planes with ld >= n")
        return Flow1D(U["rho"].data_ptr(), U["rhou"].data_ptr(), U["rhoE"].data_ptr(), U["rhoY"].data_ptr(),
                      U["rhoY"].stride(0), U["T"].data_ptr(), None if status is None else status.data_ptr()), n

    def euler1d_step(self, U, dx, dt, bc=(0, 0), status=None, stream=None):
        """chem_euler1d_step on the flow U in place."""
        f, n = self._flow(U, status)
        self._raise(self.L.chem_euler1d_step(self.h, C.byref(f), n, float(dx), float(dt), int(bc[0]), int(bc[1]),
                                             _stream(stream)))

    def euler1d_max_speed(self, U, stream=None):
        f, n = self._flow(U)
        out = C.c_double(0.0)
        self._raise(self.L.chem_euler1d_max_speed(self.h, C.byref(f), n, C.byref(out), _stream(stream)))
        return out.value

    def strang_step(self, U, dx, dt, bc=(0, 0), rtol=1e-6, atol=1e-10, status=None, stats=None, stream=None):
        """chem_strang_step on the flow U in place."""
        f, n = self._flow(U, status)
        self._raise(self.L.chem_strang_step(self.h, C.byref(f), n, float(dx), float(dt), int(bc[0]), int(bc[1]),
                                            float(rtol), float(atol), _stream(stream), _ptr(stats)))

    def surrogate_adam(self, grad, lr):
        """chem_surrogate_adam: one Adam step of the parameters with the flat gradient
        `grad` (numpy fp32) and learning rate lr."""
        g = np.ascontiguousarray(grad, dtype=np.float32)
        self._raise(self.L.chem_surrogate_adam(self.h, g.ctypes.data_as(C.c_void_p), g.size, float(lr)))

    def surrogate_project(self, Y0, Yp, out=None, stream=None):
        """chem_surrogate_project on float64 CUDA planes Y0, Yp [S, ld]: the element
        projection of Yp onto the element mass fractions of Y0 (returns out)."""
        import torch
        _check_f64_cuda("Y0", Y0)
        _check_f64_cuda("Yp", Yp)
        if Y0.shape != Yp.shape or Y0.stride() != Yp.stride() or Y0.stride(1) != 1:
            raise ChemError(ERR_INVALID, "Y0 and Yp must be planes of one shape and stride")
        out = torch.empty_like(Yp) if out is None else out
        self._raise(self.L.chem_surrogate_project(self.h, Yp.shape[1], _ptr(Y0), _ptr(Yp), Yp.stride(0),
                                                  _ptr(out), _stream(stream)))
        return out

    FWD_TC, FWD_FUSED, FWD_LAYERS = 0, 1, 2

    def surrogate_forward(self, X, impl=0, stream=None, check=False):
        """chem_surrogate_forward on an fp32 CUDA tensor X [B, 16] of normalised features:
        returns Y [B, 16] (and, with check=True, the tensor-core kernel's error word)."""
        import torch
        B = X.shape[0]
        Y = torch.empty((B, 16), dtype=torch.float32, device=X.device)
        err = C.c_int32(0)
        self._raise(self.L.chem_surrogate_forward(self.h, _ptr(X), B, _ptr(Y), impl, _stream(stream),
                                                  C.byref(err) if check else None))
        return (Y, err.value) if check else Y

    def ln_inv_kc(self, T, form=0, stream=None):
        """chem_diag_ln_inv_kc: ln(1 / K_c) of every reaction at the temperatures T (a
        float64 CUDA vector) as the mixed right-hand side (form 0) or the all-fp32 error
        test (form 1) forms it; returns a float64 [n, n_reactions] tensor."""
        import torch
        _check_f64_cuda("T", T)
        T = T.contiguous()
        out = torch.empty((T.numel(), int(self._mech.n_reactions)), dtype=torch.float64, device=T.device)
        self._raise(self.L.chem_diag_ln_inv_kc(self.h, int(form), T.numel(), _ptr(T), _ptr(out),
                                               _stream(stream)))
        return out

    def integrate_host(self, rho, e, Y, T, dt, rtol=1e-6, atol=1e-10, h=None, status=None,
                       nsteps=None, stream=None):
        """chem_integrate_host on numpy arrays (Y is [S, ld], C-contiguous planes);
        Y, T and the optional outputs are updated in place."""
        n = rho.size
        for nm, a in (("rho", rho), ("e", e), ("Y", Y), ("T", T)):
            if a.dtype != np.float64 or not a.flags.c_contiguous:
                raise ChemError(ERR_INVALID, f"{nm} must be a C-contiguous float64 array")

        def p(a):
            return None if a is None else C.c_void_p(a.ctypes.data)

        self._raise(self.L.chem_integrate_host(self.h, n, p(rho), p(e), p(Y), Y.strides[0] // 8, p(T),
                                               p(h), p(status), p(nsteps), float(dt), float(rtol),
                                               float(atol), _stream(stream)))
