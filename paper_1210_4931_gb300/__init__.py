"""Python binding of the GB300 messenger-field Wiener filter (include/wf.h).

Argument marshalling only: every step of the solve runs in the CUDA library
``libwf.so`` built from ``csrc/``.  There is no CPU fallback: importing this
package without the built library raises.

Device arrays are torch CUDA tensors (FP64 maps and harmonic vectors as
complex128 or as float64 views with a trailing re/im axis, uint8 masks); the
functions take the same arguments, in the same order, as the C functions.
"""
import ctypes
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libwf.so")

WF_OK, WF_EINVAL, WF_ENOMEM, WF_ECUDA, WF_ENOCONV, WF_EDIVERGE, WF_ETIMEOUT, WF_EUNSUPPORTED = range(8)
WF_GEOM_FLAT, WF_GEOM_HEALPIX = 0, 1
WF_PREC_FP64, WF_PREC_MIXED_FP32, WF_PREC_MIXED_TF32, WF_PREC_MIXED_SPLITBF16 = 0, 1, 2, 3
PRECISIONS = {"fp64": WF_PREC_FP64, "mixed": WF_PREC_MIXED_FP32, "fp32": WF_PREC_MIXED_FP32,
              "tf32": WF_PREC_MIXED_TF32, "bf16": WF_PREC_MIXED_SPLITBF16}


class WfError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s (status %d): %s" % (msg, status, last_error()))
        self.status = status


class wf_geometry(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("nside", ctypes.c_int), ("ncomp", ctypes.c_int)]


class wf_options(ctypes.Structure):
    _fields_ = [("maxiter", ctypes.c_int), ("level_cap", ctypes.c_int), ("eta", ctypes.c_double),
                ("ell0", ctypes.c_int), ("ell_step_max", ctypes.c_int), ("band_margin", ctypes.c_int),
                ("lambda_max", ctypes.c_double), ("refine_sweeps", ctypes.c_int), ("profile", ctypes.c_int),
                ("mixed_kappa", ctypes.c_double), ("mixed_lc", ctypes.c_int), ("schedule", ctypes.c_int),
                ("m_sigma", ctypes.c_double), ("stall_tol", ctypes.c_double),
                ("mixed_table_bytes", ctypes.c_longlong), ("fp64_emulation", ctypes.c_int),
                ("mixed_tol_factor", ctypes.c_double), ("tile_syn", ctypes.c_int), ("tile_ana", ctypes.c_int),
                ("mixed_correction", ctypes.c_double)]


class wf_info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("converged", ctypes.c_int), ("final_residual", ctypes.c_double),
                ("chi2_over_ndof", ctypes.c_double), ("n_dof", ctypes.c_longlong), ("tau", ctypes.c_double),
                ("n_levels", ctypes.c_int), ("refine_sweeps", ctypes.c_int), ("mixed_lc", ctypes.c_int),
                ("lambda_trace", ctypes.POINTER(ctypes.c_double)), ("L_trace", ctypes.POINTER(ctypes.c_int)),
                ("chi2_trace", ctypes.POINTER(ctypes.c_double)), ("resid_trace", ctypes.POINTER(ctypes.c_double)),
                ("iter_ms_trace", ctypes.POINTER(ctypes.c_double)), ("trace_cap", ctypes.c_int),
                ("launches", ctypes.c_longlong), ("kernel_ms", ctypes.c_double * 6),
                ("kernel_launches", ctypes.c_longlong * 6)]


KERNEL_FAMILIES = ["leg_syn", "ring_syn", "ring_ana", "leg_ana", "other", "flat"]

WF_REQ_WF, WF_REQ_FLUCT, WF_REQ_CR = 0, 1, 2
REQUEST_KINDS = {"wf": WF_REQ_WF, "fluct": WF_REQ_FLUCT, "cr": WF_REQ_CR}


class wf_request(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_ulonglong), ("kind", ctypes.c_int), ("nside", ctypes.c_int), ("lmax", ctypes.c_int),
                ("precision", ctypes.c_int), ("tol", ctypes.c_double), ("opt", wf_options),
                ("d", ctypes.c_void_p), ("noise_var", ctypes.c_void_p), ("mask", ctypes.c_void_p),
                ("C_ell", ctypes.c_void_p), ("g1", ctypes.c_void_p), ("g2", ctypes.c_void_p),
                ("s_out", ctypes.c_void_p), ("f_out", ctypes.c_void_p), ("ncomp", ctypes.c_int)]


class wf_result(ctypes.Structure):
    _fields_ = [("tag", ctypes.c_ulonglong), ("status", ctypes.c_int), ("iters", ctypes.c_int),
                ("converged", ctypes.c_int), ("final_residual", ctypes.c_double),
                ("chi2_over_ndof", ctypes.c_double), ("t_submit", ctypes.c_double), ("t_start", ctypes.c_double),
                ("t_done", ctypes.c_double), ("slot", ctypes.c_int), ("plan_reused", ctypes.c_int)]


class wf_batch_item(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("d", ctypes.c_void_p), ("noise_var", ctypes.c_void_p),
                ("mask", ctypes.c_void_p), ("C_ell", ctypes.c_void_p), ("g1", ctypes.c_void_p),
                ("g2", ctypes.c_void_p), ("tol", ctypes.c_double), ("s_out", ctypes.c_void_p),
                ("alm_out", ctypes.c_void_p), ("info", ctypes.c_void_p)]


class wf_server_stats(ctypes.Structure):
    _fields_ = [("pending", ctypes.c_longlong), ("active", ctypes.c_longlong), ("completed", ctypes.c_longlong),
                ("rejected", ctypes.c_longlong), ("bytes_in_use", ctypes.c_longlong),
                ("peak_bytes", ctypes.c_longlong), ("budget", ctypes.c_longlong), ("plans", ctypes.c_int),
                ("max_active", ctypes.c_int), ("plans_created", ctypes.c_longlong),
                ("plans_evicted", ctypes.c_longlong)]


_lib = None
ABI_STRUCTS = (wf_geometry, wf_options, wf_info, wf_batch_item, wf_request, wf_result, wf_server_stats)

EXPORTS = ["wf_plan_create", "wf_plan_destroy", "wf_set_options", "wf_set_schedule", "wf_set_start", "wf_solve", "wf_solve_host",
           "wf_fluct", "wf_alm2map", "wf_map2alm_adjoint", "wf_npix", "wf_nalm", "wf_plan_device_bytes",
           "wf_strerror", "wf_last_error", "wf_flat_solve_noalloc", "wf_remove_templates", "wf_fluct_host",
           "wf_plan_estimate_bytes", "wf_plan_set_stream", "wf_server_create", "wf_server_submit", "wf_server_poll",
           "wf_server_wait", "wf_server_get_stats", "wf_server_destroy", "wf_solve_batch", "wf_plan_autotune",
           "wf_plan_tiles", "wf_probe_fp32_fma", "wf_combine_datasets", "wf_abi_sizeof"]


def load(path: str = LIB_PATH):
    """Load libwf.so; raises if it has not been built (no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError("libwf.so is not built (run __graft_entry__.build()); there is no CPU fallback")
    L = ctypes.CDLL(path)
    vp, dp, u8p = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p
    L.wf_plan_create.argtypes = [ctypes.POINTER(wf_geometry), ctypes.c_int, ctypes.c_int, vp, ctypes.POINTER(vp)]
    L.wf_plan_destroy.argtypes = [vp]
    L.wf_plan_destroy.restype = None
    L.wf_set_options.argtypes = [vp, ctypes.POINTER(wf_options)]
    L.wf_set_schedule.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int), ctypes.c_int]
    L.wf_set_start.argtypes = [vp, dp]
    sig = [vp, dp, dp, u8p, dp, ctypes.c_double, dp, dp, ctypes.POINTER(wf_info)]
    L.wf_solve.argtypes = sig
    L.wf_solve_host.argtypes = sig
    L.wf_fluct.argtypes = [vp, dp, u8p, dp, dp, dp, ctypes.c_double, dp, dp, ctypes.POINTER(wf_info)]
    L.wf_alm2map.argtypes = [vp, dp, ctypes.c_int, dp]
    L.wf_map2alm_adjoint.argtypes = [vp, dp, ctypes.c_int, dp]
    for f in ("wf_npix", "wf_nalm", "wf_plan_device_bytes"):
        getattr(L, f).argtypes = [vp]
        getattr(L, f).restype = ctypes.c_longlong
    L.wf_flat_solve_noalloc.argtypes = [ctypes.c_int, dp, dp, u8p, dp, ctypes.c_double, ctypes.POINTER(wf_options),
                                        vp, dp, dp, ctypes.POINTER(wf_info)]
    L.wf_flat_solve_noalloc.restype = ctypes.c_int
    L.wf_remove_templates.argtypes = [vp, dp, u8p, dp, ctypes.POINTER(ctypes.c_double)]
    L.wf_remove_templates.restype = ctypes.c_int
    L.wf_fluct_host.argtypes = [vp, dp, u8p, dp, dp, dp, ctypes.c_double, dp, dp, ctypes.POINTER(wf_info)]
    L.wf_fluct_host.restype = ctypes.c_int
    L.wf_plan_estimate_bytes.argtypes = [ctypes.POINTER(wf_geometry), ctypes.c_int, ctypes.c_int, ctypes.c_int]
    L.wf_plan_estimate_bytes.restype = ctypes.c_longlong
    L.wf_plan_set_stream.argtypes = [vp, vp]
    L.wf_plan_set_stream.restype = ctypes.c_int
    L.wf_server_create.argtypes = [ctypes.c_int, ctypes.c_longlong, ctypes.c_int, ctypes.POINTER(vp)]
    L.wf_server_create.restype = ctypes.c_int
    L.wf_server_submit.argtypes = [vp, ctypes.POINTER(wf_request)]
    L.wf_server_submit.restype = ctypes.c_int
    L.wf_server_poll.argtypes = [vp, ctypes.POINTER(wf_result), ctypes.c_int]
    L.wf_server_poll.restype = ctypes.c_int
    L.wf_server_wait.argtypes = [vp, ctypes.POINTER(wf_result), ctypes.c_int, ctypes.c_double]
    L.wf_server_wait.restype = ctypes.c_int
    L.wf_server_get_stats.argtypes = [vp, ctypes.POINTER(wf_server_stats)]
    L.wf_server_get_stats.restype = ctypes.c_int
    L.wf_plan_autotune.argtypes = [vp, ctypes.c_int]
    L.wf_plan_autotune.restype = ctypes.c_int
    L.wf_plan_tiles.argtypes = [vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    L.wf_plan_tiles.restype = ctypes.c_int
    L.wf_solve_batch.argtypes = [ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(wf_batch_item), vp,
                                 ctypes.POINTER(ctypes.c_int)]
    L.wf_solve_batch.restype = ctypes.c_int
    L.wf_server_destroy.argtypes = [vp]
    L.wf_server_destroy.restype = None
    L.wf_combine_datasets.argtypes = [vp, ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                      dp, dp, u8p]
    L.wf_combine_datasets.restype = ctypes.c_int
    L.wf_probe_fp32_fma.argtypes = [vp, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]
    L.wf_probe_fp32_fma.restype = ctypes.c_int
    L.wf_strerror.argtypes = [ctypes.c_int]
    L.wf_strerror.restype = ctypes.c_char_p
    L.wf_last_error.argtypes = []
    L.wf_last_error.restype = ctypes.c_char_p
    L.wf_abi_sizeof.argtypes = [ctypes.c_char_p]
    L.wf_abi_sizeof.restype = ctypes.c_longlong
    # the structs above mirror include/wf.h field by field: a library built from another
    # header would read them wrongly, so their sizes must agree before any call passes one
    for st in ABI_STRUCTS:
        n = L.wf_abi_sizeof(st.__name__.encode())
        if n != ctypes.sizeof(st):
            raise ImportError("%s: %d bytes in libwf.so, %d in this binding (rebuild the library)"
                              % (st.__name__, n, ctypes.sizeof(st)))
    for f in ("wf_plan_create", "wf_set_options", "wf_set_schedule", "wf_solve", "wf_solve_host", "wf_fluct",
              "wf_alm2map", "wf_map2alm_adjoint"):
        getattr(L, f).restype = ctypes.c_int
    _lib = L
    return L


def wf_combine_datasets(plan, d_list, noise_list, mask_list, d_out, noise_out, mask_out):
    """Inverse-noise-weighted combination of k data sets of one signal (see
    include/wf.h); every map is a CUDA tensor of npix entries (masks uint8,
    None entries: all observed)."""
    k = len(d_list)
    if not (len(noise_list) == k and (mask_list is None or len(mask_list) == k)):
        raise ValueError("d_list, noise_list and mask_list must have the same length")
    n8 = plan.npix * 8
    arr = ctypes.c_void_p * k
    dp_ = arr(*[_ptr(x, None, n8, "d") for x in d_list])
    np_ = arr(*[_ptr(x, None, n8, "noise_var") for x in noise_list])
    mp_ = arr(*[_ptr(x, None, plan.npix, "mask") for x in mask_list]) if mask_list is not None else None
    _check(load().wf_combine_datasets(plan.handle, k, dp_, np_, mp_, _ptr(d_out, None, n8, "d_out"),
                                      _ptr(noise_out, None, n8, "noise_out"), _ptr(mask_out, None, plan.npix,
                                                                                    "mask_out")),
           "wf_combine_datasets")


def wf_probe_fp32_fma(packed: bool = True, stream=None) -> float:
    """Measured FP32 FMA throughput of this GPU in TFLOP/s (see include/wf.h)."""
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    out = ctypes.c_double(0.0)
    _check(load().wf_probe_fp32_fma(ctypes.c_void_p(stream.cuda_stream), int(bool(packed)), ctypes.byref(out)),
           "wf_probe_fp32_fma")
    return float(out.value)


def last_error() -> str:
    return (_lib.wf_last_error() or b"").decode() if _lib is not None else ""


def _ptr(t, dtype=None, n=None, what="array"):
    """Device pointer of a contiguous torch CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA torch tensor" % what)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % what)
    if dtype is not None and t.dtype not in dtype:
        raise TypeError("%s has dtype %s" % (what, t.dtype))
    if n is not None and t.numel() * t.element_size() < n:
        raise ValueError("%s is too small (%d bytes, need %d)" % (what, t.numel() * t.element_size(), n))
    return ctypes.c_void_p(t.data_ptr())


class Plan:
    """Owns one wf_plan (freed on close / garbage collection)."""

    def __init__(self, handle, geometry, lmax, precision):
        self.handle = handle
        self.geometry = geometry
        self.lmax = lmax
        self.precision = precision
        self.npix = int(load().wf_npix(handle))
        self.nalm = int(load().wf_nalm(handle))
        self.ncomp = int(geometry.get("ncomp", 1))

    @property
    def sizes(self):
        """Bytes of (a map argument, the noise argument, a harmonic argument):
        polarised plans take 3 maps, 6 noise maps and 3 harmonic vectors."""
        nc = self.ncomp
        return nc * self.npix * 8, (6 if nc == 3 else 1) * self.npix * 8, nc * self.nalm * 16

    @property
    def device_bytes(self):
        return int(load().wf_plan_device_bytes(self.handle))

    def close(self):
        if self.handle:
            load().wf_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _check(st, what, allow=()):
    if st != WF_OK and st not in allow:
        raise WfError(st, what)
    return st


def wf_plan_create(kind: str, *, nside: int = 0, lmax: int = 0, n: int = 0, precision: str = "fp64",
                   stream=None, ncomp: int = 1) -> Plan:
    """kind 'healpix' (nside, lmax) or 'flat' (n x n); ncomp 3 for polarised
    (I, Q, U) HEALPix plans (FP64).  stream: torch CUDA stream (default: the
    current stream)."""
    import torch

    L = load()
    g = wf_geometry()
    g.kind = WF_GEOM_HEALPIX if kind == "healpix" else WF_GEOM_FLAT
    g.nside, g.nx, g.ny, g.ncomp = nside, n, n, int(ncomp)
    if stream is None:
        stream = torch.cuda.current_stream()
    h = ctypes.c_void_p()
    _check(L.wf_plan_create(ctypes.byref(g), lmax, PRECISIONS[precision], ctypes.c_void_p(stream.cuda_stream),
                            ctypes.byref(h)), "wf_plan_create")
    return Plan(h, {"kind": kind, "nside": nside, "n": n, "ncomp": int(ncomp)}, lmax, precision)


def wf_plan_destroy(plan: Plan):
    plan.close()


def wf_set_options(plan: Plan, **kw):
    o = wf_options()
    for k, v in kw.items():
        setattr(o, k, v)
    _check(load().wf_set_options(plan.handle, ctypes.byref(o)), "wf_set_options")


def solve_record(rep: dict, **meta) -> dict:
    """One solve's metrics as a JSON-ready dict: iterations, per-iteration time
    p50 / p99 (ms, when the plan profiled), the (lambda, L) trace, chi^2 / n_dof,
    the final residual, status and launches; ``meta`` (e.g. the geometry, or
    an error against a reference) is merged in."""
    ms = rep.get("iter_ms_trace")
    rec = {"status": int(rep["status"]), "iters": int(rep["iters"]), "converged": bool(rep["converged"]),
           "final_residual": float(rep["final_residual"]), "chi2_over_ndof": float(rep["chi2_over_ndof"]),
           "n_dof": int(rep["n_dof"]), "tau": float(rep["tau"]), "launches": int(rep["launches"]),
           "refine_sweeps": int(rep["refine_sweeps"]), "mixed_lc": int(rep["mixed_lc"])}
    if ms is not None and len(ms) and np.all(np.isfinite(ms)) and np.any(ms > 0):
        rec["iter_ms_p50"] = float(np.percentile(ms, 50))
        rec["iter_ms_p99"] = float(np.percentile(ms, 99))
    if rep.get("lambda_trace") is not None:
        rec["lambda_trace"] = [float(x) for x in rep["lambda_trace"]]
        rec["L_trace"] = [int(x) for x in rep["L_trace"]]
    rec.update(meta)
    return rec


def append_jsonl(path: str, rep: dict, **meta) -> dict:
    """Append solve_record(rep, **meta) to a JSON-lines log; returns the record."""
    import json

    rec = solve_record(rep, **meta)
    with open(path, "a") as fh:
        fh.write(json.dumps(rec) + "\n")
    return rec


def wf_set_start(plan: Plan, alm0=None):
    """Start the next solves on this plan from alm0 (a CUDA complex128 tensor in
    the alm_out layout, kept referenced here) instead of zero; None clears."""
    n = plan.nalm * 16 * plan.ncomp
    _check(load().wf_set_start(plan.handle, _ptr(alm0, None, n, "alm0")), "wf_set_start")
    plan._start = alm0


def wf_set_schedule(plan: Plan, lam, L=None):
    lam = np.ascontiguousarray(lam, dtype=np.float64)
    n = lam.size
    Lp = None
    if L is not None:
        Larr = np.ascontiguousarray(L, dtype=np.int32)
        Lp = Larr.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    _check(load().wf_set_schedule(plan.handle, lam.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), Lp, n),
           "wf_set_schedule")


def _info(cap):
    info = wf_info()
    bufs = {}
    if cap:
        bufs = {"lambda": np.full(cap, np.nan), "L": np.full(cap, -1, dtype=np.int32),
                "chi2": np.full(cap, np.nan), "resid": np.full(cap, np.nan), "iter_ms": np.full(cap, np.nan)}
        info.iter_ms_trace = bufs["iter_ms"].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        info.lambda_trace = bufs["lambda"].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        info.L_trace = bufs["L"].ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        info.chi2_trace = bufs["chi2"].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        info.resid_trace = bufs["resid"].ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        info.trace_cap = cap
    return info, bufs


def _info_dict(st, info, bufs):
    k = info.iters
    out = {"status": st, "iters": k, "converged": bool(info.converged), "final_residual": info.final_residual,
           "chi2_over_ndof": info.chi2_over_ndof, "n_dof": info.n_dof, "tau": info.tau,
           "n_levels": info.n_levels, "refine_sweeps": info.refine_sweeps, "mixed_lc": info.mixed_lc,
           "launches": info.launches,
           "kernel_ms": {f: info.kernel_ms[i] for i, f in enumerate(KERNEL_FAMILIES)},
           "kernel_launches": {f: info.kernel_launches[i] for i, f in enumerate(KERNEL_FAMILIES)}}
    for key, v in bufs.items():
        out[key + "_trace"] = v[: min(k, v.size)].copy()
    return out


def _f64(t):
    import torch

    return (torch.float64, torch.complex128)


def wf_solve(plan: Plan, d, noise_var, mask, C_ell, tol, s_wf, alm_out=None, trace_cap=0) -> dict:
    """Wiener filter; returns the report as a dict (status WF_OK or
    WF_ENOCONV; other statuses raise)."""
    info, bufs = _info(trace_cap)
    n8, nn, nh = plan.sizes
    st = load().wf_solve(plan.handle, _ptr(d, _f64(d), n8, "d"), _ptr(noise_var, _f64(d), nn, "noise_var"),
                         _ptr(mask, None, plan.npix, "mask"), _ptr(C_ell, _f64(d), None, "C_ell"), float(tol),
                         _ptr(s_wf, _f64(d), n8, "s_wf"), _ptr(alm_out, _f64(d), nh, "alm_out"),
                         ctypes.byref(info))
    _check(st, "wf_solve", allow=(WF_ENOCONV,))
    return _info_dict(st, info, bufs)


def wf_solve_host(plan: Plan, d, noise_var, mask, C_ell, tol, s_wf, alm_out=None, trace_cap=0) -> dict:
    """wf_solve on host numpy arrays; the library copies in and out."""
    info, bufs = _info(trace_cap)

    def hp(a, dt, n=None):
        if a is None:
            return None
        assert a.dtype == dt and a.flags.c_contiguous
        if n is not None and a.nbytes < n:
            raise ValueError("host array too small (%d bytes, need %d)" % (a.nbytes, n))
        return ctypes.c_void_p(a.ctypes.data)

    n8, nn, nh = plan.sizes

    st = load().wf_solve_host(plan.handle, hp(d, np.float64, n8), hp(noise_var, np.float64, nn),
                              hp(mask, np.uint8, plan.npix), hp(C_ell, np.float64), float(tol),
                              hp(s_wf, np.float64, n8), hp(alm_out, np.complex128, nh), ctypes.byref(info))
    _check(st, "wf_solve_host", allow=(WF_ENOCONV,))
    return _info_dict(st, info, bufs)


def wf_fluct(plan: Plan, noise_var, mask, C_ell, g1, g2, tol, f_out, alm_out=None, trace_cap=0) -> dict:
    info, bufs = _info(trace_cap)
    n8, nn, nh = plan.sizes
    st = load().wf_fluct(plan.handle, _ptr(noise_var, None, nn, "noise_var"), _ptr(mask, None, plan.npix, "mask"),
                         _ptr(C_ell, None, None, "C_ell"), _ptr(g1, None, n8, "g1"),
                         _ptr(g2, None, nh, "g2"), float(tol), _ptr(f_out, None, n8, "f_out"),
                         _ptr(alm_out, None, nh, "alm_out"), ctypes.byref(info))
    _check(st, "wf_fluct", allow=(WF_ENOCONV,))
    return _info_dict(st, info, bufs)


def wf_flat_solve_noalloc(n, d, noise_var, mask, S, tol, s_wf, alm_out=None, trace_cap=0, stream=None,
                          **options) -> dict:
    """Flat-grid solve that allocates no device memory (see include/wf.h):
    same arguments as wf_solve without a plan; n <= 128."""
    import torch

    info, bufs = _info(trace_cap)
    o = wf_options()
    for k, v in options.items():
        setattr(o, k, v)
    if stream is None:
        stream = torch.cuda.current_stream()
    n8 = n * n * 8
    st = load().wf_flat_solve_noalloc(int(n), _ptr(d, None, n8, "d"), _ptr(noise_var, None, n8, "noise_var"),
                                      _ptr(mask, None, n * n, "mask"), _ptr(S, None, None, "S"), float(tol),
                                      ctypes.byref(o), ctypes.c_void_p(stream.cuda_stream),
                                      _ptr(s_wf, None, n8, "s_wf"),
                                      _ptr(alm_out, None, n * (n // 2 + 1) * 16, "alm_out"), ctypes.byref(info))
    _check(st, "wf_flat_solve_noalloc", allow=(WF_ENOCONV,))
    return _info_dict(st, info, bufs)


def wf_fluct_host(plan: Plan, noise_var, mask, C_ell, g1, g2, tol, f_out, alm_out=None, trace_cap=0) -> dict:
    """wf_fluct with numpy (host) arrays; copies are made inside the call."""
    info, bufs = _info(trace_cap)

    def hp(a, dt, n=None):
        if a is None:
            return None
        assert a.dtype == dt and a.flags.c_contiguous
        if n is not None and a.nbytes < n:
            raise ValueError("host array too small (%d bytes, need %d)" % (a.nbytes, n))
        return ctypes.c_void_p(a.ctypes.data)

    n8, nn, nh = plan.sizes

    st = load().wf_fluct_host(plan.handle, hp(noise_var, np.float64, nn), hp(mask, np.uint8, plan.npix),
                              hp(C_ell, np.float64), hp(g1, np.float64, n8), hp(g2, np.complex128, nh), float(tol),
                              hp(f_out, np.float64, n8), hp(alm_out, np.complex128, nh), ctypes.byref(info))
    _check(st, "wf_fluct_host", allow=(WF_ENOCONV,))
    return _info_dict(st, info, bufs)


def wf_plan_autotune(plan: Plan, reps: int = 3) -> tuple:
    """Time the mixed Legendre tile variants on this plan and keep the fastest;
    returns (synthesis pairs per thread, analysis pairs per lane)."""
    _check(load().wf_plan_autotune(plan.handle, int(reps)), "wf_plan_autotune")
    return wf_plan_tiles(plan)


def wf_plan_tiles(plan: Plan) -> tuple:
    s, a = ctypes.c_int(), ctypes.c_int()
    _check(load().wf_plan_tiles(plan.handle, ctypes.byref(s), ctypes.byref(a)), "wf_plan_tiles")
    return int(s.value), int(a.value)


def wf_solve_batch(plans, items, trace_cap=0, stream=None) -> list:
    """Several solves advanced together (one CUDA graph per step).  items:
    dicts with kind ('wf' or 'fluct'), d / g1 / g2, noise_var, mask, C_ell, tol,
    s_out and optional alm_out (CUDA tensors; polarised plans take the
    three-component layouts of wf_solve / wf_fluct).  Returns one report per
    item (with its 'status'); argument or CUDA errors of the batch raise."""
    import torch

    n = len(plans)
    assert len(items) == n
    arr = (wf_batch_item * n)()
    hv = (ctypes.c_void_p * n)(*[pl.handle for pl in plans])
    st = (ctypes.c_int * n)()
    infos = []
    for i, (pl, it) in enumerate(zip(plans, items)):
        info, bufs = _info(trace_cap)
        infos.append((info, bufs))
        n8, nn, nh = pl.sizes
        b = arr[i]
        b.kind = REQUEST_KINDS[it.get("kind", "wf")]
        b.d = _ptr(it.get("d"), None, n8, "d")
        b.noise_var = _ptr(it["noise_var"], None, nn, "noise_var")
        b.mask = _ptr(it.get("mask"), None, pl.npix, "mask")
        b.C_ell = _ptr(it["C_ell"], None, None, "C_ell")
        b.g1 = _ptr(it.get("g1"), None, n8, "g1")
        b.g2 = _ptr(it.get("g2"), None, nh, "g2")
        b.tol = float(it["tol"])
        b.s_out = _ptr(it["s_out"], None, n8, "s_out")
        b.alm_out = _ptr(it.get("alm_out"), None, nh, "alm_out")
        b.info = ctypes.cast(ctypes.byref(info), ctypes.c_void_p)
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(load().wf_solve_batch(n, hv, arr, ctypes.c_void_p(stream.cuda_stream), st), "wf_solve_batch")
    out = []
    for i in range(n):
        info, bufs = infos[i]
        out.append(_info_dict(int(st[i]), info, bufs))
    return out


def wf_plan_estimate_bytes(kind: str, *, nside: int = 0, lmax: int = 0, n: int = 0, precision: str = "fp64",
                           host_staging: bool = True, ncomp: int = 1) -> int:
    g = wf_geometry()
    if kind == "healpix":
        g.kind, g.nside, g.ncomp = WF_GEOM_HEALPIX, nside, int(ncomp)
    else:
        g.kind, g.nx, g.ny, g.ncomp = WF_GEOM_FLAT, n, n, 1
    return int(load().wf_plan_estimate_bytes(ctypes.byref(g), int(lmax), PRECISIONS[precision], int(host_staging)))


class Server:
    """The request loop of include/wf.h (wf_server_*): host numpy buffers in,
    results with timings out.  Buffers are held here until their result has
    been collected."""

    def __init__(self, device: int = 0, mem_budget: int = 8 << 30, slots: int = 4):
        h = ctypes.c_void_p()
        _check(load().wf_server_create(int(device), int(mem_budget), int(slots), ctypes.byref(h)), "wf_server_create")
        self.handle = h
        self._held = {}
        self._next = 1

    def submit(self, kind: str, *, nside: int, lmax: int, noise_var, C_ell, s_out, d=None, mask=None, g1=None,
               g2=None, f_out=None, precision: str = "mixed", tol: float = 1e-6, tag=None, ncomp: int = 1,
               **options) -> int:
        def hp(a, dt):
            if a is None:
                return None
            if a.dtype != dt or not a.flags.c_contiguous:
                raise TypeError("request buffers must be C-contiguous %s arrays" % np.dtype(dt).name)
            return a.ctypes.data

        r = wf_request()
        if tag is None:
            tag = self._next
            self._next += 1
        r.tag, r.kind, r.nside, r.lmax = int(tag), REQUEST_KINDS[kind], int(nside), int(lmax)
        r.precision, r.tol, r.ncomp = PRECISIONS[precision], float(tol), int(ncomp)
        for k, v in options.items():
            setattr(r.opt, k, v)
        r.d, r.noise_var, r.mask = hp(d, np.float64), hp(noise_var, np.float64), hp(mask, np.uint8)
        r.C_ell, r.g1, r.g2 = hp(C_ell, np.float64), hp(g1, np.float64), hp(g2, np.complex128)
        r.s_out, r.f_out = hp(s_out, np.float64), hp(f_out, np.float64)
        self._held[int(tag)] = (d, noise_var, mask, C_ell, g1, g2, s_out, f_out)
        _check(load().wf_server_submit(self.handle, ctypes.byref(r)), "wf_server_submit")
        return int(tag)

    def _collect(self, arr, n):
        out = []
        for i in range(n):
            x = arr[i]
            self._held.pop(int(x.tag), None)
            out.append({"tag": int(x.tag), "status": int(x.status), "iters": int(x.iters),
                        "converged": bool(x.converged), "final_residual": float(x.final_residual),
                        "chi2_over_ndof": float(x.chi2_over_ndof), "t_submit": float(x.t_submit),
                        "t_start": float(x.t_start), "t_done": float(x.t_done), "slot": int(x.slot),
                        "plan_reused": bool(x.plan_reused)})
        return out

    def poll(self, cap: int = 256) -> list:
        arr = (wf_result * cap)()
        return self._collect(arr, load().wf_server_poll(self.handle, arr, cap))

    def wait(self, cap: int = 256, timeout: float = 1.0) -> list:
        arr = (wf_result * cap)()
        return self._collect(arr, load().wf_server_wait(self.handle, arr, cap, float(timeout)))

    def stats(self) -> dict:
        s = wf_server_stats()
        _check(load().wf_server_get_stats(self.handle, ctypes.byref(s)), "wf_server_get_stats")
        return {f: int(getattr(s, f)) for f, _ in s._fields_}

    def close(self):
        if self.handle:
            load().wf_server_destroy(self.handle)
            self.handle = None
            self._held.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def wf_remove_templates(plan: Plan, d_raw, mask, d_out):
    """Monopole/dipole marginalisation of Eq. (12); returns the 4 removed
    template amplitudes (monopole, dipole x, y, z)."""
    coef = (ctypes.c_double * 4)()
    n8 = plan.npix * 8
    _check(load().wf_remove_templates(plan.handle, _ptr(d_raw, None, n8, "d_raw"), _ptr(mask, None, plan.npix, "mask"),
                                      _ptr(d_out, None, n8, "d_out"), coef), "wf_remove_templates")
    return np.array(list(coef))


def wf_alm2map(plan: Plan, alm, L, map_out):
    _check(load().wf_alm2map(plan.handle, _ptr(alm, None, plan.nalm * 16, "alm"), int(L),
                             _ptr(map_out, None, plan.npix * 8, "map")), "wf_alm2map")


def wf_map2alm_adjoint(plan: Plan, map_in, L, alm_out):
    _check(load().wf_map2alm_adjoint(plan.handle, _ptr(map_in, None, plan.npix * 8, "map"), int(L),
                                     _ptr(alm_out, None, plan.nalm * 16, "alm")), "wf_map2alm_adjoint")


__all__ = ["Plan", "Server", "WfError", "load", "wf_fluct_host", "wf_plan_estimate_bytes", "wf_solve_batch", "wf_plan_autotune", "wf_plan_tiles", "wf_alm2map", "wf_flat_solve_noalloc", "wf_remove_templates", "wf_fluct", "wf_map2alm_adjoint", "wf_plan_create",
           "wf_plan_destroy", "wf_set_options", "wf_set_schedule", "wf_solve", "wf_solve_host", "EXPORTS",
           "LIB_PATH"]
