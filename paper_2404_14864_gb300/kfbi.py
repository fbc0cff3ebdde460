"""Thin ctypes binding of the KFBI C ABI (``include/kfbi.h``).

Argument marshalling only: every step of the operator application and of
the time steppers runs in the library's CUDA kernels.  Device buffers are
torch CUDA tensors (float64 or complex128, contiguous); streams are torch
CUDA streams (default: the current stream).  The library must have been
built (``paper_2404_14864_gb300.build.build()``); there is no fallback.
"""

import ctypes
import math
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libkfbi.so")

KFBI_OK = 0
(KFBI_ERR_ARG, KFBI_ERR_GEOMETRY, KFBI_ERR_OOM, KFBI_ERR_NOT_CONVERGED, KFBI_ERR_NONFINITE,
 KFBI_ERR_TIMEOUT, KFBI_ERR_CUDA, KFBI_ERR_UNSUPPORTED) = range(1, 9)
STATUS_NAMES = {0: "KFBI_OK", 1: "KFBI_ERR_ARG", 2: "KFBI_ERR_GEOMETRY", 3: "KFBI_ERR_OOM",
                4: "KFBI_ERR_NOT_CONVERGED", 5: "KFBI_ERR_NONFINITE", 6: "KFBI_ERR_TIMEOUT",
                7: "KFBI_ERR_CUDA", 8: "KFBI_ERR_UNSUPPORTED"}
KFBI_FP64, KFBI_MIXED_TF32, KFBI_MIXED_FFT32 = 0, 1, 2
KFBI_GMRES, KFBI_RICHARDSON = 0, 1
KFBI_CURVE_POLAR, KFBI_CURVE_ELLIPSE = 0, 1
KFBI_HEAT, KFBI_WAVE, KFBI_SCHRODINGER = 0, 1, 2

PLAN_FIELDS = {
    "edge_i": (1, np.int32), "edge_j": (2, np.int32), "edge_dir": (3, np.int32),
    "edge_coord": (4, np.float64), "edge_theta": (5, np.float64), "inside": (6, np.uint8),
    "irregular": (8, np.int32), "arm_node": (10, np.int32), "arm_k0": (11, np.int32),
    "arm_alpha": (12, np.float64), "arm_beta": (13, np.float64), "arm_fidx": (14, np.int32),
    "arm_fcoef": (15, np.float64), "node_gidx": (16, np.int32), "node_w": (17, np.float64),
    "node_a": (18, np.float64), "node_b": (19, np.float64), "node_fidx": (20, np.int32),
    "node_fcoef": (21, np.float64),
    "arm_delta": (22, np.float64), "node_wn": (23, np.float64), "node_e": (24, np.float64),
    "node_fcoef_n": (25, np.float64),
}


class KfbiError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, status), msg))
        self.status = status


class DomainDesc(ctypes.Structure):
    _fields_ = [("M", ctypes.c_int), ("box_lo", ctypes.c_double), ("box_hi", ctypes.c_double),
                ("n_boundary", ctypes.c_int), ("curve_kind", ctypes.c_int),
                ("cx", ctypes.c_double), ("cy", ctypes.c_double),
                ("params", ctypes.c_double * 6), ("precision", ctypes.c_int),
                ("gmres_restart", ctypes.c_int), ("gmres_tol", ctypes.c_double),
                ("gmres_maxit", ctypes.c_int), ("solver", ctypes.c_int),
                ("richardson_gamma", ctypes.c_double)]


class SolveInfo(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("rel_residual", ctypes.c_double),
                ("converged", ctypes.c_int), ("applications", ctypes.c_int)]

    def as_dict(self):
        return {"iters": self.iters, "rel_residual": self.rel_residual,
                "converged": bool(self.converged), "applications": self.applications}


class ServerDesc(ctypes.Structure):
    _fields_ = [("max_resident", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_longlong),
                ("hbm_reserve_bytes", ctypes.c_longlong), ("gmres_restart", ctypes.c_int),
                ("plan_threads", ctypes.c_int), ("lanes", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("domain", DomainDesc), ("equation", ctypes.c_int), ("steps", ctypes.c_int),
                ("dt", ctypes.c_double), ("theta", ctypes.c_double), ("arrival", ctypes.c_double),
                ("u0", ctypes.c_void_p), ("lap_u0", ctypes.c_void_p), ("u1", ctypes.c_void_p),
                ("lap_u1", ctypes.c_void_p), ("g", ctypes.c_void_p), ("src_init", ctypes.c_void_p),
                ("src_profile", ctypes.c_void_p), ("src_coef", ctypes.c_void_p),
                ("potential", ctypes.c_void_p), ("u_out", ctypes.c_void_p)]


class RequestInfo(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int), ("status", ctypes.c_int), ("arrival", ctypes.c_double),
                ("admitted", ctypes.c_double), ("finished", ctypes.c_double),
                ("admit_tick", ctypes.c_int), ("finish_tick", ctypes.c_int),
                ("steps_done", ctypes.c_int), ("max_iters", ctypes.c_int),
                ("max_rel_residual", ctypes.c_double), ("device_bytes", ctypes.c_longlong)]


class ServerStats(ctypes.Structure):
    _fields_ = [("ticks", ctypes.c_int), ("admitted", ctypes.c_int), ("completed", ctypes.c_int),
                ("failed", ctypes.c_int), ("busy_seconds", ctypes.c_double),
                ("admit_seconds", ctypes.c_double), ("resident_ticks", ctypes.c_double),
                ("peak_device_bytes", ctypes.c_longlong), ("h2d_bytes", ctypes.c_longlong),
                ("d2h_bytes", ctypes.c_longlong), ("grid_point_steps", ctypes.c_double)]


REQ_QUEUED, REQ_RESIDENT, REQ_DONE, REQ_FAILED = 0, 1, 2, 3


class BatchTuning(ctypes.Structure):
    _fields_ = [("engine", ctypes.c_int), ("M", ctypes.c_int), ("instances", ctypes.c_int),
                ("n_candidates", ctypes.c_int), ("chosen", ctypes.c_int),
                ("param", (ctypes.c_int * 2) * 4), ("us", ctypes.c_double * 4)]

    def as_dict(self):
        n = int(self.n_candidates)
        if self.engine == 1:
            cands = [{"rows_per_block": int(self.param[c][0]), "us": float(self.us[c])}
                     for c in range(n)]
        else:
            cands = [{"tile_order": int(self.param[c][0]), "ctas": int(self.param[c][1]),
                      "us": float(self.us[c])} for c in range(n)]
        return {"engine": "fft32" if self.engine == 1 else "tf32", "M": int(self.M),
                "instances": int(self.instances), "chosen": int(self.chosen),
                "candidates": cands}

_lib = None
_VP = ctypes.c_void_p


def lib():
    """Load libkfbi.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libkfbi.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    S = ctypes.c_int
    sig = {
        "kfbi_create_domain": (S, [ctypes.POINTER(DomainDesc), _VP, ctypes.POINTER(_VP)]),
        "kfbi_destroy_domain": (None, [_VP]),
        "kfbi_apply_operator": (S, [_VP, ctypes.c_double, ctypes.c_double, _VP, _VP, _VP, _VP]),
        "kfbi_interface_solve": (S, [_VP, ctypes.c_double, ctypes.c_double, _VP, _VP, _VP, _VP, _VP]),
        "kfbi_solve_density": (S, [_VP, ctypes.c_double, ctypes.c_double, _VP, _VP,
                                   ctypes.POINTER(SolveInfo), _VP]),
        "kfbi_apply_neumann": (S, [_VP, ctypes.c_double, ctypes.c_double, _VP, _VP, _VP, _VP]),
        "kfbi_solve_neumann": (S, [_VP, ctypes.c_double, ctypes.c_double, _VP, _VP, _VP, _VP,
                                   ctypes.POINTER(SolveInfo), _VP]),
        "kfbi_state_create": (S, [_VP, ctypes.c_int, ctypes.POINTER(_VP)]),
        "kfbi_state_set_neumann": (S, [_VP, ctypes.c_int]),
        "kfbi_state_set_w": (S, [_VP, ctypes.c_double]),
        "kfbi_state_blob_bytes": (ctypes.c_longlong, [_VP]),
        "kfbi_state_export": (S, [_VP, _VP, ctypes.c_longlong]),
        "kfbi_state_import": (S, [_VP, _VP, ctypes.c_longlong]),
        "kfbi_state_destroy": (None, [_VP]),
        "kfbi_state_init_heat": (S, [_VP, ctypes.c_double, _VP, _VP, _VP, _VP]),
        "kfbi_state_init_wave": (S, [_VP, ctypes.c_double, ctypes.c_double, _VP, _VP, _VP, _VP, _VP]),
        "kfbi_state_init_schrodinger": (S, [_VP, ctypes.c_double, _VP, _VP, _VP]),
        "kfbi_step_heat": (S, [_VP, _VP, _VP, _VP, ctypes.POINTER(SolveInfo), _VP]),
        "kfbi_step_wave": (S, [_VP, _VP, _VP, ctypes.POINTER(SolveInfo), _VP]),
        "kfbi_step_schrodinger": (S, [_VP, _VP, _VP, ctypes.c_double, _VP,
                                      ctypes.POINTER(SolveInfo), _VP]),
        "kfbi_state_get_u": (S, [_VP, _VP, _VP]),
        "kfbi_state_get_phi": (S, [_VP, _VP, _VP]),
        "kfbi_last_error": (ctypes.c_char_p, [_VP]),
        "kfbi_last_global_error": (ctypes.c_char_p, []),
        "kfbi_launch_count": (ctypes.c_longlong, []),
        "kfbi_domain_device_bytes": (ctypes.c_longlong, [_VP]),
        "kfbi_state_device_bytes": (ctypes.c_longlong, [_VP]),
        "kfbi_table_cache_bytes": (ctypes.c_longlong, []),
        "kfbi_profile_enable": (None, [ctypes.c_int]),
        "kfbi_profile_reset": (None, []),
        "kfbi_profile_read": (S, [ctypes.c_int, ctypes.POINTER(ctypes.c_longlong),
                                  ctypes.POINTER(ctypes.c_double)]),
        "kfbi_profile_work": (S, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
        "kfbi_profile_bytes": (S, [ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
        "kfbi_check_conversions": (S, [ctypes.c_ulonglong, ctypes.c_longlong,
                                       ctypes.POINTER(ctypes.c_longlong), ctypes.c_void_p]),
        "kfbi_check_wait_timeout": (S, [ctypes.c_double, ctypes.c_void_p]),
        "kfbi_box_solve_noalloc": (S, [ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, ctypes.c_double, _VP, _VP, _VP]),
        "kfbi_batch_create": (S, [ctypes.POINTER(_VP), ctypes.c_int, _VP, ctypes.POINTER(_VP)]),
        "kfbi_batch_destroy": (None, [_VP]),
        "kfbi_batch_step": (S, [_VP, ctypes.POINTER(_VP), ctypes.POINTER(_VP), ctypes.POINTER(_VP),
                                ctypes.POINTER(SolveInfo), _VP]),
        "kfbi_batch_tuning": (S, [_VP, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.c_double)]),
        "kfbi_batch_last_error": (ctypes.c_char_p, [_VP]),
        "kfbi_batch_tuning_count": (ctypes.c_int, [_VP]),
        "kfbi_batch_tuning_get": (S, [_VP, ctypes.c_int, ctypes.POINTER(BatchTuning)]),
        "kfbi_batch_force_candidate": (S, [_VP, ctypes.c_int]),
        "kfbi_plan_create": (S, [ctypes.POINTER(DomainDesc), ctypes.POINTER(_VP)]),
        "kfbi_plan_destroy": (None, [_VP]),
        "kfbi_plan_size": (ctypes.c_longlong, [_VP, ctypes.c_int]),
        "kfbi_plan_export": (S, [_VP, ctypes.c_int, _VP]),
        "kfbi_plan_device_bytes": (ctypes.c_longlong, [_VP, ctypes.c_int]),
        "kfbi_server_create": (S, [ctypes.POINTER(ServerDesc), _VP, ctypes.POINTER(_VP)]),
        "kfbi_server_destroy": (None, [_VP]),
        "kfbi_server_submit": (S, [_VP, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_int)]),
        "kfbi_server_tick": (S, [_VP, ctypes.c_double, ctypes.POINTER(ctypes.c_int)]),
        "kfbi_server_run": (S, [_VP, ctypes.c_double]),
        "kfbi_server_request_info": (S, [_VP, ctypes.c_int, ctypes.POINTER(RequestInfo)]),
        "kfbi_server_get_stats": (S, [_VP, ctypes.POINTER(ServerStats)]),
        "kfbi_server_last_error": (ctypes.c_char_p, [_VP]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def exported_symbols():
    """Names of the entry points the binding declares (all must resolve)."""
    lib()
    return [n for n in dir(_lib) if n.startswith("kfbi_")]


# ----------------------------------------------------------------------------
# descriptors
# ----------------------------------------------------------------------------


def make_desc(d, precision=KFBI_FP64, restart=50, tol=1e-10, maxit=500, solver=None, gamma=0.5):
    """kfbi_domain_desc from a workload dict (see ``workloads.domain_desc``)."""
    c = d["curve"]
    p = (ctypes.c_double * 6)()
    if c["kind"] == "polar":
        kind = KFBI_CURVE_POLAR
        vals = [c["r0"], c["eps"], c["k"], c.get("phase", 0.0)]
    elif c["kind"] == "ellipse":
        kind = KFBI_CURVE_ELLIPSE
        vals = [c["a"], c["b"], c["alpha"]]
    else:
        raise ValueError("unknown curve kind")
    for q, v in enumerate(vals):
        p[q] = float(v)
    return DomainDesc(int(d["M"]), float(d["lo"]), float(d["hi"]), int(d["nb"]), kind,
                      float(c["cx"]), float(c["cy"]), p, int(precision), int(restart),
                      float(tol), int(maxit), KFBI_GMRES if solver is None else int(solver),
                      float(gamma))


def _ptr(t):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check(status, dom=None):
    if status != KFBI_OK:
        L = lib()
        msg = L.kfbi_last_error(dom) if dom else L.kfbi_last_global_error()
        raise KfbiError(status, (msg or b"").decode())


def launch_count():
    return int(lib().kfbi_launch_count())


PROF_DST, PROF_CORRECT, PROF_EXTRACT, PROF_KRYLOV, PROF_GRID, PROF_SPARSE = 0, 1, 2, 3, 4, 5
PROF_NAMES = {0: "dst", 1: "correct", 2: "extract", 3: "krylov", 4: "grid", 5: "sparse"}


def kfbi_profile_enable(classes=True):
    """Enable event timing for kernel classes: True = all, False = none, or
    an iterable of class ids (PROF_*)."""
    if classes is True:
        mask = (1 << len(PROF_NAMES)) - 1
    elif classes is False or classes is None:
        mask = 0
    else:
        mask = 0
        for c in classes:
            mask |= 1 << int(c)
    lib().kfbi_profile_enable(mask)


def kfbi_profile_reset():
    lib().kfbi_profile_reset()


def kfbi_profile_read(cls):
    """(launches, total_ms) of a kernel class since the last reset."""
    n = ctypes.c_longlong()
    ms = ctypes.c_double()
    _check(lib().kfbi_profile_read(int(cls), ctypes.byref(n), ctypes.byref(ms)))
    return int(n.value), float(ms.value)


def kfbi_profile_work(cls):
    """Floating-point operations issued by the recorded launches of a class."""
    w = ctypes.c_double()
    _check(lib().kfbi_profile_work(int(cls), ctypes.byref(w)))
    return float(w.value)


def kfbi_profile_bytes(cls):
    """Algorithmic bytes moved by the recorded launches of a class."""
    w = ctypes.c_double()
    _check(lib().kfbi_profile_bytes(int(cls), ctypes.byref(w)))
    return float(w.value)


def kfbi_check_conversions(seed, n, stream=None):
    """Bit mismatches of the integer-pipe FP32/FP64 conversions against the
    hardware ones over n seeded patterns (0 expected)."""
    m = ctypes.c_longlong()
    _check(lib().kfbi_check_conversions(int(seed), int(n), ctypes.byref(m), _stream(stream)))
    return int(m.value)


def kfbi_check_wait_timeout(seconds, stream=None):
    """Status of the bounded-wait self-check (KFBI_ERR_TIMEOUT expected)."""
    return int(lib().kfbi_check_wait_timeout(float(seconds), _stream(stream)))


# ----------------------------------------------------------------------------
# C-ABI entry points with the same names
# ----------------------------------------------------------------------------


def kfbi_create_domain(desc, stream=None):
    h = ctypes.c_void_p()
    _check(lib().kfbi_create_domain(ctypes.byref(desc), _stream(stream), ctypes.byref(h)))
    return h


def kfbi_destroy_domain(h):
    lib().kfbi_destroy_domain(h)


def kfbi_apply_operator(h, kappa, phi, f, out, stream=None):
    k = complex(kappa)
    _check(lib().kfbi_apply_operator(h, k.real, k.imag, _ptr(phi), _ptr(f), _ptr(out),
                                     _stream(stream)), h)


def kfbi_interface_solve(h, kappa, phi, f, u_grid, u_plus=None, stream=None):
    k = complex(kappa)
    _check(lib().kfbi_interface_solve(h, k.real, k.imag, _ptr(phi), _ptr(f), _ptr(u_grid),
                                      _ptr(u_plus), _stream(stream)), h)


def kfbi_solve_density(h, kappa, b, phi, stream=None):
    k = complex(kappa)
    info = SolveInfo()
    _check(lib().kfbi_solve_density(h, k.real, k.imag, _ptr(b), _ptr(phi), ctypes.byref(info),
                                    _stream(stream)), h)
    return info.as_dict()


def fft_supported(M):
    """Whether KFBI_MIXED_FFT32 has a transform for grid size M (M = 32 N1,
    N1 in {2, 4, 6, 8, 12, 16, 24, 32, 48, 64})."""
    M = int(M)
    return M % 32 == 0 and M // 32 in (2, 4, 6, 8, 12, 16, 24, 32, 48, 64)


def kfbi_box_solve_noalloc(M, box_lo, box_hi, kappa, rhs, u, stream=None):
    """Box solve with no device allocation (static scratch, M - 1 <= 256).
    rhs and u: contiguous CUDA tensors of (M - 1)^2 values, complex128 when
    kappa has an imaginary part and float64 otherwise."""
    import torch
    k = complex(kappa)
    want = torch.complex128 if k.imag != 0.0 else torch.float64
    n = (int(M) - 1) ** 2 if int(M) >= 2 else 0
    for name, t in (("rhs", rhs), ("u", u)):
        if t is None or not t.is_cuda or not t.is_contiguous():
            raise KfbiError(KFBI_ERR_ARG, "%s must be a contiguous CUDA tensor" % name)
        if t.dtype != want:
            raise KfbiError(KFBI_ERR_ARG, "%s must be %s for kappa = %r" % (name, want, kappa))
        if t.numel() != n:
            raise KfbiError(KFBI_ERR_ARG, "%s must hold (M - 1)^2 = %d values, not %d"
                            % (name, n, t.numel()))
    _check(lib().kfbi_box_solve_noalloc(int(M), float(box_lo), float(box_hi), k.real, k.imag,
                                        _ptr(rhs), _ptr(u), _stream(stream)))


class Domain:
    """Owning wrapper of a kfbi_domain."""

    def __init__(self, desc_dict, precision=KFBI_FP64, restart=50, tol=1e-10, maxit=500,
                 stream=None, solver=None, gamma=0.5):
        self.d = dict(desc_dict)
        self.M, self.nb = int(desc_dict["M"]), int(desc_dict["nb"])
        self.n1 = self.M - 1
        self.precision = precision
        self.solver = KFBI_GMRES if solver is None else int(solver)
        self.h = kfbi_create_domain(make_desc(desc_dict, precision, restart, tol, maxit,
                                              self.solver, gamma), stream)

    def close(self):
        if self.h:
            kfbi_destroy_domain(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def device_bytes(self):
        return int(lib().kfbi_domain_device_bytes(self.h))

    def apply_operator(self, kappa, phi, f=None, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty_like(phi)
        kfbi_apply_operator(self.h, kappa, phi, f, out, stream)
        return out

    def interface_solve(self, kappa, phi, f=None, stream=None):
        import torch
        dt = phi.dtype
        U = torch.empty(self.n1 * self.n1, dtype=dt, device=phi.device)
        up = torch.empty_like(phi)
        kfbi_interface_solve(self.h, kappa, phi, f, U, up, stream)
        return up, U.view(self.n1, self.n1)

    def solve_density(self, kappa, b, phi, stream=None):
        return kfbi_solve_density(self.h, kappa, b, phi, stream)

    def apply_neumann(self, kappa, psi, f=None, out=None, stream=None):
        """d_n u+ of the interface solution with Psi = psi (Eq. 3.19's operator
        for f = None)."""
        import torch
        if out is None:
            out = torch.empty_like(psi)
        k = complex(kappa)
        _check(lib().kfbi_apply_neumann(self.h, k.real, k.imag, _ptr(psi), _ptr(f), _ptr(out),
                                        _stream(stream)), self.h)
        return out

    def solve_neumann(self, kappa, gn, psi, f=None, u_grid=None, stream=None):
        """Neumann BVP: psi (initial guess in, density out), optional grid u."""
        k = complex(kappa)
        info = SolveInfo()
        _check(lib().kfbi_solve_neumann(self.h, k.real, k.imag, _ptr(gn), _ptr(f), _ptr(psi),
                                        _ptr(u_grid), ctypes.byref(info), _stream(stream)),
               self.h)
        return info.as_dict()


def table_cache_bytes():
    """Device bytes of the DST-I tables shared per grid."""
    return int(lib().kfbi_table_cache_bytes())


class State:
    """Owning wrapper of a kfbi_state (time-level fields of one equation)."""

    def __init__(self, dom, equation):
        self.dom = dom
        self.eq = equation
        h = ctypes.c_void_p()
        _check(lib().kfbi_state_create(dom.h, int(equation), ctypes.byref(h)), dom.h)
        self.h = h

    def close(self):
        if self.h:
            lib().kfbi_state_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init_heat(self, dt, u0, lap_u0, src_sum=None, stream=None):
        _check(lib().kfbi_state_init_heat(self.h, float(dt), _ptr(u0), _ptr(lap_u0),
                                          _ptr(src_sum), _stream(stream)), self.dom.h)

    def init_wave(self, dt, theta, u0, lap_u0, u1, lap_u1, stream=None):
        _check(lib().kfbi_state_init_wave(self.h, float(dt), float(theta), _ptr(u0), _ptr(lap_u0),
                                          _ptr(u1), _ptr(lap_u1), _stream(stream)), self.dom.h)

    def init_schrodinger(self, dt, u0, lap_u0, stream=None):
        _check(lib().kfbi_state_init_schrodinger(self.h, float(dt), _ptr(u0), _ptr(lap_u0),
                                                 _stream(stream)), self.dom.h)

    def step_heat(self, g_next, src_sum_next=None, stream=None):
        info = SolveInfo()
        _check(lib().kfbi_step_heat(self.dom.h, self.h, _ptr(g_next), _ptr(src_sum_next),
                                    ctypes.byref(info), _stream(stream)), self.dom.h)
        return info.as_dict()

    def step_wave(self, g_next, stream=None):
        info = SolveInfo()
        _check(lib().kfbi_step_wave(self.dom.h, self.h, _ptr(g_next), ctypes.byref(info),
                                    _stream(stream)), self.dom.h)
        return info.as_dict()

    def step_schrodinger(self, v, g_next, w=0.0, stream=None):
        info = SolveInfo()
        _check(lib().kfbi_step_schrodinger(self.dom.h, self.h, _ptr(v), float(w), _ptr(g_next),
                                           ctypes.byref(info), _stream(stream)), self.dom.h)
        return info.as_dict()

    def export(self):
        """Checkpoint: the state's time-level data as bytes."""
        n = int(lib().kfbi_state_blob_bytes(self.h))
        buf = ctypes.create_string_buffer(n)
        _check(lib().kfbi_state_export(self.h, buf, n), self.dom.h)
        return buf.raw

    def import_(self, blob):
        """Resume from bytes written by export()."""
        buf = ctypes.create_string_buffer(bytes(blob), len(blob))
        _check(lib().kfbi_state_import(self.h, buf, len(blob)), self.dom.h)

    def set_w(self, w):
        """Nonlinear coefficient of this Schroedinger state's batched steps."""
        _check(lib().kfbi_state_set_w(self.h, float(w)), self.dom.h)

    def set_neumann(self, on=True):
        """Steps take Neumann data d_n u = g (float64 domains)."""
        _check(lib().kfbi_state_set_neumann(self.h, 1 if on else 0), self.dom.h)

    def get_u(self, out=None, stream=None):
        import torch
        n1 = self.dom.n1
        if out is None:
            dt = torch.complex128 if self.eq == KFBI_SCHRODINGER else torch.float64
            out = torch.empty(n1 * n1, dtype=dt, device="cuda")
        _check(lib().kfbi_state_get_u(self.h, _ptr(out), _stream(stream)), self.dom.h)
        return out.view(n1, n1)

    def device_bytes(self):
        return int(lib().kfbi_state_device_bytes(self.h))

    def get_phi(self, out=None, stream=None):
        import torch
        if out is None:
            dt = torch.complex128 if self.eq == KFBI_SCHRODINGER else torch.float64
            out = torch.empty(self.dom.nb, dtype=dt, device="cuda")
        _check(lib().kfbi_state_get_phi(self.h, _ptr(out), _stream(stream)), self.dom.h)
        return out


class Batch:
    """Owning wrapper of a kfbi_batch: grouped time steps of many domains."""

    def __init__(self, domains, stream=None):
        L = lib()
        self.domains = list(domains)
        arr = (_VP * len(self.domains))(*[d.h for d in self.domains])
        h = ctypes.c_void_p()
        _check(L.kfbi_batch_create(arr, len(self.domains), _stream(stream), ctypes.byref(h)))
        self.h = h

    def close(self):
        if self.h:
            lib().kfbi_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, states, g_next, src_or_v=None, stream=None):
        """One step of every instance; returns the per-instance solve infos."""
        n = len(self.domains)
        st = (_VP * n)(*[s.h for s in states])
        gs = (_VP * n)(*[_ptr(g) for g in g_next])
        sv = None
        if src_or_v is not None:
            sv = (_VP * n)(*[(_ptr(x) if x is not None else None) for x in src_or_v])
        infos = (SolveInfo * n)()
        status = lib().kfbi_batch_step(self.h, st, gs, sv, infos, _stream(stream))
        if status != KFBI_OK:
            msg = lib().kfbi_batch_last_error(self.h) or b""
            raise KfbiError(status, msg.decode())
        return [infos[i].as_dict() for i in range(n)]

    def tuning(self):
        """The autotuner's records: one per FFT grid size and one for the TF32
        instances (candidates, their measured microseconds, the kept one)."""
        L = lib()
        out = []
        for i in range(L.kfbi_batch_tuning_count(self.h)):
            t = BatchTuning()
            _check(L.kfbi_batch_tuning_get(self.h, i, ctypes.byref(t)))
            out.append(t.as_dict())
        return out

    def force_candidate(self, candidate):
        """Use candidate (modulo each group's count) everywhere from the next
        step on, without timing; -1 restores the autotuner."""
        _check(lib().kfbi_batch_force_candidate(self.h, int(candidate)))


class Server:
    """Owning wrapper of a kfbi_server (continuous batching of requests).

    Request data are host numpy arrays; the wrapper keeps them alive until
    the request is done and returns the final field from ``result``."""

    def __init__(self, max_resident=64, hbm_budget_bytes=0, hbm_reserve_bytes=4 << 30,
                 restart=50, plan_threads=4, lanes=1, stream=None):
        d = ServerDesc(int(max_resident), int(hbm_budget_bytes), int(hbm_reserve_bytes),
                       int(restart), int(plan_threads), int(lanes))
        h = ctypes.c_void_p()
        _check(lib().kfbi_server_create(ctypes.byref(d), _stream(stream), ctypes.byref(h)))
        self.h = h
        self.restart = int(restart)
        self._keep = {}
        self._out = {}

    def close(self):
        if self.h:
            lib().kfbi_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _raise(self, status):
        msg = lib().kfbi_server_last_error(self.h) or b""
        raise KfbiError(status, msg.decode())

    def submit(self, desc_dict, equation, steps, dt, arrival, u0, lap_u0, g, theta=0.25, u1=None,
               lap_u1=None, src_init=None, src_profile=None, src_coef=None, potential=None,
               tol=1e-10, maxit=2000, precision=KFBI_MIXED_TF32):
        """Queue a request (grids (M-1, M-1); g (steps, nb)); returns its id.
        precision: KFBI_MIXED_TF32 or KFBI_MIXED_FFT32 (sizes with an FFT pass)."""
        cplx = equation == KFBI_SCHRODINGER
        gt = np.complex128 if cplx else np.float64

        def arr(a, dt_=np.float64):
            return None if a is None else np.ascontiguousarray(a, dtype=dt_)

        keep = {"u0": arr(u0, gt), "lap_u0": arr(lap_u0, gt), "u1": arr(u1), "lap_u1": arr(lap_u1),
                "g": arr(g, gt), "src_init": arr(src_init), "src_profile": arr(src_profile),
                "src_coef": arr(src_coef), "potential": arr(potential)}
        n1 = int(desc_dict["M"]) - 1
        out = np.empty((n1, n1), dtype=gt)
        if keep["g"].shape != (int(steps), int(desc_dict["nb"])):
            raise ValueError("g must have shape (steps, nb)")

        def p(a):
            return None if a is None else ctypes.c_void_p(a.ctypes.data)

        r = Request(make_desc(desc_dict, int(precision), self.restart, tol, maxit), int(equation),
                    int(steps), float(dt), float(theta), float(arrival), p(keep["u0"]),
                    p(keep["lap_u0"]), p(keep["u1"]), p(keep["lap_u1"]), p(keep["g"]),
                    p(keep["src_init"]), p(keep["src_profile"]), p(keep["src_coef"]),
                    p(keep["potential"]), ctypes.c_void_p(out.ctypes.data))
        i = ctypes.c_int()
        status = lib().kfbi_server_submit(self.h, ctypes.byref(r), ctypes.byref(i))
        if status != KFBI_OK:
            self._raise(status)
        self._keep[i.value] = keep
        self._out[i.value] = out
        return int(i.value)

    def tick(self, now=-1.0):
        """One tick at server time now (< 0: wall clock); returns how many stepped."""
        n = ctypes.c_int()
        status = lib().kfbi_server_tick(self.h, float(now), ctypes.byref(n))
        if status != KFBI_OK:
            self._raise(status)
        return int(n.value)

    def run(self, time_limit=0.0):
        status = lib().kfbi_server_run(self.h, float(time_limit))
        if status != KFBI_OK:
            self._raise(status)

    def info(self, i):
        r = RequestInfo()
        _check(lib().kfbi_server_request_info(self.h, int(i), ctypes.byref(r)))
        d = {f: getattr(r, f) for f, _ in RequestInfo._fields_}
        if d["state"] in (REQ_RESIDENT, REQ_DONE, REQ_FAILED):
            k = self._keep.get(int(i))
            if k is not None and d["state"] != REQ_RESIDENT:
                self._keep.pop(int(i), None)
        return d

    def result(self, i):
        """Final field of a completed request (None while it is not done)."""
        if self.info(i)["state"] != REQ_DONE:
            return None
        return self._out[int(i)]

    def stats(self):
        st = ServerStats()
        _check(lib().kfbi_server_get_stats(self.h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}


# ----------------------------------------------------------------------------
# host-only plan (no GPU needed)
# ----------------------------------------------------------------------------


class Plan:
    """The geometry and coefficient tables kfbi_create_domain would upload."""

    def __init__(self, desc_dict, precision=KFBI_FP64, restart=50):
        L = lib()
        h = ctypes.c_void_p()
        _check(L.kfbi_plan_create(ctypes.byref(make_desc(desc_dict, precision, restart)),
                                  ctypes.byref(h)))
        self.h = h
        self.n_edges = int(L.kfbi_plan_size(h, 0))
        self.n_irregular = int(L.kfbi_plan_size(h, 7))
        self.n_arms = int(L.kfbi_plan_size(h, 9))

    def field(self, name):
        L = lib()
        fid, dt = PLAN_FIELDS[name]
        n = int(L.kfbi_plan_size(self.h, fid))
        a = np.zeros(max(n, 1), dtype=dt)
        _check(L.kfbi_plan_export(self.h, fid, a.ctypes.data_as(ctypes.c_void_p)))
        return a[:n]

    def device_bytes(self, equation):
        """Exact device bytes of a domain from this plan plus one state."""
        return int(lib().kfbi_plan_device_bytes(self.h, int(equation)))

    def close(self):
        if self.h:
            lib().kfbi_plan_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
