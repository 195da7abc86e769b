"""ctypes binding of the C ABI declared in include/rve.h.

Argument marshalling only: every function below forwards to the entry point
of the same name in librve.so.  Field arguments of the operator-level calls
are CUDA float64 tensors (contiguous, component-major); the library never
falls back to a CPU path and raises ``RVEError`` when it is not built or a
call fails.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "librve.so")

RVE_OK = 0
RVE_ERR_ARG = -1
RVE_ERR_STATE = -2
RVE_ERR_CUDA = -3
RVE_ERR_OOM = -4
RVE_ERR_NOT_CONVERGED = -5
RVE_ERR_NUMERIC = -6
RVE_ERR_TIMEOUT = -7
RVE_ERR_LOAD_PATH_END = -8
RVE_FP64 = 0
RVE_MIXED = 1

FIELD_STRAIN, FIELD_STRESS, FIELD_DAMAGE, FIELD_ABAR, FIELD_EP, FIELD_PLASTIC = range(6)


class RVEError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s failed: %s (%d)" % (where, rve_status_string(status), status))


class PhaseParams(ctypes.Structure):
    _fields_ = [("E", ctypes.c_double), ("nu", ctypes.c_double), ("sigma_y", ctypes.c_double),
                ("H", ctypes.c_double), ("damage_law", ctypes.c_int), ("nonlocal_var", ctypes.c_int),
                ("eps_C", ctypes.c_double), ("eps_R", ctypes.c_double), ("D_max", ctypes.c_double),
                ("hardening", ctypes.c_int), ("reserved", ctypes.c_int), ("N", ctypes.c_double),
                ("q1", ctypes.c_double), ("q2", ctypes.c_double), ("q3", ctypes.c_double),
                ("f_C", ctypes.c_double), ("f_F", ctypes.c_double), ("f_N", ctypes.c_double),
                ("eps_N", ctypes.c_double), ("s_N", ctypes.c_double), ("f_0", ctypes.c_double),
                ("fstar_max", ctypes.c_double)]

# GTN parameters of Section 4.1 (used when a phase dict leaves them out)
GTN_DEFAULTS = dict(q1=1.5, q2=1.0, q3=2.25, f_C=0.15, f_F=0.25, f_N=0.04, eps_N=0.3, s_N=0.1, f0=0.0,
                    fstar_max=0.6)


class SolverOptions(ctypes.Structure):
    _fields_ = [("tol_stag", ctypes.c_double), ("tol_newton", ctypes.c_double),
                ("cg_rtol", ctypes.c_double), ("pcg_rtol", ctypes.c_double),
                ("max_stag", ctypes.c_int), ("max_newton", ctypes.c_int), ("max_cg", ctypes.c_int),
                ("max_pcg", ctypes.c_int), ("min_stag", ctypes.c_int), ("check_every", ctypes.c_int)]


class AdjointInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("increments", ctypes.c_int), ("recomputed", ctypes.c_int),
                ("checkpoints", ctypes.c_int), ("transposed_staggered_iters", ctypes.c_int),
                ("max_transposed_staggered_iters", ctypes.c_int), ("cg_iters", ctypes.c_longlong),
                ("pcg_iters", ctypes.c_longlong)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class StepInfo(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("increment", ctypes.c_int),
                ("staggered_iters", ctypes.c_int), ("newton_iters", ctypes.c_int),
                ("cg_iters", ctypes.c_longlong), ("pcg_iters", ctypes.c_longlong),
                ("err", ctypes.c_double), ("voxel_iterations", ctypes.c_double),
                ("sigma", ctypes.c_double * 6), ("eps", ctypes.c_double * 6),
                ("D_mean", ctypes.c_double), ("D_max", ctypes.c_double),
                ("fail_stage", ctypes.c_int), ("reserved", ctypes.c_int)]

    def as_dict(self):
        d = {k: getattr(self, k) for k, _ in self._fields_}
        d["sigma"] = np.array(self.sigma[:])
        d["eps"] = np.array(self.eps[:])
        return d


_P = ctypes.c_void_p
_D = ctypes.c_double
_I = ctypes.c_int
_SIGNATURES = {
    "rve_default_options": (_I, [_I, ctypes.POINTER(SolverOptions)]),
    "rve_create": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(_I), ctypes.POINTER(_D), _I, _I, _P]),
    "rve_free": (None, [_P]),
    "rve_set_options": (_I, [_P, ctypes.POINTER(SolverOptions)]),
    "rve_set_phases": (_I, [_P, _P, _I, ctypes.POINTER(PhaseParams), ctypes.POINTER(_D)]),
    "rve_set_load_path": (_I, [_P, _I, ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(_D)]),
    "rve_step_increment": (_I, [_P, ctypes.POINTER(StepInfo)]),
    "rve_step_increment_adaptive": (_I, [_P, _I, ctypes.POINTER(StepInfo)]),
    "rve_homogenized_stress": (_I, [_P, ctypes.POINTER(_D)]),
    "rve_homogenized_strain": (_I, [_P, ctypes.POINTER(_D)]),
    "rve_get_field": (_I, [_P, _I, _P, ctypes.c_size_t]),
    "rve_get_sizes": (_I, [_P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "rve_status_string": (ctypes.c_char_p, [_I]),
    "rve_op_return_map": (_I, [_P] * 10),
    "rve_op_return_map_ex": (_I, [_P] * 13),
    "rve_op_tangent_apply": (_I, [_P, _P, _P]),
    "rve_op_apply_gamma": (_I, [_P, _P, _P]),
    "rve_op_matvec": (_I, [_P, _P, _P]),
    "rve_test_tile_wait": (_I, [_P, _D, _I]),
    "rve_op_cg": (_I, [_P, _P, _P, _D, _I, ctypes.POINTER(_I)]),
    "rve_op_helmholtz_apply": (_I, [_P, _I, _P, _P]),
    "rve_op_helmholtz_solve": (_I, [_P, _I, _P, _P, _D, _I, ctypes.POINTER(_I)]),
    "rve_op_apply_gamma_noalloc": (_I, [_I, ctypes.POINTER(_I), ctypes.POINTER(_D),
                                        ctypes.POINTER(ctypes.c_uint8), _P, _P, _P]),
    "rve_state_bytes": (ctypes.c_longlong, [_P]),
    "rve_save_state": (_I, [_P, _P, ctypes.c_longlong]),
    "rve_load_state": (_I, [_P, _P, ctypes.c_longlong]),
    "rve_set_stiffness_field": (_I, [_P, _P]),
    "rve_adjoint_forward": (_I, [_P, _I, ctypes.POINTER(_D)]),
    "rve_adjoint_backward": (_I, [_P, _D, _P, _P, _P, ctypes.POINTER(AdjointInfo)]),
    "rve_set_graphs": (_I, [_P, _I]),
    "rve_set_gamma_tile": (_I, [_P, _I]),
    "rve_get_gamma_tile": (_I, [_P, ctypes.POINTER(_I)]),
    "rve_autotune": (_I, [_P, _I, ctypes.POINTER(_D), ctypes.POINTER(_I), ctypes.POINTER(_I)]),
    "rve_batch_create": (_I, [ctypes.POINTER(_P), _I, ctypes.POINTER(_P), _I]),
    "rve_batch_step": (_I, [_P, ctypes.POINTER(StepInfo)]),
    "rve_batch_size": (_I, [_P]),
    "rve_batch_free": (None, [_P]),
    "rve_profile": (_I, [_P, _I]),
    "rve_profile_read": (_I, [_P, _I, ctypes.POINTER(_D), ctypes.POINTER(ctypes.c_longlong),
                              ctypes.POINTER(_D)]),
    "rve_profile_reset": (_I, [_P]),
    "rve_profile_class_name": (ctypes.c_char_p, [_I]),
}

_lib = None


def lib():
    """Load librve.so (built in-tree by ``__graft_entry__.build()``)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("librve.so is not built (expected at %s); run __graft_entry__.build()"
                               % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status, where):
    if status != RVE_OK:
        raise RVEError(status, where)
    return status


def _ptr(t):
    """Device pointer of a contiguous CUDA float64/uint8 tensor (or None)."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        if not t.is_cuda:
            raise ValueError("operator-level calls take CUDA tensors")
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(t.data_ptr())
    if isinstance(t, int):
        return ctypes.c_void_p(t)
    raise TypeError("expected a CUDA tensor or a device address")


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


# ----------------------------------------------------------------- handle
def rve_status_string(status):
    return lib().rve_status_string(int(status)).decode()


def rve_default_options(precision=RVE_FP64):
    o = SolverOptions()
    _check(lib().rve_default_options(int(precision), ctypes.byref(o)), "rve_default_options")
    return o


def rve_create(dim, n, L, precision=RVE_FP64, n_nonlocal=1, stream=None):
    n3 = (ctypes.c_int * 3)(*(list(n) + [1] * (3 - len(n))))
    L3 = (ctypes.c_double * 3)(*(list(map(float, L)) + [1.0] * (3 - len(L))))
    h = ctypes.c_void_p()
    _check(lib().rve_create(ctypes.byref(h), int(dim), n3, L3, int(precision), int(n_nonlocal),
                            _stream_handle(stream)), "rve_create")
    return h


def rve_free(h):
    if h:
        lib().rve_free(h)


def rve_set_options(h, opt):
    _check(lib().rve_set_options(h, ctypes.byref(opt)), "rve_set_options")


def phase_params_array(params):
    arr = (PhaseParams * len(params))()
    for i, p in enumerate(params):
        d = dict(GTN_DEFAULTS, **{k: v for k, v in p.items() if k in GTN_DEFAULTS})
        arr[i] = PhaseParams(p["E"], p["nu"], p.get("sigma_y", 0.0), p.get("H", 0.0),
                             int(p.get("law", 0)), int(p.get("var", -1)), p.get("eps_C", 0.0),
                             p.get("eps_R", 1.0), p.get("D_max", 0.0), int(p.get("hard", 0)), 0,
                             p.get("N", 0.1), d["q1"], d["q2"], d["q3"], d["f_C"], d["f_F"], d["f_N"],
                             d["eps_N"], d["s_N"], d["f0"], d["fstar_max"])
    return arr


def rve_set_phases(h, phase, params, ell):
    """phase: numpy uint8 array (host) or CUDA uint8 tensor; params: list of
    dicts (E, nu, sigma_y, H, law, var, eps_C, eps_R, D_max and optionally
    hard, N and the GTN parameters q1, q2, q3, f_C, f_F, f_N, eps_N, s_N, f0,
    fstar_max); ell: [J][n_phases]."""
    if hasattr(phase, "data_ptr"):
        pp = _ptr(phase)
        keep = phase
    else:
        keep = np.ascontiguousarray(phase, dtype=np.uint8)
        pp = ctypes.c_void_p(keep.ctypes.data)
    arr = phase_params_array(params)
    ell = np.ascontiguousarray(ell, dtype=np.float64).reshape(-1)
    ep = ell.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if ell.size else None
    _check(lib().rve_set_phases(h, pp, len(params), arr, ep), "rve_set_phases")
    del keep


def rve_set_load_path(h, strain_ctrl, target):
    c = (ctypes.c_uint8 * 6)(*[int(x) for x in strain_ctrl])
    t = np.ascontiguousarray(target, dtype=np.float64).reshape(-1, 6)
    _check(lib().rve_set_load_path(h, t.shape[0], c, t.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
           "rve_set_load_path")


def rve_step_increment(h, raise_on_error=True):
    info = StepInfo()
    s = lib().rve_step_increment(h, ctypes.byref(info))
    if raise_on_error:
        _check(s, "rve_step_increment")
    d = info.as_dict()
    d["status"] = s
    return d


def rve_step_increment_adaptive(h, max_cuts=7, raise_on_error=True):
    """Next increment with cut-back; the result's "substeps" is the number of
    converged sub-steps (info.reserved)."""
    info = StepInfo()
    s = lib().rve_step_increment_adaptive(h, int(max_cuts), ctypes.byref(info))
    if raise_on_error:
        _check(s, "rve_step_increment_adaptive")
    d = info.as_dict()
    d["status"] = s
    d["substeps"] = d.pop("reserved")
    return d


def rve_homogenized_stress(h):
    out = (ctypes.c_double * 6)()
    _check(lib().rve_homogenized_stress(h, out), "rve_homogenized_stress")
    return np.array(out[:])


def rve_homogenized_strain(h):
    out = (ctypes.c_double * 6)()
    _check(lib().rve_homogenized_strain(h, out), "rve_homogenized_strain")
    return np.array(out[:])


def rve_get_sizes(h):
    nv = ctypes.c_longlong()
    nc = ctypes.c_int()
    J = ctypes.c_int()
    _check(lib().rve_get_sizes(h, ctypes.byref(nv), ctypes.byref(nc), ctypes.byref(J)), "rve_get_sizes")
    return nv.value, nc.value, J.value


def rve_get_field(h, which, dst):
    """dst: a CUDA float64 tensor, or a host float64 buffer (numpy array or
    CPU tensor)."""
    if hasattr(dst, "data_ptr") and dst.is_cuda:
        _check(lib().rve_get_field(h, int(which), _ptr(dst), dst.numel()), "rve_get_field")
        return dst
    if str(getattr(dst, "dtype", "")) not in ("float64", "torch.float64"):
        raise ValueError("rve_get_field writes float64")
    addr, nbytes = _host_buffer(dst)
    _check(lib().rve_get_field(h, int(which), ctypes.c_void_p(addr), nbytes // 8), "rve_get_field")
    return dst


# ----------------------------------------------------------- operator level
def rve_op_return_map(h, eps, epsp_n, ep_n, abar, sigma, epsp, ep, D, alpha):
    _check(lib().rve_op_return_map(h, _ptr(eps), _ptr(epsp_n), _ptr(ep_n), _ptr(abar), _ptr(sigma),
                                   _ptr(epsp), _ptr(ep), _ptr(D), _ptr(alpha)), "rve_op_return_map")


def rve_op_return_map_ex(h, eps, epsp_n, ep_n, abar, abar_n, f_n, sigma, epsp, ep, D, alpha, f):
    """rve_op_return_map with the GTN history given (abar_n, f_n) and the new
    porosity returned (f); any of abar_n, f_n, f may be None."""
    def opt(t):
        return None if t is None else _ptr(t)
    _check(lib().rve_op_return_map_ex(h, _ptr(eps), _ptr(epsp_n), _ptr(ep_n), opt(abar), opt(abar_n), opt(f_n),
                                      _ptr(sigma), _ptr(epsp), _ptr(ep), _ptr(D), opt(alpha), opt(f)),
           "rve_op_return_map_ex")


def rve_op_tangent_apply(h, p, tau):
    _check(lib().rve_op_tangent_apply(h, _ptr(p), _ptr(tau)), "rve_op_tangent_apply")


def rve_op_apply_gamma(h, tau, out):
    _check(lib().rve_op_apply_gamma(h, _ptr(tau), _ptr(out)), "rve_op_apply_gamma")


def rve_test_tile_wait(h, wait_s=2.0, extra_tx_bytes=0):
    """Test hook of the tile-wait timeout path (see rve.h)."""
    _check(lib().rve_test_tile_wait(h, float(wait_s), int(extra_tx_bytes)), "rve_test_tile_wait")


def rve_op_matvec(h, p, Ap):
    _check(lib().rve_op_matvec(h, _ptr(p), _ptr(Ap)), "rve_op_matvec")


def rve_op_cg(h, b, x, rtol, maxit, allow_budget=False):
    """CG iterations taken; with allow_budget, running out of maxit is not an
    error (a fixed number of iterations, e.g. for timing)."""
    it = ctypes.c_int()
    s = lib().rve_op_cg(h, _ptr(b), _ptr(x), float(rtol), int(maxit), ctypes.byref(it))
    if not (allow_budget and s == RVE_ERR_NOT_CONVERGED):
        _check(s, "rve_op_cg")
    return it.value


def rve_op_helmholtz_apply(h, j, a, out):
    _check(lib().rve_op_helmholtz_apply(h, int(j), _ptr(a), _ptr(out)), "rve_op_helmholtz_apply")


def rve_op_helmholtz_solve(h, j, alpha, abar, rtol, maxit):
    it = ctypes.c_int()
    _check(lib().rve_op_helmholtz_solve(h, int(j), _ptr(alpha), _ptr(abar), float(rtol), int(maxit),
                                        ctypes.byref(it)), "rve_op_helmholtz_solve")
    return it.value


def rve_op_apply_gamma_noalloc(dim, n, L, strain_ctrl, tau, out, stream=None):
    """G*(tau) without a handle and without any device allocation (static
    device scratch inside the library); tau/out are CUDA float64 tensors
    [nc][V]."""
    n3 = (ctypes.c_int * 3)(*(list(n) + [1] * (3 - len(n))))
    L3 = (ctypes.c_double * 3)(*(list(map(float, L)) + [1.0] * (3 - len(L))))
    c = (ctypes.c_uint8 * 6)(*[int(x) for x in strain_ctrl])
    _check(lib().rve_op_apply_gamma_noalloc(int(dim), n3, L3, c, _ptr(tau), _ptr(out),
                                            _stream_handle(stream)), "rve_op_apply_gamma_noalloc")


# ---------------------------------------------------- checkpoint / resume
def rve_state_bytes(h):
    return int(lib().rve_state_bytes(h))


def _host_buffer(buf):
    """(address, bytes) of a writable C-contiguous host buffer: a numpy
    array or a CPU torch tensor (pinned or not)."""
    if hasattr(buf, "data_ptr"):
        if buf.is_cuda or not buf.is_contiguous():
            raise ValueError("expected a contiguous host tensor")
        return buf.data_ptr(), buf.numel() * buf.element_size()
    a = np.asarray(buf)
    if not a.flags.c_contiguous:
        raise ValueError("expected a C-contiguous host array")
    return a.ctypes.data, a.nbytes


def rve_save_state(h, out=None):
    """The converged state (see rve_save_state in rve.h): as bytes, or
    written into the host buffer ``out`` (numpy array or CPU tensor of at
    least rve_state_bytes bytes), which is returned."""
    n = lib().rve_state_bytes(h)
    if out is None:
        buf = ctypes.create_string_buffer(int(n))
        _check(lib().rve_save_state(h, ctypes.cast(buf, ctypes.c_void_p), n), "rve_save_state")
        return buf.raw
    addr, nb = _host_buffer(out)
    _check(lib().rve_save_state(h, ctypes.c_void_p(addr), nb), "rve_save_state")
    return out


def rve_load_state(h, data):
    """Restore a state image: bytes, or a host buffer (numpy array or CPU
    tensor) read in place."""
    if isinstance(data, (bytes, bytearray)):
        buf = ctypes.create_string_buffer(bytes(data), len(data))
        _check(lib().rve_load_state(h, ctypes.cast(buf, ctypes.c_void_p), len(data)), "rve_load_state")
        return
    addr, nb = _host_buffer(data)
    _check(lib().rve_load_state(h, ctypes.c_void_p(addr), nb), "rve_load_state")


# ------------------------------------------------------------- adjoint
def rve_set_stiffness_field(h, s):
    """s: per-voxel Young's modulus factor (host array, x1 fastest) or None."""
    if s is None:
        _check(lib().rve_set_stiffness_field(h, None), "rve_set_stiffness_field")
        return
    a = np.ascontiguousarray(np.asarray(s, dtype=np.float64).reshape(-1))
    _check(lib().rve_set_stiffness_field(h, a.ctypes.data), "rve_set_stiffness_field")


def rve_adjoint_forward(h, checkpoint_every=5):
    J = ctypes.c_double()
    _check(lib().rve_adjoint_forward(h, int(checkpoint_every), ctypes.byref(J)), "rve_adjoint_forward")
    return J.value


def rve_adjoint_backward(h, dJ, n_phases, n_vars, n_voxels):
    """Returns (grad_params [n_phases, 4], grad_ell [n_vars], grad_stiff [V], info)."""
    gp = np.zeros((n_phases, 4))
    ge = np.zeros(max(n_vars, 1))
    gs = np.zeros(n_voxels)
    info = AdjointInfo()
    s = lib().rve_adjoint_backward(h, float(dJ), gp.ctypes.data, ge.ctypes.data, gs.ctypes.data,
                                   ctypes.byref(info))
    _check(s, "rve_adjoint_backward")
    return gp, ge[:n_vars], gs, info.as_dict()


# ------------------------------------------- graphs, autotuning, batches
def rve_set_graphs(h, enable=True):
    _check(lib().rve_set_graphs(h, 1 if enable else 0), "rve_set_graphs")


def rve_set_gamma_tile(h, narrow):
    _check(lib().rve_set_gamma_tile(h, int(narrow)), "rve_set_gamma_tile")


def rve_get_gamma_tile(h):
    v = ctypes.c_int()
    _check(lib().rve_get_gamma_tile(h, ctypes.byref(v)), "rve_get_gamma_tile")
    return v.value


def rve_autotune(h, reps=3):
    """Time candidate FFT schedules of the mechanical matvec and keep the
    fastest; returns (ms per matvec, tile width, radices per axis)."""
    ms = ctypes.c_double()
    tx = ctypes.c_int()
    rad = (ctypes.c_int * 24)()
    _check(lib().rve_autotune(h, int(reps), ctypes.byref(ms), ctypes.byref(tx), rad), "rve_autotune")
    radices = [[v for v in rad[8 * j:8 * j + 8] if v] for j in range(3)]
    return ms.value, tx.value, radices


def rve_batch_create(handles, autotune_reps=3):
    arr = (_P * len(handles))(*handles)
    b = _P()
    _check(lib().rve_batch_create(ctypes.byref(b), len(handles), arr, int(autotune_reps)),
           "rve_batch_create")
    return b.value


def rve_batch_step(b, count, raise_on_error=True):
    infos = (StepInfo * count)()
    s = lib().rve_batch_step(b, infos)
    if raise_on_error:
        _check(s, "rve_batch_step")
    return s, [i.as_dict() for i in infos]


def rve_batch_size(b):
    return lib().rve_batch_size(b)


def rve_batch_free(b):
    lib().rve_batch_free(b)


# -------------------------------------------------------------- profiling
def rve_profile(h, enable=True):
    _check(lib().rve_profile(h, 1 if enable else 0), "rve_profile")


def rve_profile_reset(h):
    _check(lib().rve_profile_reset(h), "rve_profile_reset")


def rve_profile_class_name(k):
    r = lib().rve_profile_class_name(int(k))
    return None if r is None else r.decode()


def rve_profile_read(h):
    """{class name: (total device ms, launches, algorithmic bytes)}"""
    n = 32
    ms = (ctypes.c_double * n)()
    ln = (ctypes.c_longlong * n)()
    by = (ctypes.c_double * n)()
    k = lib().rve_profile_read(h, n, ms, ln, by)
    if k < 0:
        raise RVEError(k, "rve_profile_read")
    return {rve_profile_class_name(i): (ms[i], ln[i], by[i]) for i in range(k)}


# ------------------------------------------------------------ convenience
class RVE:
    """Owning wrapper of a handle built from an ``rve_inputs.RVEConfig``-like
    object (n, L, phase, params, ell, strain_ctrl, target, precision)."""

    def __init__(self, cfg, precision=None, stream=None, options=None):
        prec = cfg.precision if precision is None else precision
        self.cfg = cfg
        self.precision = prec
        J = int(np.asarray(cfg.ell).shape[0])
        self.h = rve_create(len(cfg.n), cfg.n, cfg.L, prec, J, stream)
        try:
            if options is not None:
                rve_set_options(self.h, options)
            rve_set_phases(self.h, cfg.phase, cfg.params, cfg.ell)
            rve_set_load_path(self.h, cfg.strain_ctrl, cfg.target)
        except Exception:
            rve_free(self.h)
            self.h = None
            raise

    def step(self, raise_on_error=True):
        return rve_step_increment(self.h, raise_on_error)

    def step_adaptive(self, max_cuts=7, raise_on_error=True):
        return rve_step_increment_adaptive(self.h, max_cuts, raise_on_error)

    def stress(self):
        return rve_homogenized_stress(self.h)

    def strain(self):
        return rve_homogenized_strain(self.h)

    def close(self):
        if self.h:
            rve_free(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class RVEBatch:
    """Owning wrapper of a batch of RVE configs advanced together (one
    stream, graph-replayed Krylov chunks and one host worker per member)."""

    def __init__(self, cfgs, precision=None, options=None, autotune_reps=3):
        self.members = []
        self.b = None
        try:
            for c in cfgs:
                self.members.append(RVE(c, precision=precision, options=options))
            self.b = rve_batch_create([m.h for m in self.members], autotune_reps)
        except Exception:
            self.close()
            raise

    def step(self, raise_on_error=True):
        s, infos = rve_batch_step(self.b, len(self.members), raise_on_error)
        return infos

    def stresses(self):
        return np.array([m.stress() for m in self.members])

    def close(self):
        if self.b:
            rve_batch_free(self.b)
            self.b = None
        for m in self.members:
            m.close()
        self.members = []

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
