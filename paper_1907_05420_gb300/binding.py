"""ctypes binding of the C ABI in include/kkt_schur.h (argument marshalling only).

Every step of the factor and of the solve runs in the CUDA library
libkkt_schur.so; this module converts numpy arrays / torch tensors into
pointers and returns the status.  There is no CPU fallback: if the library
cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

KKT_FP64, KKT_TF32, KKT_BF16, KKT_F64_EMULATED = 0, 1, 2, 3
PRECISIONS = {"fp64": KKT_FP64, "tf32": KKT_TF32, "bf16": KKT_BF16, "f64emu": KKT_F64_EMULATED}

STATUS = {
    0: "KKT_OK", 1: "KKT_ERR_INVALID", 2: "KKT_ERR_OOM", 3: "KKT_ERR_CUDA",
    4: "KKT_ERR_ZERO_PIVOT", 5: "KKT_ERR_INERTIA", 6: "KKT_ERR_NOT_CONVERGED",
    7: "KKT_ERR_TIMEOUT", 8: "KKT_ERR_STATE", 9: "KKT_ERR_NONFINITE",
}


class KKTError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class kkt_pattern(C.Structure):
    _fields_ = [("N", C.c_int32), ("nA", C.c_int32), ("nP", C.c_int32), ("nC", C.c_int32),
                ("a_rowptr", C.c_void_p), ("a_col", C.c_void_p), ("b_blockptr", C.c_void_p),
                ("b_row", C.c_void_p), ("b_col", C.c_void_p), ("c_kind", C.c_int32),
                ("a_vals_hint", C.c_void_p)]


class kkt_options(C.Structure):
    _fields_ = [("prec", C.c_int), ("refine_tol", C.c_double), ("max_refine", C.c_int32),
                ("pivot_eps", C.c_double), ("use_graphs", C.c_int32),
                ("fp64_fallback", C.c_int32), ("reduced_contraction", C.c_int32),
                ("structured_s", C.c_int32), ("dense_tail", C.c_int32), ("autotune", C.c_int32),
                ("early_solve", C.c_int32), ("time_kernels", C.c_int32), ("tail_ratio", C.c_double),
                ("refine_mode", C.c_int32), ("gmres_restart", C.c_int32),
                ("device_refine", C.c_int32)]


class kkt_info(C.Structure):
    _fields_ = [("n_pos", C.c_int64), ("n_neg", C.c_int64), ("n_zero", C.c_int64),
                ("n_perturbed", C.c_int64), ("refine_steps", C.c_int32),
                ("fell_back_fp64", C.c_int32), ("rel_residual", C.c_double),
                ("ms_analyze", C.c_double), ("ms_factor", C.c_double), ("ms_solve", C.c_double),
                ("nnz_l", C.c_int64), ("panel_doubles", C.c_int64), ("n_supernodes", C.c_int32),
                ("n_levels", C.c_int32), ("k_coupling_rows", C.c_int32), ("w_rows", C.c_int32),
                ("factor_flops", C.c_double), ("device_bytes", C.c_int64),
                ("ms_block_factor", C.c_double), ("ms_schur_assembly", C.c_double),
                ("ms_dense_factor", C.c_double), ("ms_solve_device", C.c_double),
                ("n_launches", C.c_int64), ("dense_tail_cols", C.c_int32), ("tail_augmented", C.c_int32),
                ("tail_ratio", C.c_double), ("autotune_candidates", C.c_int32), ("schur_block", C.c_int32)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class kkt_inertia_options(C.Structure):
    _fields_ = [("delta_w_init", C.c_double), ("delta_w_min", C.c_double), ("delta_w_max", C.c_double),
                ("grow_first", C.c_double), ("grow", C.c_double), ("shrink", C.c_double),
                ("delta_c", C.c_double), ("max_trials", C.c_int32), ("coupling_dual", C.c_int32)]


class kkt_inertia_result(C.Structure):
    _fields_ = [("delta_w", C.c_double), ("delta_c", C.c_double), ("trials", C.c_int32),
                ("reserved", C.c_int32)]


# every symbol the header declares
EXPORTS = ["kkt_default_options", "kkt_analyze", "kkt_factor", "kkt_solve", "kkt_get_info",
           "kkt_destroy", "kkt_status_string", "kkt_last_error", "kkt_measure_fp64_peak",
           "kkt_solve_noalloc", "kkt_batch_factor_solve", "kkt_server_create", "kkt_server_submit",
           "kkt_server_poll", "kkt_server_destroy", "kkt_default_inertia_options", "kkt_factor_inertia",
           "kkt_factor_blocks", "kkt_schur_matrix", "kkt_factor_schur", "kkt_schur_factor_copy", "kkt_accumulate",
           "kkt_solve_front", "kkt_solve_coupling", "kkt_solve_back", "kkt_residual", "kkt_abs_rowsums",
           "kkt_norm_inf", "kkt_kernel_stats", "kkt_slack_create", "kkt_slack_reduce", "kkt_slack_recover",
           "kkt_slack_destroy", "kkt_server_set_cache", "kkt_server_submit_pattern", "kkt_server_cache_info",
           "kkt_schur_blocks", "kkt_probe_pivot_reciprocal"]

KERNEL_FAMILIES = ["k_tc_update_emu", "k_tc_update_wide", "k_tc_update", "k_dense_update", "k_factor_update",
                   "k_dense_diag_t", "k_tc_update_emu_wide", "k_tc_panel_emu"]


class kkt_ipm_state(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in ("x", "z", "s", "y", "la", "le", "lcd", "lb", "lf")]


class kkt_kernel_stat(C.Structure):
    _fields_ = [("launches", C.c_int64), ("ms_total", C.c_double), ("ms_max", C.c_double), ("flops", C.c_double)]

_lib = None


def lib_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libkkt_schur.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing:
        path = _build.build()
    if not os.path.exists(path):
        raise OSError(f"CUDA library not built: {path}")
    L = C.CDLL(path)
    L.kkt_default_options.argtypes = [C.POINTER(kkt_options)]
    L.kkt_default_options.restype = None
    L.kkt_analyze.argtypes = [C.POINTER(kkt_pattern), C.POINTER(kkt_options), C.POINTER(C.c_void_p)]
    L.kkt_analyze.restype = C.c_int
    L.kkt_factor.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]
    L.kkt_factor.restype = C.c_int
    L.kkt_solve.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p]
    L.kkt_solve.restype = C.c_int
    L.kkt_get_info.argtypes = [C.c_void_p, C.POINTER(kkt_info)]
    L.kkt_get_info.restype = C.c_int
    L.kkt_destroy.argtypes = [C.c_void_p]
    L.kkt_destroy.restype = C.c_int
    L.kkt_status_string.argtypes = [C.c_int]
    L.kkt_status_string.restype = C.c_char_p
    L.kkt_last_error.argtypes = []
    L.kkt_last_error.restype = C.c_char_p
    L.kkt_measure_fp64_peak.argtypes = [C.POINTER(C.c_double)]
    L.kkt_measure_fp64_peak.restype = C.c_int
    L.kkt_solve_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    L.kkt_solve_noalloc.restype = C.c_int
    pp = C.POINTER(C.c_void_p)
    L.kkt_batch_factor_solve.argtypes = [pp, C.c_int32, pp, pp, pp, pp, pp, C.c_int32, C.c_int32,
                                         C.POINTER(C.c_int)]
    L.kkt_batch_factor_solve.restype = C.c_int
    L.kkt_server_create.argtypes = [C.c_int32, C.c_int64, C.POINTER(C.c_void_p)]
    L.kkt_server_create.restype = C.c_int
    L.kkt_server_submit.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(C.c_int64)]
    L.kkt_server_submit.restype = C.c_int
    L.kkt_server_poll.argtypes = [C.c_void_p, C.c_int64, C.c_int32, C.POINTER(C.c_int),
                                  C.POINTER(C.c_double)]
    L.kkt_server_poll.restype = C.c_int
    L.kkt_server_destroy.argtypes = [C.c_void_p]
    L.kkt_server_destroy.restype = C.c_int
    L.kkt_default_inertia_options.argtypes = [C.POINTER(kkt_inertia_options)]
    L.kkt_default_inertia_options.restype = None
    L.kkt_factor_inertia.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p,
                                     C.POINTER(kkt_inertia_options), C.POINTER(kkt_inertia_result)]
    L.kkt_factor_inertia.restype = C.c_int
    vp = C.c_void_p
    for name, args in (("kkt_factor_blocks", [vp, vp, vp, vp, C.c_int32, vp]),
                       ("kkt_schur_matrix", [vp, C.POINTER(C.c_void_p), C.POINTER(C.c_int64)]),
                       ("kkt_factor_schur", [vp, vp]),
                       ("kkt_schur_factor_copy", [vp, vp, vp]),
                       ("kkt_schur_blocks", [vp, vp, vp, vp]),
                       ("kkt_probe_pivot_reciprocal", [vp, C.c_int64, vp, vp, vp]),
                       ("kkt_accumulate", [vp, C.c_int64, vp, C.c_int64, C.c_int64, C.c_int64, vp]),
                       ("kkt_solve_front", [vp, vp, vp, vp]),
                       ("kkt_solve_coupling", [vp, vp, vp, vp]),
                       ("kkt_solve_back", [vp, vp, vp, vp]),
                       ("kkt_residual", [vp, vp, vp, vp, vp]),
                       ("kkt_abs_rowsums", [vp, vp, vp]),
                       ("kkt_norm_inf", [vp, vp, C.c_int64, C.POINTER(C.c_double), vp])):
        getattr(L, name).argtypes = args
        getattr(L, name).restype = C.c_int
    L.kkt_kernel_stats.argtypes = [vp, C.c_int32, C.POINTER(kkt_kernel_stat)]
    L.kkt_kernel_stats.restype = C.c_int
    L.kkt_slack_create.argtypes = [vp, C.c_int32, vp, C.POINTER(C.c_void_p)]
    L.kkt_slack_create.restype = C.c_int
    L.kkt_slack_reduce.argtypes = [vp, C.POINTER(kkt_ipm_state), vp, vp, vp, vp, vp, vp]
    L.kkt_slack_reduce.restype = C.c_int
    L.kkt_slack_recover.argtypes = [vp, C.POINTER(kkt_ipm_state), vp, vp, vp, vp, vp]
    L.kkt_slack_recover.restype = C.c_int
    L.kkt_slack_destroy.argtypes = [vp]
    L.kkt_slack_destroy.restype = C.c_int
    L.kkt_server_set_cache.argtypes = [vp, C.POINTER(kkt_options), C.c_int64]
    L.kkt_server_set_cache.restype = C.c_int
    L.kkt_server_submit_pattern.argtypes = [vp, C.c_int64, C.POINTER(kkt_pattern), vp, vp, vp, vp, vp, C.c_int32,
                                            C.POINTER(C.c_int64)]
    L.kkt_server_submit_pattern.restype = C.c_int
    L.kkt_server_cache_info.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64), C.POINTER(C.c_int64)]
    L.kkt_server_cache_info.restype = C.c_int
    _lib = L
    return L


def _check(status, allow=()):
    if status != 0 and status not in allow:
        L = load()
        raise KKTError(status, L.kkt_last_error().decode(errors="replace"))
    return status


def _ptr(a):
    """(pointer, on_device) of a numpy array or torch tensor."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data, 0
    # torch tensor
    if not a.is_contiguous():
        raise ValueError("tensors must be contiguous")
    return a.data_ptr(), 1 if a.is_cuda else 0


def _stream_ptr(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return torch.cuda.current_stream().cuda_stream
        except Exception:  # pragma: no cover
            pass
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def kkt_default_options(prec="fp64", **kw) -> kkt_options:
    opt = kkt_options()
    load().kkt_default_options(C.byref(opt))
    opt.prec = PRECISIONS[prec] if isinstance(prec, str) else int(prec)
    for k, v in kw.items():
        setattr(opt, k, v)
    return opt


def make_pattern(prob, hint=True):
    """(kkt_pattern, the arrays it points to) of `prob`; keep both alive while
    the pattern may be read."""
    keep = {
        "a_rowptr": np.ascontiguousarray(prob.a_rowptr, dtype=np.int32),
        "a_col": np.ascontiguousarray(prob.a_col, dtype=np.int32),
        "b_blockptr": np.ascontiguousarray(prob.b_blockptr, dtype=np.int32),
        "b_row": np.ascontiguousarray(prob.b_row, dtype=np.int32),
        "b_col": np.ascontiguousarray(prob.b_col, dtype=np.int32),
    }
    hint_arr = None
    if hint:
        hint_arr = np.ascontiguousarray(np.asarray(prob.a_vals).reshape(prob.N, -1)[0], dtype=np.float64)
    pat = kkt_pattern(int(prob.N), int(prob.nA), int(prob.nP), int(prob.nC),
                      keep["a_rowptr"].ctypes.data, keep["a_col"].ctypes.data,
                      keep["b_blockptr"].ctypes.data, keep["b_row"].ctypes.data,
                      keep["b_col"].ctypes.data, int(prob.c_kind),
                      hint_arr.ctypes.data if hint_arr is not None else None)
    keep["hint"] = hint_arr
    return pat, keep


def kkt_analyze(prob, opt: kkt_options | None = None, hint=True):
    """Analyze the pattern of `prob` (any object with the KKTProblem fields).

    Returns an opaque handle (int).  Host arrays are read during the call only.
    """
    L = load()
    pat, keep = make_pattern(prob, hint)
    if opt is None:
        opt = kkt_default_options()
    h = C.c_void_p()
    _check(L.kkt_analyze(C.byref(pat), C.byref(opt), C.byref(h)))
    del keep
    return h.value


def kkt_factor(h, a_vals, b_vals, c_vals, stream=None):
    pa, da = _ptr(a_vals)
    pb, db = _ptr(b_vals)
    pc, dc = _ptr(c_vals)
    if len({da, db, dc}) != 1:
        raise ValueError("a_vals, b_vals and c_vals must all be host or all device arrays")
    return _check(load().kkt_factor(h, pa, pb, pc, da, _stream_ptr(stream)))


def kkt_default_inertia_options(**kw) -> kkt_inertia_options:
    opt = kkt_inertia_options()
    load().kkt_default_inertia_options(C.byref(opt))
    for k, v in kw.items():
        setattr(opt, k, v)
    return opt


def kkt_factor_inertia(h, a_vals, b_vals, c_vals, opt: kkt_inertia_options | None = None, stream=None,
                       allow_wrong_inertia=False) -> dict:
    """kkt_factor with inertia correction; returns the shifts of the factor
    the handle holds and the number of factorizations (include/kkt_schur.h)."""
    pa, da = _ptr(a_vals)
    pb, db = _ptr(b_vals)
    pc, dc = _ptr(c_vals)
    if len({da, db, dc}) != 1:
        raise ValueError("a_vals, b_vals and c_vals must all be host or all device arrays")
    res = kkt_inertia_result()
    st = load().kkt_factor_inertia(h, pa, pb, pc, da, _stream_ptr(stream),
                                   C.byref(opt) if opt is not None else None, C.byref(res))
    _check(st, (5,) if allow_wrong_inertia else ())
    return {"status": st, "delta_w": res.delta_w, "delta_c": res.delta_c, "trials": res.trials}


def kkt_solve(h, rhs, x, nrhs=1, stream=None, allow_not_converged=False):
    pr, dr = _ptr(rhs)
    px, dx = _ptr(x)
    if dr != dx:
        raise ValueError("rhs and x must both be host or both device arrays")
    allow = (6,) if allow_not_converged else ()
    return _check(load().kkt_solve(h, pr, px, int(nrhs), dr, _stream_ptr(stream)), allow)


def kkt_get_info(h) -> dict:
    info = kkt_info()
    _check(load().kkt_get_info(h, C.byref(info)))
    return info.as_dict()


def kkt_kernel_stats(h) -> dict:
    """Per-family device times of the handle's last factor (kkt_options.time_kernels)."""
    out = {}
    for f, name in enumerate(KERNEL_FAMILIES):
        st = kkt_kernel_stat()
        _check(load().kkt_kernel_stats(h, f, C.byref(st)))
        out[name] = {"launches": st.launches, "ms_total": st.ms_total, "ms_max": st.ms_max, "flops": st.flops}
    return out


class Slack:
    """Slack elimination around the solve (kkt_slack_*; device tensors)."""

    FIELDS = ("x", "z", "s", "y", "la", "le", "lcd", "lb", "lf")

    def __init__(self, h, ineq_rows):
        rows = np.ascontiguousarray(ineq_rows, dtype=np.int32)
        self.sl = C.c_void_p()
        _check(load().kkt_slack_create(h, int(rows.size), rows.ctypes.data if rows.size else None,
                                       C.byref(self.sl)))

    def _state(self, st):
        """st: a mapping or object with device tensors named as kkt_ipm_state's fields."""
        get = (lambda k: st[k]) if isinstance(st, dict) else (lambda k: getattr(st, k))
        return kkt_ipm_state(*[_dev(get(k)) if get(k) is not None and get(k).numel() else None
                               for k in self.FIELDS])

    def reduce(self, st, a_base, c_base, a_vals, c_vals, rhs, stream=None):
        s = self._state(st)
        return _check(load().kkt_slack_reduce(self.sl, C.byref(s), _dev(a_base), _dev(c_base), _dev(a_vals),
                                              _dev(c_vals), _dev(rhs), _stream_ptr(stream)))

    def recover(self, st, dsol, ds, dz, dy, stream=None):
        s = self._state(st)
        return _check(load().kkt_slack_recover(self.sl, C.byref(s), _dev(dsol), _dev(ds) if ds.numel() else None,
                                               _dev(dz), _dev(dy) if dy.numel() else None, _stream_ptr(stream)))

    def close(self):
        if self.sl:
            load().kkt_slack_destroy(self.sl)
            self.sl = C.c_void_p()


def kkt_solve_noalloc(h, rhs, x, stream=None):
    """One application of the factorization to device arrays, without any
    allocation (see include/kkt_schur.h); returns the status."""
    pr, dr = _ptr(rhs)
    px, dx = _ptr(x)
    if not (dr and dx):
        raise ValueError("kkt_solve_noalloc takes device arrays only")
    return _check(load().kkt_solve_noalloc(h, pr, px, _stream_ptr(stream)))


def kkt_batch_factor_solve(handles, a_vals, b_vals, c_vals, rhs, x, streams=8):
    """Factor and solve independent systems concurrently; returns the per-system statuses."""
    n = len(handles)
    if not all(len(v) == n for v in (a_vals, b_vals, c_vals, rhs, x)):
        raise ValueError("one set of arrays per handle")
    ptrs = [[_ptr(a) for a in v] for v in (a_vals, b_vals, c_vals, rhs, x)]
    dev = {d for v in ptrs for _, d in v}
    if len(dev) > 1:
        raise ValueError("all arrays must be host arrays or all device arrays")
    on_device = dev.pop() if dev else 0
    arr = lambda v: (C.c_void_p * n)(*[p for p, _ in v])  # noqa: E731
    hs = (C.c_void_p * n)(*handles)
    st = (C.c_int * n)()
    rc = load().kkt_batch_factor_solve(hs, n, arr(ptrs[0]), arr(ptrs[1]), arr(ptrs[2]), arr(ptrs[3]),
                                       arr(ptrs[4]), on_device, int(streams), st)
    _check(rc, allow=(6,))
    return list(st)


KKT_ERR_STATE = 8


# ---- the steps of Algorithm 1 one at a time (include/kkt_schur.h) ----
# Arrays are torch tensors on the handle's device (float64, contiguous).

def _dev(t):
    p, d = _ptr(t)
    if t is not None and not d:
        raise ValueError("device arrays only")
    return p


def kkt_factor_blocks(h, a_vals, b_vals, c_vals, stream=None):
    pa, da = _ptr(a_vals)
    pb, db = _ptr(b_vals)
    pc, dc = _ptr(c_vals)
    if len({da, db, dc}) != 1:
        raise ValueError("a_vals, b_vals and c_vals must all be host or all device arrays")
    return _check(load().kkt_factor_blocks(h, pa, pb, pc, da, _stream_ptr(stream)))


def kkt_schur_matrix(h):
    """(device address, leading dimension) of the handle's S buffer."""
    ptr, ld = C.c_void_p(), C.c_int64()
    _check(load().kkt_schur_matrix(h, C.byref(ptr), C.byref(ld)))
    return ptr.value, ld.value


def kkt_factor_schur(h, stream=None):
    return _check(load().kkt_factor_schur(h, _stream_ptr(stream)))


def kkt_schur_factor_copy(h, out, stream=None):
    return _check(load().kkt_schur_factor_copy(h, _dev(out), _stream_ptr(stream)))


def kkt_schur_blocks(h, Sd, So, stream=None):
    """The structured S (structured_s = 2): S_d (N x ns x ns) into Sd and S_o
    ((N-1) x ns x ns) into So, device tensors, each block column-major."""
    return _check(load().kkt_schur_blocks(h, _dev(Sd), _dev(So) if So is not None else None, _stream_ptr(stream)))


def kkt_probe_pivot_reciprocal(d, recip, quotient, stream=None):
    """recip = the factor kernels' pivot reciprocal of d, quotient = 1.0 / d (device tensors)."""
    return _check(load().kkt_probe_pivot_reciprocal(_dev(d), int(d.numel()), _dev(recip), _dev(quotient),
                                                    _stream_ptr(stream)))


def kkt_accumulate(dst_ptr, ld_dst, src, ld_src, rows, cols, stream=None):
    """dst[i + j ld_dst] += src[i + j ld_src]; dst_ptr an address or a tensor."""
    if not isinstance(dst_ptr, int):
        dst_ptr = _dev(dst_ptr)
    return _check(load().kkt_accumulate(dst_ptr, int(ld_dst), _dev(src), int(ld_src), int(rows), int(cols),
                                        _stream_ptr(stream)))


def kkt_solve_front(h, rhs, t, stream=None):
    return _check(load().kkt_solve_front(h, _dev(rhs), _dev(t), _stream_ptr(stream)))


def kkt_solve_coupling(h, t, xg, stream=None):
    return _check(load().kkt_solve_coupling(h, _dev(t), _dev(xg), _stream_ptr(stream)))


def kkt_solve_back(h, xg, x, stream=None):
    return _check(load().kkt_solve_back(h, _dev(xg), _dev(x), _stream_ptr(stream)))


def kkt_residual(h, rhs, x, rho, stream=None):
    return _check(load().kkt_residual(h, _dev(rhs), _dev(x), _dev(rho), _stream_ptr(stream)))


def kkt_abs_rowsums(h, out, stream=None):
    return _check(load().kkt_abs_rowsums(h, _dev(out), _stream_ptr(stream)))


def kkt_norm_inf(h, v, n=None, stream=None):
    out = C.c_double()
    n = v.numel() if n is None else int(n)
    _check(load().kkt_norm_inf(h, _dev(v), n, C.byref(out), _stream_ptr(stream)))
    return out.value


class KKTServer:
    """Continuous-batching request loop (kkt_server_*)."""

    def __init__(self, slots=4, device_budget_bytes=0):
        self.s = C.c_void_p()
        _check(load().kkt_server_create(int(slots), int(device_budget_bytes), C.byref(self.s)))
        self._keep = {}

    def submit(self, h, a_vals, b_vals, c_vals, rhs, x):
        ptrs = [_ptr(v) for v in (a_vals, b_vals, c_vals, rhs, x)]
        dev = {d for _, d in ptrs}
        if len(dev) > 1:
            raise ValueError("all arrays must be host arrays or all device arrays")
        rid = C.c_int64()
        _check(load().kkt_server_submit(self.s, h, *[p for p, _ in ptrs], dev.pop(), C.byref(rid)))
        self._keep[rid.value] = (a_vals, b_vals, c_vals, rhs, x)
        return rid.value

    def set_cache(self, opt: kkt_options | None = None, reserve_bytes=0):
        """Pattern cache with admission by free device memory (kkt_server_set_cache)."""
        _check(load().kkt_server_set_cache(self.s, C.byref(opt) if opt is not None else None, int(reserve_bytes)))

    def submit_pattern(self, key, prob, a_vals, b_vals, c_vals, rhs, x, pattern=None):
        """Queue a solve of cached pattern `key` (prob's pattern; `pattern` may
        pass a (kkt_pattern, arrays) pair from make_pattern to reuse it)."""
        pat, keep = pattern if pattern is not None else make_pattern(prob)
        ptrs = [_ptr(v) for v in (a_vals, b_vals, c_vals, rhs, x)]
        dev = {d for _, d in ptrs}
        if len(dev) > 1:
            raise ValueError("all arrays must be host arrays or all device arrays")
        rid = C.c_int64()
        _check(load().kkt_server_submit_pattern(self.s, int(key), C.byref(pat), *[p for p, _ in ptrs], dev.pop(),
                                                C.byref(rid)))
        self._keep[rid.value] = (pat, keep, a_vals, b_vals, c_vals, rhs, x)
        return rid.value

    def cache_info(self):
        res, an, ev = C.c_int64(), C.c_int64(), C.c_int64()
        _check(load().kkt_server_cache_info(self.s, C.byref(res), C.byref(an), C.byref(ev)))
        return {"resident": res.value, "analyses": an.value, "evictions": ev.value}

    def wait(self, rid):
        st, lat = C.c_int(), C.c_double()
        _check(load().kkt_server_poll(self.s, int(rid), 1, C.byref(st), C.byref(lat)))
        self._keep.pop(rid, None)
        return st.value, lat.value

    def poll(self, rid):
        """(status, latency_ms) if request rid has finished, else None."""
        st, lat = C.c_int(), C.c_double()
        r = load().kkt_server_poll(self.s, int(rid), 0, C.byref(st), C.byref(lat))
        if r == KKT_ERR_STATE:
            return None
        _check(r)
        self._keep.pop(rid, None)
        return st.value, lat.value

    def close(self):
        if self.s:
            _check(load().kkt_server_destroy(self.s))
            self.s = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass


def kkt_measure_fp64_peak() -> float:
    """Measured FP64 FMA throughput of the current device, GFLOP/s."""
    v = C.c_double()
    _check(load().kkt_measure_fp64_peak(C.byref(v)))
    return v.value


def kkt_destroy(h):
    if h:
        _check(load().kkt_destroy(h))


class KKTSolver:
    """Convenience owner of one handle: analyze once, then factor/solve."""

    def __init__(self, prob, prec="fp64", **opts):
        self.prob = prob
        self.opt = kkt_default_options(prec, **opts)
        self.h = kkt_analyze(prob, self.opt)

    def factor(self, a_vals=None, b_vals=None, c_vals=None, stream=None):
        p = self.prob
        a = np.ascontiguousarray(p.a_vals, dtype=np.float64) if a_vals is None else a_vals
        b = np.ascontiguousarray(p.b_vals, dtype=np.float64) if b_vals is None else b_vals
        c = np.ascontiguousarray(p.c_vals, dtype=np.float64) if c_vals is None else c_vals
        return kkt_factor(self.h, a, b, c, stream)

    def solve(self, rhs=None, stream=None, allow_not_converged=False):
        r = np.ascontiguousarray(self.prob.rhs if rhs is None else rhs, dtype=np.float64)
        x = np.empty_like(r)
        kkt_solve(self.h, r, x, 1, stream, allow_not_converged)
        return x

    def info(self):
        return kkt_get_info(self.h)

    def close(self):
        if self.h:
            kkt_destroy(self.h)
            self.h = None

    def __del__(self):  # pragma: no cover
        try:
            self.close()
        except Exception:
            pass
