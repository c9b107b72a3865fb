"""Python binding of ``libfds.so`` (the C ABI in ``include/fds.h``).

Argument marshalling only: every step of the solver runs in the library's CUDA
kernels.  Device buffers are PyTorch CUDA tensors (complex128 / int32 /
float64 / int64), passed by ``data_ptr()``; streams are ``torch.cuda.Stream``
handles.  The library must have been built (``build.build()``); loading fails
loudly otherwise.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# FDS_LIB selects another build of the library (e.g. the bounds-checked libfds_checked.so)
LIB_PATH = os.environ.get("FDS_LIB") or os.path.join(HERE, "libfds.so")

FDS_OK = 0
FDS_ERR_ARG = -1
FDS_ERR_CUDA = -2
FDS_ERR_OOM = -3
FDS_ERR_SINGULAR = -4
FDS_ERR_NOT_CONVERGED = -5
FDS_ERR_TIMEOUT = -6
FDS_ERR_STATE = -7
FDS_FP64 = 0
FDS_MIXED = 1
FDS_APPLY_FF = 0
FDS_APPLY_FP64 = 1
FDS_C64_SIMT = 0
FDS_C64_TENSOR = 1
FDS_FW_FF = 0
FDS_FW_TENSOR = 1
FDS_VARIANT_LU = 0
FDS_VARIANT_MR2005 = 1
FDS_RANK_ADAPTIVE = 0
FDS_RANK_LEARNED = 1
FDS_FAULT_NONE = 0
FDS_FAULT_ALLOC = 1
FDS_FAULT_NAN_BLOCK = 2
FDS_FAULT_TC_STALL_FW = 3
FDS_FAULT_TC_STALL_C64 = 4
FDS_MLP_NIN = 16
FDS_MLP_NTRAIN = 5313
FDS_MLP_NPARAM = 5345


class FdsError(RuntimeError):
    def __init__(self, code, what):
        detail = ""
        if code in (FDS_ERR_CUDA, FDS_ERR_OOM):
            try:
                detail = " [" + lib().fds_last_error_detail().decode() + "]"
            except Exception:
                detail = ""
        super().__init__("%s failed: %s (%d)%s" % (what, _lib_err(code), code, detail))
        self.code = code


class fds_physics(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("mu", ctypes.c_double), ("rho", ctypes.c_double),
                ("omega", ctypes.c_double), ("alpha_re", ctypes.c_double), ("alpha_im", ctypes.c_double),
                ("alpha_set", ctypes.c_int32)]


class fds_geometry(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("xy", ctypes.POINTER(ctypes.c_double)), ("rho", ctypes.c_double)]


class fds_options(ctypes.Structure):
    _fields_ = [("leaf_size", ctypes.c_int32), ("proxy_ratio", ctypes.c_double),
                ("proxy_points", ctypes.c_int32), ("top_level", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("alpha_re", ctypes.c_double), ("alpha_im", ctypes.c_double),
                ("alpha_set", ctypes.c_int32), ("cuda_stream", ctypes.c_uint64), ("ir_tol", ctypes.c_double),
                ("ir_max_iter", ctypes.c_int32), ("ir_apply", ctypes.c_int32), ("sweep_fp64_levels", ctypes.c_int32),
                ("sweep_ff", ctypes.c_int32), ("merge_c64", ctypes.c_int32), ("rank_mode", ctypes.c_int32),
                ("mlp_params", ctypes.POINTER(ctypes.c_float)), ("sketch_extra", ctypes.c_int32),
                ("record_features", ctypes.c_int32), ("c64_engine", ctypes.c_int32), ("tol_decay", ctypes.c_double),
                ("variant", ctypes.c_int32), ("use_graph", ctypes.c_int32), ("fw_engine", ctypes.c_int32),
                ("merge_c64_levels", ctypes.c_int32)]


class fds_stats(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int32), ("levels", ctypes.c_int32), ("top_level", ctypes.c_int32),
                ("top_size", ctypes.c_int32), ("skeleton_dofs", ctypes.c_int64 * 32),
                ("max_rank", ctypes.c_int32 * 32), ("build_ms", ctypes.c_double), ("solve_ms", ctypes.c_double),
                ("factor_bytes", ctypes.c_int64), ("ir_iters", ctypes.c_int32), ("ir_residual", ctypes.c_double),
                ("id_sketched", ctypes.c_int64), ("id_fallback", ctypes.c_int64),
                ("features_recorded", ctypes.c_int64)]


_lib = None


def lib():
    """The loaded library; raises if it is missing (no fallback exists)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libfds.so not built: run paper_2411_18026_gb300.build.build() first")
    L = ctypes.CDLL(LIB_PATH)
    vp, dp, ip, lp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p, ctypes.c_void_p
    u64, i32, f64 = ctypes.c_uint64, ctypes.c_int32, ctypes.c_double
    L.fds_default_options.argtypes = [ctypes.POINTER(fds_options)]
    L.fds_default_options.restype = None
    L.fds_error_string.argtypes = [ctypes.c_int]
    L.fds_error_string.restype = ctypes.c_char_p
    L.fds_last_error_detail.argtypes = []
    L.fds_last_error_detail.restype = ctypes.c_char_p
    L.fds_build.argtypes = [ctypes.POINTER(fds_geometry), f64, f64, f64, f64, ctypes.POINTER(vp)]
    L.fds_build_ex.argtypes = [ctypes.POINTER(fds_geometry), f64, f64, f64, f64, ctypes.POINTER(fds_options),
                               ctypes.POINTER(vp)]
    L.fds_rhs_plane_wave.argtypes = [vp, ctypes.POINTER(i32), dp, i32, dp]
    L.fds_rhs_plane_wave_device.argtypes = [vp, vp, vp, i32, vp, u64]
    L.fds_solve.argtypes = [vp, dp, i32]
    L.fds_solve_device.argtypes = [vp, vp, i32, u64]
    L.fds_stats_get.argtypes = [vp, ctypes.POINTER(fds_stats)]
    L.fds_level_ranks.argtypes = [vp, i32, ctypes.POINTER(i32), i32]
    L.fds_destroy.argtypes = [vp]
    L.fds_destroy.restype = None
    L.fds_eval_entries.argtypes = [ctypes.POINTER(fds_physics), vp, i32, vp, i32, vp, i32, vp, u64]
    L.fds_eval_cross.argtypes = [ctypes.POINTER(fds_physics), vp, i32, vp, i32, vp, i32, vp, i32, i32, vp, u64]
    L.fds_id_batched.argtypes = [i32, vp, vp, vp, vp, f64, vp, vp, vp, vp, vp, u64]
    L.fds_lu_batched.argtypes = [i32, vp, vp, vp, vp, vp, vp, u64]
    L.fds_lu_batched_noalloc.argtypes = [i32, vp, vp, vp, vp, vp, vp, u64]
    L.fds_field.argtypes = [vp, vp, i32, ctypes.POINTER(i32), dp, vp, i32, vp, u64]
    L.fds_field_compressed.argtypes = [vp, vp, i32, ctypes.POINTER(i32), dp, vp, i32, vp, u64]
    i64p = ctypes.POINTER(ctypes.c_int64)
    L.fds_cgemm_c64_batched.argtypes = [i32, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32), i64p,
                                        i64p, i64p, vp, vp, vp, i32, ctypes.c_float, ctypes.c_float, i32, u64]
    L.fds_alu_peak.argtypes = [i32, ctypes.POINTER(ctypes.c_double)]
    L.fds_zgemm_blocks_tc.argtypes = [i32, ctypes.POINTER(i32), vp, vp, vp, i32, u64]
    L.fds_zgemm_jobs_tc.argtypes = [i32] + [vp] * 11 + [vp, vp, ctypes.c_int64, vp, ctypes.c_int64, i32, u64]
    L.fds_fault_inject.argtypes = [i32, ctypes.c_int64]
    L.fds_solve_batch_levels.argtypes = [i32, vp, vp, vp, i32, u64]
    L.fds_bounds_violations.argtypes = [ctypes.POINTER(ctypes.c_int64)]
    L.fds_autotune_enable.argtypes = [i32]
    L.fds_autotune_enable.restype = None
    L.fds_autotune_reset.argtypes = []
    L.fds_autotune_reset.restype = None
    L.fds_autotune_report.argtypes = [ctypes.c_char_p, i32]
    L.fds_timing_enable.argtypes = [i32]
    L.fds_timing_enable.restype = None
    L.fds_timing_reset.argtypes = []
    L.fds_timing_reset.restype = None
    L.fds_timing_report.argtypes = [ctypes.c_char_p, i32]
    L.fds_timing_report.restype = ctypes.c_int
    L.fds_launch_count.argtypes = []
    L.fds_launch_count.restype = ctypes.c_int64
    fp = ctypes.POINTER(ctypes.c_float)
    L.fds_features_get.argtypes = [vp, fp, fp, i32]
    L.fds_mlp_forward.argtypes = [vp, vp, i32, vp, u64]
    L.fds_mlp_loss_grad.argtypes = [vp, vp, vp, i32, vp, vp, u64]
    L.fds_mlp_adam.argtypes = [vp, vp, vp, vp, i32, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                               u64]
    L.fds_mlp_train.argtypes = [vp, vp, vp, i32, vp, i32, i32, ctypes.c_float, vp, u64]
    L.fds_build_batch.argtypes = [i32, ctypes.POINTER(fds_geometry), dp, f64, f64, f64, ctypes.POINTER(fds_options),
                                  i32, ctypes.POINTER(vp)]
    L.fds_solve_batch.argtypes = [i32, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(i32), i32]
    L.fds_handle_stream.argtypes = [vp]
    L.fds_handle_stream.restype = ctypes.c_uint64
    for f in ("fds_build", "fds_build_ex", "fds_rhs_plane_wave", "fds_rhs_plane_wave_device", "fds_solve",
              "fds_solve_device", "fds_stats_get", "fds_level_ranks", "fds_eval_entries", "fds_eval_cross",
              "fds_id_batched", "fds_lu_batched", "fds_lu_batched_noalloc", "fds_features_get", "fds_mlp_forward",
              "fds_mlp_loss_grad", "fds_mlp_adam", "fds_mlp_train", "fds_build_batch", "fds_solve_batch"):
        getattr(L, f).restype = ctypes.c_int
    _lib = L
    return L


def _lib_err(code):
    try:
        return lib().fds_error_string(int(code)).decode()
    except Exception:
        return "error"


def _check(rc, what):
    if rc < 0:
        raise FdsError(rc, what)
    return rc


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return ctypes.c_uint64(stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))


def physics(lam, mu, rho, omega, alpha=None):
    p = fds_physics(lam, mu, rho, omega, 0.0, 0.0, 0)
    if alpha is not None:
        p.alpha_re, p.alpha_im, p.alpha_set = float(np.real(alpha)), float(np.imag(alpha)), 1
    return p


def default_options():
    o = fds_options()
    lib().fds_default_options(ctypes.byref(o))
    return o


class Handle:
    """Owns an ``fds_handle*``; ``close()`` (or garbage collection) destroys it."""

    def __init__(self, ptr, n_nodes):
        self.ptr = ptr
        self.n = n_nodes

    def close(self):
        if self.ptr:
            lib().fds_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fds_build(xy, omega, lam, mu, tol, rho=1.0, leaf_size=64, top_level=1, proxy_ratio=1.5, proxy_points=64,
              alpha=None, stream=0, precision=FDS_FP64, ir_tol=None, ir_max_iter=None, ir_apply=None,
              mlp_params=None, sketch_extra=None, record_features=False, sweep_fp64_levels=None, merge_c64=False,
              sweep_ff=1, c64_engine=FDS_C64_SIMT, tol_decay=None, variant=FDS_VARIANT_LU, use_graph=False,
              fw_engine=FDS_FW_FF, merge_c64_levels=0):
    """Factorise; mlp_params (FDS_MLP_NPARAM floats) selects the learned-rank ID."""
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    g = fds_geometry(len(xy), xy.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(rho))
    o = default_options()
    o.leaf_size, o.top_level, o.proxy_ratio, o.proxy_points = leaf_size, top_level, proxy_ratio, proxy_points
    if alpha is not None:
        o.alpha_re, o.alpha_im, o.alpha_set = float(np.real(alpha)), float(np.imag(alpha)), 1
    o.cuda_stream = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    o.precision = precision
    if ir_tol is not None:
        o.ir_tol = ir_tol
    if ir_max_iter is not None:
        o.ir_max_iter = ir_max_iter
    if ir_apply is not None:
        o.ir_apply = ir_apply
    prm = None
    if mlp_params is not None:
        prm = np.ascontiguousarray(mlp_params, dtype=np.float32)
        if prm.size != FDS_MLP_NPARAM:
            raise ValueError("mlp_params must hold %d floats" % FDS_MLP_NPARAM)
        o.rank_mode = FDS_RANK_LEARNED
        o.mlp_params = prm.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    if sketch_extra is not None:
        o.sketch_extra = sketch_extra
    if sweep_fp64_levels is not None:
        o.sweep_fp64_levels = sweep_fp64_levels
    o.merge_c64 = 1 if merge_c64 else 0
    o.sweep_ff = int(sweep_ff)
    o.record_features = 1 if record_features else 0
    o.c64_engine = int(c64_engine)
    if tol_decay is not None:
        o.tol_decay = float(tol_decay)
    o.variant = int(variant)
    o.use_graph = 1 if use_graph else 0
    o.fw_engine = int(fw_engine)
    o.merge_c64_levels = int(merge_c64_levels)
    out = ctypes.c_void_p()
    _check(lib().fds_build_ex(ctypes.byref(g), float(omega), float(lam), float(mu), float(tol), ctypes.byref(o),
                              ctypes.byref(out)), "fds_build")
    return Handle(out, len(xy))


def fds_build_batch(cavities, lam, mu, tol, n_streams=8, rho=1.0, leaf_size=64, top_level=1, precision=FDS_FP64,
                    ir_tol=None, use_graph=False):
    """Build many cavities concurrently (dicts with 'xy' and 'omega'); returns handles."""
    n = len(cavities)
    xys = [np.ascontiguousarray(c["xy"], dtype=np.float64) for c in cavities]
    geoms = (fds_geometry * n)(*[fds_geometry(len(x), x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(rho))
                                 for x in xys])
    om = np.ascontiguousarray([c["omega"] for c in cavities], dtype=np.float64)
    o = default_options()
    o.leaf_size, o.top_level, o.precision = leaf_size, top_level, precision
    o.use_graph = 1 if use_graph else 0
    if ir_tol is not None:
        o.ir_tol = ir_tol
    out = (ctypes.c_void_p * n)()
    _check(lib().fds_build_batch(n, geoms, om.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), float(lam), float(mu),
                                 float(tol), ctypes.byref(o), int(n_streams), out), "fds_build_batch")
    return [Handle(ctypes.c_void_p(out[i]), len(xys[i])) for i in range(n)]


def fds_solve_batch(handles, d_rhs_list, n_streams=8):
    """Solve in place: d_rhs_list[i] complex128 CUDA tensor (nrhs_i, 2 n_i) for handle i."""
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*[h.ptr.value for h in handles])
    ps = (ctypes.c_void_p * n)(*[t.data_ptr() for t in d_rhs_list])
    nr = (ctypes.c_int32 * n)(*[t.shape[0] for t in d_rhs_list])
    _check(lib().fds_solve_batch(n, hs, ps, nr, int(n_streams)), "fds_solve_batch")


def fds_solve_batch_levels(handles, d_rhs_list, use_graph=False, stream=None):
    """Solve in place with one launch per tree level and phase across the
    cavities (FP64, LU-variant handles): d_rhs_list[i] complex128 CUDA
    tensor (nrhs_i, 2 n_i) for handle i."""
    n = len(handles)
    hs = (ctypes.c_void_p * n)(*[h.ptr.value for h in handles])
    ps = (ctypes.c_void_p * n)(*[t.data_ptr() for t in d_rhs_list])
    nr = (ctypes.c_int32 * n)(*[t.shape[0] for t in d_rhs_list])
    _check(lib().fds_solve_batch_levels(n, hs, ps, nr, 1 if use_graph else 0, _stream(stream)),
           "fds_solve_batch_levels")


def fds_handle_stream(h):
    return int(lib().fds_handle_stream(h.ptr))


def fds_rhs_plane_wave(h, kinds, angles):
    kinds = np.ascontiguousarray(kinds, dtype=np.int32)
    angles = np.ascontiguousarray(angles, dtype=np.float64)
    f = np.zeros((len(kinds), 2 * h.n), dtype=np.complex128)      # row j = column j (col-major)
    _check(lib().fds_rhs_plane_wave(h.ptr, kinds.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                    angles.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), len(kinds),
                                    f.view(np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
           "fds_rhs_plane_wave")
    return f.T


def fds_rhs_plane_wave_device(h, d_kinds, d_angles, d_f, stream=None):
    """d_f: complex128 CUDA tensor of shape (nrhs, 2n) (column-major 2n x nrhs)."""
    _check(lib().fds_rhs_plane_wave_device(h.ptr, _ptr(d_kinds), _ptr(d_angles), int(d_kinds.numel()),
                                           _ptr(d_f), _stream(stream)), "fds_rhs_plane_wave_device")


def fds_solve(h, F):
    """Host solve: F (2n,) or (2n, nrhs) complex; returns the solution."""
    F = np.asarray(F, dtype=np.complex128)
    one = F.ndim == 1
    X = np.array((F[:, None] if one else F).T, dtype=np.complex128, order="C", copy=True)   # (nrhs, 2n)
    _check(lib().fds_solve(h.ptr, X.view(np.float64).ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                           X.shape[0]), "fds_solve")
    return X[0] if one else X.T


def fds_solve_device(h, d_rhs, stream=None):
    """d_rhs: complex128 CUDA tensor (nrhs, 2n), solved in place."""
    nrhs = d_rhs.shape[0] if d_rhs.dim() == 2 else 1
    _check(lib().fds_solve_device(h.ptr, _ptr(d_rhs), nrhs, _stream(stream)), "fds_solve_device")


def fds_stats_get(h):
    s = fds_stats()
    _check(lib().fds_stats_get(h.ptr, ctypes.byref(s)), "fds_stats_get")
    return s


def fds_features_get(h):
    """(features [rows, 16] float32, adaptive rank fractions [rows]) recorded by a
    build with record_features=True."""
    n = int(fds_stats_get(h).features_recorded)
    feat = np.zeros((max(n, 1), FDS_MLP_NIN), dtype=np.float32)
    frac = np.zeros(max(n, 1), dtype=np.float32)
    fp = ctypes.POINTER(ctypes.c_float)
    got = _check(lib().fds_features_get(h.ptr, feat.ctypes.data_as(fp), frac.ctypes.data_as(fp), n),
                 "fds_features_get")
    return feat[:got], frac[:got]


def fds_mlp_forward(d_params, d_X, d_y, stream=None):
    _check(lib().fds_mlp_forward(_ptr(d_params), _ptr(d_X), d_X.shape[0], _ptr(d_y), _stream(stream)),
           "fds_mlp_forward")


def fds_mlp_loss_grad(d_params, d_X, d_t, d_grad, d_loss, stream=None):
    _check(lib().fds_mlp_loss_grad(_ptr(d_params), _ptr(d_X), _ptr(d_t), d_X.shape[0], _ptr(d_grad), _ptr(d_loss),
                                   _stream(stream)), "fds_mlp_loss_grad")


def fds_mlp_adam(d_params, d_grad, d_m, d_v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    _check(lib().fds_mlp_adam(_ptr(d_params), _ptr(d_grad), _ptr(d_m), _ptr(d_v), int(step), float(lr), float(beta1),
                              float(beta2), float(eps), _stream(stream)), "fds_mlp_adam")


def fds_mlp_train(d_params, d_X, d_t, d_order, batch, lr, d_losses=None, stream=None):
    _check(lib().fds_mlp_train(_ptr(d_params), _ptr(d_X), _ptr(d_t), d_X.shape[0], _ptr(d_order), d_order.numel(),
                               int(batch), float(lr), _ptr(d_losses), _stream(stream)), "fds_mlp_train")


def fds_level_ranks(h, level, nb):
    k = (ctypes.c_int32 * (2 * nb))()
    n = _check(lib().fds_level_ranks(h.ptr, level, k, 2 * nb), "fds_level_ranks")
    return np.array(k[:n], dtype=np.int32).reshape(-1, 2)


def fds_eval_entries(phys, d_xy, d_rows, d_cols, d_out, stream=None):
    """d_out: complex128 CUDA tensor, (2 nc, 2 nr) row-major = (2nr x 2nc) column-major."""
    _check(lib().fds_eval_entries(ctypes.byref(phys), _ptr(d_xy), d_xy.shape[0], _ptr(d_rows), d_rows.numel(),
                                  _ptr(d_cols), d_cols.numel(), _ptr(d_out), _stream(stream)), "fds_eval_entries")


def fds_eval_cross(phys, d_X, d_rows, d_Y, d_cols, q, d_out, stream=None):
    _check(lib().fds_eval_cross(ctypes.byref(phys), _ptr(d_X), d_X.shape[0], _ptr(d_rows), d_rows.numel(),
                                _ptr(d_Y), d_Y.shape[0], _ptr(d_cols), d_cols.numel(), int(q), _ptr(d_out),
                                _stream(stream)), "fds_eval_cross")


def fds_id_batched(d_m, d_n, d_off, d_Y, tol, d_rank, d_perm, d_poff, d_T, d_toff, stream=None):
    _check(lib().fds_id_batched(d_m.numel(), _ptr(d_m), _ptr(d_n), _ptr(d_off), _ptr(d_Y), float(tol),
                                _ptr(d_rank), _ptr(d_perm), _ptr(d_poff), _ptr(d_T), _ptr(d_toff),
                                _stream(stream)), "fds_id_batched")


def fds_lu_batched_noalloc(d_d, d_off, d_A, d_piv, d_poff, d_info, stream=None):
    """Allocation-free variant of fds_lu_batched (see include/fds.h)."""
    _check(lib().fds_lu_batched_noalloc(d_d.numel(), _ptr(d_d), _ptr(d_off), _ptr(d_A), _ptr(d_piv), _ptr(d_poff),
                                        _ptr(d_info), _stream(stream)), "fds_lu_batched_noalloc")


def fds_lu_batched(d_d, d_off, d_A, d_piv, d_poff, d_info, stream=None):
    _check(lib().fds_lu_batched(d_d.numel(), _ptr(d_d), _ptr(d_off), _ptr(d_A), _ptr(d_piv), _ptr(d_poff),
                                _ptr(d_info), _stream(stream)), "fds_lu_batched")


def fds_field(h, d_u, kinds, angles, pts, stream=None, compressed=False):
    """Displacement at points off the boundary (eq. integ_rep) from the device
    solution d_u ((nrhs, 2n) complex128 CUDA tensor) of the given waves.
    pts: (npts, 2).  compressed: through the tree's skeletons
    (fds_field_compressed) instead of direct summation.  Returns
    (2, npts, nrhs) complex numpy."""
    import torch
    kinds = np.ascontiguousarray(kinds, dtype=np.int32)
    angles = np.ascontiguousarray(angles, dtype=np.float64)
    nrhs = len(kinds)
    d_pts = torch.tensor(np.ascontiguousarray(pts, dtype=np.float64).ravel(), device=d_u.device)
    npts = d_pts.numel() // 2
    d_out = torch.zeros((nrhs, 2 * npts), dtype=torch.complex128, device=d_u.device)
    fn = lib().fds_field_compressed if compressed else lib().fds_field
    _check(fn(h.ptr, _ptr(d_u), nrhs, kinds.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
              angles.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), _ptr(d_pts), npts, _ptr(d_out),
              _stream(stream)), "fds_field")
    return d_out.cpu().numpy().T.reshape(2, npts, nrhs)


def fds_cgemm_c64_batched(m, n, k, aoff, boff, coff, d_A, d_B, d_C, opA=0, alpha=1.0, beta=0.0,
                          engine=FDS_C64_TENSOR, stream=None):
    """Batched complex64 C_b = alpha op(A_b) B_b + beta C_b (device complex64 buffers, host sizes)."""
    batch = len(m)
    arr = lambda v, t: np.ascontiguousarray(v, dtype=t)
    m, n, k = arr(m, np.int32), arr(n, np.int32), arr(k, np.int32)
    aoff, boff, coff = arr(aoff, np.int64), arr(boff, np.int64), arr(coff, np.int64)
    i32p, i64p = ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int64)
    _check(lib().fds_cgemm_c64_batched(batch, m.ctypes.data_as(i32p), n.ctypes.data_as(i32p),
                                       k.ctypes.data_as(i32p), aoff.ctypes.data_as(i64p),
                                       boff.ctypes.data_as(i64p), coff.ctypes.data_as(i64p), _ptr(d_A), _ptr(d_B),
                                       _ptr(d_C), int(opA), float(alpha), float(beta), int(engine),
                                       _stream(stream)), "fds_cgemm_c64_batched")


def fds_alu_peak(kind):
    """Measured FMA peak of the current device in TFLOP/s: kind 0 FP64, 1 FP32."""
    v = ctypes.c_double()
    _check(lib().fds_alu_peak(int(kind), ctypes.byref(v)), "fds_alu_peak")
    return v.value


def fds_zgemm_blocks_tc(d, d_A, d_X, d_Y, stream=None):
    """Y_b += A_b X_b on the tensor cores (six bf16 slices per FP64 operand).
    d: block sizes; d_A: complex128 CUDA tensor of the blocks back to back
    (column-major); d_X, d_Y: complex128 (nc, sum d) tensors (column-major
    (sum d) x nc); d_Y updated in place."""
    d = np.ascontiguousarray(d, dtype=np.int32)
    nc = d_X.shape[0] if d_X.dim() == 2 else 1
    _check(lib().fds_zgemm_blocks_tc(len(d), d.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _ptr(d_A),
                                     _ptr(d_X), _ptr(d_Y), nc, _stream(stream)), "fds_zgemm_blocks_tc")


def fds_fault_inject(kind, arg=0):
    """Arms one injected fault (FDS_FAULT_*; fires once) or, with
    FDS_FAULT_NONE, disarms all of them."""
    _check(lib().fds_fault_inject(int(kind), int(arg)), "fds_fault_inject")


def fds_bounds_violations():
    """Out-of-range mapped accesses since the last call (bounds-checked
    library only; FdsError with FDS_ERR_STATE otherwise)."""
    n = ctypes.c_int64(0)
    _check(lib().fds_bounds_violations(ctypes.byref(n)), "fds_bounds_violations")
    return int(n.value)


def fds_zgemm_jobs_tc(m, k, op, a_off, lda, x_row, xmap_off, y_row, ymap_off, set_, maps, d_A, d_X, d_Y,
                      stream=None):
    """General block products on the tensor cores (see include/fds.h):
    per-job host arrays, maps (int32 host array), d_A complex128 CUDA
    tensor, d_X / d_Y complex128 (nc, rows) tensors (column-major rows x nc,
    leading dimension = rows); d_Y updated in place."""
    a = [np.ascontiguousarray(v, dtype=t) for v, t in
         ((m, np.int32), (k, np.int32), (op, np.int32), (a_off, np.int64), (lda, np.int32), (x_row, np.int64),
          (xmap_off, np.int64), (y_row, np.int64), (ymap_off, np.int64), (set_, np.int32))]
    mp = np.ascontiguousarray(maps if maps is not None and len(maps) else np.zeros(1), dtype=np.int32)
    nc = d_X.shape[0]
    _check(lib().fds_zgemm_jobs_tc(len(a[0]), *[v.ctypes.data for v in a], mp.ctypes.data, _ptr(d_A), _ptr(d_X),
                                   d_X.shape[1], _ptr(d_Y), d_Y.shape[1], nc, _stream(stream)), "fds_zgemm_jobs_tc")


def fds_autotune_enable(on=True):
    lib().fds_autotune_enable(1 if on else 0)


def fds_autotune_reset():
    lib().fds_autotune_reset()


def fds_autotune_report():
    """[dict(arith, opA, rows, cols, batch, mapped, mi, tj, best_us, rule_us)] of the tuned classes."""
    n = lib().fds_autotune_report(None, 0)
    buf = ctypes.create_string_buffer(n + 16)
    lib().fds_autotune_report(buf, n + 16)
    out = []
    for line in buf.value.decode().splitlines():
        v = line.split()
        out.append(dict(arith=v[0], opA=int(v[1]), rows=int(v[2]), cols=int(v[3]), batch=int(v[4]), mapped=int(v[5]),
                        mi=int(v[6]), tj=int(v[7]), best_us=float(v[8]), rule_us=float(v[9])))
    return out


def fds_timing_enable(on=True):
    lib().fds_timing_enable(1 if on else 0)


def fds_timing_reset():
    lib().fds_timing_reset()


def fds_timing_report():
    """{phase: dict(launches, ms, flops, bytes)} accumulated since the last reset."""
    n = lib().fds_timing_report(None, 0)
    buf = ctypes.create_string_buffer(n + 16)
    lib().fds_timing_report(buf, n + 16)
    out = {}
    for line in buf.value.decode().splitlines():
        name, launches, ms, flops, nbytes, units = line.split()
        out[name] = dict(launches=int(launches), ms=float(ms), flops=float(flops), bytes=float(nbytes),
                         units=float(units))
    return out


def fds_launch_count():
    return int(lib().fds_launch_count())
