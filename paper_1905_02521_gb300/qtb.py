"""Thin Python binding of the C ABI in ``include/qtb.h`` (argument marshalling only).

Every function keeps the C name and calls straight into ``_lib/libqtb.so``;
all arithmetic of the step runs in the library's CUDA kernels.  Device memory
is requested from PyTorch's caching allocator through the allocator callbacks
of ``qtb_params``, and work is issued on PyTorch's current CUDA stream.

Importing this module loads the shared library and raises if it has not been
built (``paper_1905_02521_gb300.build.build()``): there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

NREC = 23
TC_FILTER = True        # the BF16 tcgen05 Toeplitz-GEMM filter is available (QTB_FILTER_BF16)
OK, ERR_ARG, ERR_CUDA, ERR_OOM, ERR_TIMEOUT, ERR_NONFINITE, ERR_SOLVE, ERR_OVERFLOW, ERR_STATE = \
    0, -1, -2, -3, -4, -5, -6, -7, -8
FP64, MIXED = 0, 1
FILTER_FP64, FILTER_FP32, FILTER_BF16 = 0, 1, 2
NOISE_WHITE, NOISE_QTB, NOISE_QTB_PIMD, NOISE_QTB_PIMD_MLP = 0, 1, 2, 3
POT_PAIR, POT_HARMONIC, POT_DOUBLEWELL = 0, 1, 2
GEN_FILTER, GEN_FOURIER = 0, 1


class QtbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"qtb error {code}: {msg}")
        self.code = code


class qtb_system(C.Structure):
    _fields_ = [("n_atoms", C.c_int), ("n_beads", C.c_int), ("type", C.c_void_p), ("pos", C.c_void_p),
                ("vel", C.c_void_p), ("box", C.c_double * 3), ("T", C.c_double), ("gamma", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)


class qtb_params(C.Structure):
    _fields_ = [("n_types", C.c_int), ("mass", C.c_void_p), ("charge", C.c_void_p), ("buck_A", C.c_void_p),
                ("buck_rho", C.c_void_p), ("buck_C", C.c_void_p), ("dsf_alpha", C.c_double),
                ("r_cut", C.c_double), ("potential", C.c_int), ("ext_omega", C.c_double),
                ("ext_V0", C.c_double), ("ext_a", C.c_double), ("dt", C.c_double), ("precision", C.c_int),
                ("filter_prec", C.c_int), ("seed", C.c_ulonglong), ("obs_stride", C.c_int),
                ("max_records", C.c_int), ("dev_alloc", ALLOC_FN), ("dev_free", FREE_FN),
                ("alloc_user", C.c_void_p), ("skin", C.c_double), ("nm_layout", C.c_int),
                ("list_lanes", C.c_int), ("rebuild_scope", C.c_int), ("npt", C.c_int), ("pressure", C.c_double),
                ("cell_mass", C.c_double), ("cell_gamma", C.c_double)]


_lib = None


def lib_path():
    return _build.LIB


def lib():
    """Load ``libqtb.so`` (raises if missing: there is no CPU fallback)."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"CUDA library {path} is not built; run paper_1905_02521_gb300.build.build()")
        L = C.CDLL(path)
        vp, i, d, ll = C.c_void_p, C.c_int, C.c_double, C.c_longlong
        sig = {
            "qtb_init": ([C.POINTER(vp), vp, i, vp, vp], i),
            "qtb_set_filter": ([vp, i, i, i, d], i),
            "qtb_step_n": ([vp, ll], i),
            "qtb_sync": ([vp], i),
            "qtb_observables": ([vp, i, vp], i),
            "qtb_get_series": ([vp, i, vp, i, C.POINTER(i)], i),
            "qtb_get_state": ([vp, i, vp, vp], i),
            "qtb_set_state": ([vp, i, vp, vp], i),
            "qtb_get_forces": ([vp, i, vp], i),
            "qtb_get_taps": ([vp, i, vp, i, C.POINTER(i)], i),
            "qtb_get_noise": ([vp, i, vp, C.POINTER(ll)], i),
            "qtb_get_step": ([vp, C.POINTER(ll)], i),
            "qtb_get_cell": ([vp, i, vp, C.POINTER(d)], i),
            "qtb_set_cell": ([vp, i, vp, d], i),
            "qtb_fp32_peak": ([C.POINTER(d), C.POINTER(d)], i),
            "qtb_list_rebuilds": ([vp, C.POINTER(ll)], i),
            "qtb_rebuild_lists": ([vp], i),
            "qtb_wait_selftest": ([vp, C.POINTER(i), C.POINTER(d)], i),
            "qtb_set_generator": ([vp, i, i], i),
            "qtb_autotune": ([vp, i, vp, vp, i, i, d, i, i, vp, vp], i),
            "qtb_set_profiling": ([vp, i], i),
            "qtb_kernel_times": ([vp, vp, vp, i], i),
            "qtb_kappa_solve": ([i, i, d, d, vp], i),
            "qtb_kappa_solve_noalloc": ([i, i, d, d, vp, vp], i),
            "qtb_kappa_model_create": ([C.POINTER(vp), C.c_ulonglong], i),
            "qtb_kappa_model_train": ([vp, vp, i, i, i, d], i),
            "qtb_kappa_model_grad": ([vp, vp, vp, i, vp, vp], i),
            "qtb_kappa_model_eval": ([vp, i, vp, i, vp], i),
            "qtb_kappa_model_get_weights": ([vp, vp, i], i),
            "qtb_kappa_model_set_weights": ([vp, vp, i], i),
            "qtb_kappa_model_info": ([vp, vp, vp, i, C.POINTER(i), C.POINTER(d), C.POINTER(d)], i),
            "qtb_kappa_model_destroy": ([vp], None),
            "qtb_set_kappa_model": ([vp, vp], i),
            "qtb_filter_source": ([vp, i, C.POINTER(i)], i),
            "qtb_destroy": ([vp], None),
            "qtb_last_error": ([], C.c_char_p),
        }
        for name, (args, res) in sig.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = res
        _lib = L
    return _lib


def _check(rc):
    if rc != OK:
        raise QtbError(rc, lib().qtb_last_error().decode())
    return rc


def _ptr(a):
    return None if a is None else a.ctypes.data


# --- torch allocator callbacks ------------------------------------------------

_torch_cb = None


def _torch_allocator():
    global _torch_cb
    if _torch_cb is None:
        import torch

        def _alloc(nbytes, user):
            try:
                return int(torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                              torch.cuda.current_stream()))
            except Exception:   # allocation failure is reported by the library as QTB_ERR_OOM
                return None

        def _free(ptr, user):
            if ptr:
                torch.cuda.caching_allocator_delete(ptr)

        _torch_cb = (ALLOC_FN(_alloc), FREE_FN(_free))
    return _torch_cb


def torch_stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


# --- C-named entry points ---------------------------------------------------------

def _c_args(systems, params, stream):
    """C structures (systems array, params) for qtb_init / qtb_autotune and the
    host arrays they borrow (keep alive for the call)."""
    keep = []
    arr = (qtb_system * len(systems))()
    for k, s in enumerate(systems):
        pos = np.ascontiguousarray(s["pos"], np.float64)
        if pos.ndim == 2:
            pos = pos[None]
        vel = None if s.get("vel") is None else np.ascontiguousarray(s["vel"], np.float64).reshape(pos.shape)
        typ = np.ascontiguousarray(s["types"], np.int32)
        keep += [pos, vel, typ]
        arr[k].n_atoms, arr[k].n_beads = pos.shape[1], pos.shape[0]
        arr[k].type, arr[k].pos, arr[k].vel = typ.ctypes.data, pos.ctypes.data, _ptr(vel)
        box = s.get("box")
        for c in range(3):
            arr[k].box[c] = 0.0 if box is None else float(box[c])
        arr[k].T, arr[k].gamma = float(s["T"]), float(s["gamma"])
    p = qtb_params()
    nt = len(params["mass"])
    tabs = {}
    for key, shape in (("mass", nt), ("charge", nt), ("buck_A", nt * nt), ("buck_rho", nt * nt), ("buck_C", nt * nt)):
        default = np.ones(shape) if key == "buck_rho" else np.zeros(shape)
        tabs[key] = np.ascontiguousarray(np.asarray(params.get(key, default), np.float64).reshape(shape))
        setattr(p, key, tabs[key].ctypes.data)
    keep.append(tabs)
    p.n_types = nt
    p.dsf_alpha = float(params.get("dsf_alpha", 0.0))
    p.r_cut = float(params.get("r_cut", 0.0))
    p.potential = int(params.get("potential", POT_PAIR))
    p.ext_omega = float(params.get("ext_omega", 0.0))
    p.ext_V0 = float(params.get("ext_V0", 0.0))
    p.ext_a = float(params.get("ext_a", 1.0))
    p.dt = float(params["dt"])
    p.precision = int(params.get("precision", FP64))
    p.filter_prec = int(params.get("filter_prec", FILTER_FP32))
    p.seed = int(params.get("seed", 12345))
    p.obs_stride = int(params.get("obs_stride", 1))
    p.max_records = int(params.get("max_records", 4096))
    p.skin = float(params.get("skin", 0.0))
    p.nm_layout = int(params.get("nm_layout", 0))
    p.list_lanes = int(params.get("list_lanes", 0))
    p.rebuild_scope = int(params.get("rebuild_scope", 0))
    p.npt = int(params.get("npt", 0))
    p.pressure = float(params.get("pressure", 0.0))
    p.cell_mass = float(params.get("cell_mass", 0.0))
    p.cell_gamma = float(params.get("cell_gamma", 0.0))
    if params.get("torch_alloc", True):
        a, f = _torch_allocator()
        p.dev_alloc, p.dev_free = a, f
    if stream is None and params.get("torch_stream", True):
        stream = torch_stream()
    return arr, p, stream, keep


def qtb_init(systems, params, stream=None):
    """systems: list of dicts (pos [P,N,3], vel, types, box, T, gamma); params: dict.

    Returns an opaque context handle (an integer)."""
    arr, p, stream, keep = _c_args(systems, params, stream)
    h = C.c_void_p()
    _check(lib().qtb_init(C.byref(h), C.cast(arr, C.c_void_p), len(systems), C.addressof(p), stream))
    return h.value


class qtb_tuning(C.Structure):
    _fields_ = [("skin", C.c_double), ("nm_layout", C.c_int), ("list_lanes", C.c_int), ("rebuild_scope", C.c_int),
                ("ms_per_step", C.c_double),
                ("default_ms_per_step", C.c_double), ("n_tried", C.c_int)]


def qtb_autotune(systems, params, mode=0, n_taps=1, omega_max=0.0, n_blocks=2, equil_blocks=0, stream=None):
    """Times the candidate skins, lane counts, integrator layouts and rebuild
    scopes on these systems (see qtb.h), each from the state reached after
    equil_blocks blocks with the defaults, and returns (params with the fastest
    choice, tuning dict)."""
    arr, p, stream, keep = _c_args(systems, params, stream)
    best = qtb_params()
    res = qtb_tuning()
    _check(lib().qtb_autotune(C.cast(arr, C.c_void_p), len(systems), C.addressof(p), stream, int(mode), int(n_taps),
                              float(omega_max), int(n_blocks), int(equil_blocks), C.addressof(best), C.byref(res)))
    tuned = dict(params, skin=best.skin, nm_layout=best.nm_layout, list_lanes=best.list_lanes,
                 rebuild_scope=best.rebuild_scope)
    info = {k: getattr(res, k) for k, _ in qtb_tuning._fields_}
    return tuned, info


def qtb_set_filter(ctx, sys, mode, n_taps=1, omega_max=0.0):
    _check(lib().qtb_set_filter(ctx, sys, mode, n_taps, omega_max))


def qtb_set_generator(ctx, generator, segment_blocks=1):
    _check(lib().qtb_set_generator(ctx, int(generator), int(segment_blocks)))


def qtb_step_n(ctx, n):
    _check(lib().qtb_step_n(ctx, int(n)))


def qtb_sync(ctx):
    _check(lib().qtb_sync(ctx))


def qtb_observables(ctx, sys):
    out = np.zeros(NREC)
    _check(lib().qtb_observables(ctx, sys, out.ctypes.data))
    return out


def qtb_get_series(ctx, sys, max_records):
    out = np.zeros((max_records, NREC))
    n = C.c_int(0)
    _check(lib().qtb_get_series(ctx, sys, out.ctypes.data, max_records, C.byref(n)))
    return out[:n.value]


def qtb_get_state(ctx, sys, n_beads, n_atoms):
    pos = np.zeros((n_beads, n_atoms, 3))
    vel = np.zeros((n_beads, n_atoms, 3))
    _check(lib().qtb_get_state(ctx, sys, pos.ctypes.data, vel.ctypes.data))
    return pos, vel


def qtb_get_state_into(ctx, sys, pos, vel):
    """qtb_get_state into caller-owned C-contiguous float64 arrays [P][N][3]
    (e.g. views of page-locked host memory); either may be None."""
    for a in (pos, vel):
        if a is not None:
            assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
    _check(lib().qtb_get_state(ctx, sys, None if pos is None else pos.ctypes.data,
                               None if vel is None else vel.ctypes.data))


def qtb_set_state(ctx, sys, pos=None, vel=None):
    pos = None if pos is None else np.ascontiguousarray(pos, np.float64)
    vel = None if vel is None else np.ascontiguousarray(vel, np.float64)
    _check(lib().qtb_set_state(ctx, sys, _ptr(pos), _ptr(vel)))


def qtb_get_forces(ctx, sys, n_beads, n_atoms):
    f = np.zeros((n_beads, n_atoms, 3))
    _check(lib().qtb_get_forces(ctx, sys, f.ctypes.data))
    return f


def qtb_get_taps(ctx, sys, max_taps=1 << 16):
    h = np.zeros(max_taps)
    n = C.c_int(0)
    _check(lib().qtb_get_taps(ctx, sys, h.ctypes.data, max_taps, C.byref(n)))
    return h[:n.value]


def qtb_get_noise(ctx, sys, ndof):
    out = np.zeros((256, ndof))
    b = C.c_longlong(0)
    _check(lib().qtb_get_noise(ctx, sys, out.ctypes.data, C.byref(b)))
    return out, b.value


def qtb_list_rebuilds(ctx):
    n = C.c_longlong()
    _check(lib().qtb_list_rebuilds(ctx, C.byref(n)))
    return int(n.value)


def qtb_rebuild_lists(ctx):
    """Rebuild every system's neighbour lists at the next force evaluation (see qtb.h)."""
    _check(lib().qtb_rebuild_lists(ctx))


def qtb_wait_selftest(ctx):
    """Runs the bounded-wait self-test (see qtb.h); returns (gave_up, ms)."""
    g, ms = C.c_int(0), C.c_double(0.0)
    _check(lib().qtb_wait_selftest(ctx, C.byref(g), C.byref(ms)))
    return bool(g.value), ms.value


def qtb_get_step(ctx):
    s = C.c_longlong(0)
    _check(lib().qtb_get_step(ctx, C.byref(s)))
    return s.value


KERNEL_CLASSES = ("white", "filter", "integrate", "rebuild", "force", "reduce")


def qtb_get_cell(ctx, sys):
    """(cell edges [3] in A, cell momentum p_e in eV fs) of system sys."""
    box = np.zeros(3)
    pe = C.c_double(0.0)
    _check(lib().qtb_get_cell(ctx, sys, box.ctypes.data, C.byref(pe)))
    return box, pe.value


def qtb_set_cell(ctx, sys, box, p_e):
    """Set the cell edges [3] (A, isotropic scale of the initial edges) and cell momentum (eV fs)."""
    box = np.ascontiguousarray(box, np.float64)
    _check(lib().qtb_set_cell(ctx, sys, box.ctypes.data, float(p_e)))


def qtb_fp32_peak():
    """(measured FP32 FMA throughput in TFLOP/s, best launch time in ms) of the current GPU."""
    t, ms = C.c_double(0.0), C.c_double(0.0)
    _check(lib().qtb_fp32_peak(C.byref(t), C.byref(ms)))
    return t.value, ms.value


def qtb_set_profiling(ctx, enable=True):
    _check(lib().qtb_set_profiling(ctx, int(bool(enable))))


def qtb_kernel_times(ctx):
    n = len(KERNEL_CLASSES)
    ms = np.zeros(n)
    cnt = np.zeros(n, np.int32)
    _check(lib().qtb_kernel_times(ctx, ms.ctypes.data, cnt.ctypes.data, n))
    return {k: (float(ms[i]), int(cnt[i])) for i, k in enumerate(KERNEL_CLASSES)}


def qtb_kappa_solve(P, n=1024, y_max=1000.0, y0=1.0):
    F = np.zeros(n)
    _check(lib().qtb_kappa_solve(P, n, y_max, y0, F.ctypes.data))
    return F


def qtb_kappa_solve_noalloc(P, n, y_max, y0, F_dev_ptr, stream=None):
    """F_dev_ptr: device address of a caller-owned [n] float64 buffer."""
    _check(lib().qtb_kappa_solve_noalloc(P, n, y_max, y0, F_dev_ptr, stream))


NPARAM = 4417


def qtb_kappa_model_create(seed=1):
    h = C.c_void_p()
    _check(lib().qtb_kappa_model_create(C.byref(h), int(seed)))
    return h.value


def qtb_kappa_model_train(model, P_list, n_per_P=3200, iters=4000, tol=2e-3):
    P = np.ascontiguousarray(P_list, np.int32)
    _check(lib().qtb_kappa_model_train(model, P.ctypes.data, len(P), n_per_P, iters, tol))


def qtb_kappa_model_grad(model, x, t):
    x = np.ascontiguousarray(x, np.float32)
    t = np.ascontiguousarray(t, np.float32)
    g = np.zeros(NPARAM, np.float32)
    loss = np.zeros(1, np.float32)
    _check(lib().qtb_kappa_model_grad(model, x.ctypes.data, t.ctypes.data, len(t), g.ctypes.data, loss.ctypes.data))
    return float(loss[0]), g


def qtb_kappa_model_eval(model, P, y):
    y = np.ascontiguousarray(y, np.float64)
    r = np.zeros_like(y)
    _check(lib().qtb_kappa_model_eval(model, int(P), y.ctypes.data, len(y), r.ctypes.data))
    return r


def qtb_kappa_model_get_weights(model):
    w = np.zeros(NPARAM, np.float32)
    _check(lib().qtb_kappa_model_get_weights(model, w.ctypes.data, NPARAM))
    return w


def qtb_kappa_model_set_weights(model, w):
    w = np.ascontiguousarray(w, np.float32)
    _check(lib().qtb_kappa_model_set_weights(model, w.ctypes.data, len(w)))


def qtb_kappa_model_info(model, max_p=64):
    P = np.zeros(max_p, np.int32)
    e = np.zeros(max_p)
    n = C.c_int(0)
    ms, loss = C.c_double(0), C.c_double(0)
    _check(lib().qtb_kappa_model_info(model, P.ctypes.data, e.ctypes.data, max_p, C.byref(n), C.byref(ms),
                                      C.byref(loss)))
    return {"P": P[:n.value].tolist(), "err": e[:n.value].tolist(), "train_ms": ms.value, "loss": loss.value}


def qtb_kappa_model_destroy(model):
    if model:
        lib().qtb_kappa_model_destroy(model)


def qtb_set_kappa_model(ctx, model):
    _check(lib().qtb_set_kappa_model(ctx, model))


def qtb_filter_source(ctx, sys):
    s = C.c_int(0)
    _check(lib().qtb_filter_source(ctx, sys, C.byref(s)))
    return s.value


def qtb_destroy(ctx):
    if ctx:
        lib().qtb_destroy(ctx)


def qtb_last_error():
    return lib().qtb_last_error().decode()
