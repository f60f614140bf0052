"""Python binding of the C ABI in include/kkm.h (argument marshalling only).

Every computation runs in ``libkkm.so``; this module converts tensors and
arrays to pointers, calls the C function of the same name and raises
``KKMError`` on a non-OK status.  Inputs may be CUDA tensors (device pointers)
or host arrays (numpy / CPU tensors); device work runs on the current torch
stream of the input's device.  There is no fallback: a missing library is an
error.
"""

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libkkm.so")

KKM_RBF, KKM_RMSD, KKM_LINEAR = 0, 1, 2
KKM_FP32, KKM_BF16, KKM_FP8 = 0, 1, 2
PIPELINE = {"auto": 0, "serial": 1, "overlap": 2}
ITERATION = {"auto": 0, "fused": 1, "split": 2, "tc": 3}
KKM_STRIDE, KKM_BLOCK = 0, 1
KKM_ASSIGN_SUPPORTS, KKM_ASSIGN_MEDOIDS = 0, 1
KIND = {"rbf": KKM_RBF, "rmsd": KKM_RMSD, "linear": KKM_LINEAR}
SAMPLING = {"stride": KKM_STRIDE, "block": KKM_BLOCK}
MODE = {"supports": KKM_ASSIGN_SUPPORTS, "medoids": KKM_ASSIGN_MEDOIDS}
STATUS_EINVAL = 1


class KKMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


class kkm_kernel(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("sigma", ctypes.c_float), ("n_atoms", ctypes.c_int32)]


class kkm_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("sampling", ctypes.c_int32),
                ("early_stop", ctypes.c_int32), ("pipeline", ctypes.c_int32),
                ("iteration", ctypes.c_int32),
                ("init_medoids", ctypes.POINTER(ctypes.c_int64)), ("stream", ctypes.c_void_p)]


class kkm_problem(ctypes.Structure):
    _fields_ = [("X", ctypes.c_void_p), ("N", ctypes.c_int64), ("d", ctypes.c_int64),
                ("C", ctypes.c_int32), ("B", ctypes.c_int32), ("s", ctypes.c_double),
                ("kernel", kkm_kernel), ("iters", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("opt", kkm_options), ("labels_out", ctypes.c_void_p)]


class kkm_server_config(ctypes.Structure):
    _fields_ = [("budget_bytes", ctypes.c_uint64), ("n_workers", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("max_batch_rows", ctypes.c_int64)]


class kkm_serving_stats(ctypes.Structure):
    _fields_ = [("completed_fit", ctypes.c_int64), ("completed_assign", ctypes.c_int64),
                ("failed", ctypes.c_int64), ("refused", ctypes.c_int64),
                ("fused_assign_launches", ctypes.c_int64), ("queued", ctypes.c_int64),
                ("p50_fit_ms", ctypes.c_double), ("p99_fit_ms", ctypes.c_double),
                ("p50_assign_ms", ctypes.c_double), ("p99_assign_ms", ctypes.c_double),
                ("kernel_evals", ctypes.c_double), ("seconds", ctypes.c_double),
                ("bytes_in_use", ctypes.c_uint64), ("peak_bytes", ctypes.c_uint64)]


_lib = None
_P = ctypes.c_void_p
_I32, _I64, _U64, _F32, _F64 = (ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64,
                                ctypes.c_float, ctypes.c_double)

_SIGNATURES = {
    "kkm_options_default": (None, [ctypes.POINTER(kkm_options)]),
    "kkm_fit": (_I32, [_P, _I64, _I64, _I32, _I32, _F64, ctypes.POINTER(kkm_kernel), _I32, _U64,
                       ctypes.POINTER(kkm_options), _P, ctypes.POINTER(_P)]),
    "kkm_fit_batch": (_I32, [_P, _I32, _I32, _P, _P, _P]),
    "kkm_fit_range": (_I32, [_P, _I64, _I64, _I32, _I32, _F64, ctypes.POINTER(kkm_kernel), _I32, _U64,
                             ctypes.POINTER(kkm_options), _P, _I32, _P, ctypes.POINTER(_P), ctypes.POINTER(_P)]),
    "kkm_checkpoint_info": (_I32, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32), ctypes.POINTER(_I32),
                                   ctypes.POINTER(_F32), _P]),
    "kkm_checkpoint_save": (_I32, [_P, ctypes.c_char_p]),
    "kkm_checkpoint_load": (_I32, [ctypes.c_char_p, ctypes.POINTER(_P)]),
    "kkm_checkpoint_free": (None, [_P]),
    "kkm_fit_restarts": (_I32, [_P, _I64, _I64, _I32, _I32, _F64, ctypes.POINTER(kkm_kernel), _I32, _U64, _I32,
                                ctypes.POINTER(kkm_options), _P, ctypes.POINTER(_P), _P, ctypes.POINTER(_I32)]),
    "kkm_elbow": (_I32, [_P, _I64, _I64, _I32, _I32, _I32, _F64, ctypes.POINTER(kkm_kernel), _I32, _U64, _I32,
                         ctypes.POINTER(kkm_options), _P, ctypes.POINTER(_I32)]),
    "kkm_model_displacement": (_I32, [_P, _P, _I32, ctypes.POINTER(_I32)]),
    "kkm_server_create": (_I32, [ctypes.POINTER(kkm_server_config), ctypes.POINTER(_P)]),
    "kkm_server_destroy": (None, [_P]),
    "kkm_server_add_model": (_I32, [_P, _P, ctypes.POINTER(_I32)]),
    "kkm_server_remove_model": (_I32, [_P, _I32]),
    "kkm_server_submit_fit": (_I32, [_P, _P, _I32, ctypes.POINTER(_U64)]),
    "kkm_server_submit_assign": (_I32, [_P, _I32, _P, _I64, _I32, _P, _P, ctypes.POINTER(_U64)]),
    "kkm_server_wait": (_I32, [_P, _U64, _I32, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "kkm_server_stats": (_I32, [_P, ctypes.POINTER(kkm_serving_stats)]),
    "kkm_server_reset_stats": (_I32, [_P]),
    "kkm_assign": (_I32, [_P, _P, _I64, _I32, _P, _P, _P]),
    "kkm_cost": (_I32, [_P, _P, _I64, _I32, ctypes.POINTER(_F64), _P]),
    "kkm_model_info": (_I32, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I64), ctypes.POINTER(_I32),
                              ctypes.POINTER(_F32)]),
    "kkm_model_medoids": (_I32, [_P, _P, _P, _P]),
    "kkm_model_supports": (_I32, [_P, _P, _P, _P]),
    "kkm_model_trace": (_I32, [_P, _P, _P, _I32, ctypes.POINTER(_I32)]),
    "kkm_model_free": (None, [_P]),
    "kkm_model_save": (_I32, [_P, ctypes.c_char_p]),
    "kkm_model_load": (_I32, [ctypes.c_char_p, ctypes.POINTER(_P)]),
    "kkm_kernel_matrix": (_I32, [_P, _I64, _P, _I64, _I64, ctypes.POINTER(kkm_kernel), _I32, _P, _P]),
    "kkm_median_bandwidth": (_I32, [_P, _I64, _I64, ctypes.POINTER(kkm_kernel), _U64,
                                    ctypes.POINTER(_F32)]),
    "kkm_debug_step": (_I32, [_P, _I64, _I64, _P, _I32, ctypes.POINTER(kkm_kernel), _I32, _I32, _I32, _P, _P,
                              _P, _P, _P, _P, ctypes.POINTER(_F64), ctypes.POINTER(_I32), _P]),
    "kkm_debug_kmeanspp": (_I32, [_P, _I64, _I64, ctypes.POINTER(kkm_kernel), _I32, _U64, _P, _P]),
    "kkm_minibatch_plan": (_I32, [_I64, _I32, _I32, _F64, _U64, _I32, ctypes.POINTER(_I64),
                                  ctypes.POINTER(_I64), ctypes.POINTER(_I64), _P, ctypes.POINTER(_I64)]),
    "kkm_assign_noalloc": (_I32, [_P, _P, _I64, _I32, _P, _P, _P]),
    "kkm_status_string": (ctypes.c_char_p, [_I32]),
    "kkm_last_error": (ctypes.c_char_p, []),
    "kkm_prof_enable": (None, [_I32]),
    "kkm_prof_reset": (None, []),
    "kkm_prof_read": (_I32, [ctypes.c_char_p, ctypes.POINTER(_I64), ctypes.POINTER(_F64)]),
    "kkm_prof_work": (_F64, [ctypes.c_char_p]),
    "kkm_prof_names": (_I32, [ctypes.c_char_p, _I32]),
}


def load():
    """Loads libkkm.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_1710_03013_gb300.build")
        lib = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def status_string(s):
    return load().kkm_status_string(s).decode()


def last_error():
    return load().kkm_last_error().decode()


def _check(status):
    if status != 0:
        raise KKMError(status, last_error())


# ------------------------------------------------------------ marshalling
def _torch():
    import torch
    return torch


def _is_cuda(x):
    return hasattr(x, "is_cuda") and x.is_cuda


def _as_input(x, dtype):
    """(pointer, keep-alive object) of a C-contiguous input of `dtype`."""
    if hasattr(x, "data_ptr"):
        torch = _torch()
        tdt = {np.float32: torch.float32, np.int32: torch.int32, np.int64: torch.int64}[dtype]
        t = x.to(tdt).contiguous()
        return ctypes.c_void_p(t.data_ptr()), t
    a = np.ascontiguousarray(x, dtype=dtype)
    return ctypes.c_void_p(a.ctypes.data), a


def _stream_of(x):
    if _is_cuda(x):
        torch = _torch()
        return ctypes.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)
    return ctypes.c_void_p(0)


def _out_like(x, n, dtype):
    """Output buffer on the same side as x: CUDA tensor or numpy array."""
    if _is_cuda(x):
        torch = _torch()
        tdt = {np.float32: torch.float32, np.int32: torch.int32}[dtype]
        t = torch.empty(n, dtype=tdt, device=x.device)
        return ctypes.c_void_p(t.data_ptr()), t
    a = np.empty(n, dtype=dtype)
    return ctypes.c_void_p(a.ctypes.data), a


def _kernel(kind, sigma, n_atoms):
    k = KIND[kind] if isinstance(kind, str) else int(kind)
    return kkm_kernel(k, float(sigma), int(n_atoms))


# ----------------------------------------------------------------- model
class Model:
    """A fitted model (owns the C handle)."""

    def __init__(self, handle):
        self._h = handle

    @property
    def handle(self):
        return self._h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.kkm_model_free(self._h)
            self._h = None

    def release(self):
        """Gives up ownership of the C handle (e.g. to a server) and returns it."""
        h, self._h = self._h, None
        return h

    def info(self):
        C, d, nL, sig = _I32(), _I64(), _I32(), _F32()
        _check(load().kkm_model_info(self._h, ctypes.byref(C), ctypes.byref(d), ctypes.byref(nL),
                                     ctypes.byref(sig)))
        return {"C": C.value, "d": d.value, "n_support": nL.value, "sigma": sig.value}

    def medoids(self):
        inf = self.info()
        idx = np.empty(inf["C"], np.int64)
        cnt = np.empty(inf["C"], np.int64)
        coords = np.empty((inf["C"], inf["d"]), np.float32)
        _check(load().kkm_model_medoids(self._h, idx.ctypes.data, cnt.ctypes.data, coords.ctypes.data))
        return idx, cnt, coords

    def supports(self):
        inf = self.info()
        lab = np.empty(inf["n_support"], np.int32)
        gh = np.empty(inf["C"], np.float64)
        n = np.empty(inf["C"], np.int32)
        _check(load().kkm_model_supports(self._h, lab.ctypes.data, gh.ctypes.data, n.ctypes.data))
        return lab, gh, n

    def save(self, path):
        """kkm_model_save of the C ABI."""
        _check(load().kkm_model_save(self._h, os.fsencode(path)))

    @staticmethod
    def load(path):
        """kkm_model_load of the C ABI: a new Model on the current device."""
        h = ctypes.c_void_p()
        _check(load().kkm_model_load(os.fsencode(path), ctypes.byref(h)))
        return Model(h)

    def displacement(self):
        """kkm_model_displacement of the C ABI: the average centre
        displacement of every mini-batch (Section 4.1, Fig. 4b)."""
        n = _I32()
        _check(load().kkm_model_displacement(self._h, None, 0, ctypes.byref(n)))
        out = np.empty(n.value, np.float64)
        _check(load().kkm_model_displacement(self._h, out.ctypes.data, n.value, ctypes.byref(n)))
        return out

    def trace(self):
        n = _I32()
        _check(load().kkm_model_trace(self._h, None, None, 0, ctypes.byref(n)))
        om = np.empty(n.value, np.float64)
        ch = np.empty(n.value, np.int32)
        _check(load().kkm_model_trace(self._h, om.ctypes.data, ch.ctypes.data, n.value, ctypes.byref(n)))
        return om, ch


# ------------------------------------------------------------- functions
def kkm_fit(X, C, B, s, kind="rbf", sigma=0.0, n_atoms=0, iters=20, seed=0, *,
            precision=KKM_FP32, sampling="stride", early_stop=True, init_medoids=None,
            labels=True, stream=None, pipeline="auto", iteration="auto"):
    """kkm_fit of the C ABI.  Returns (labels or None, Model)."""
    lib = load()
    N, d = int(X.shape[0]), int(np.prod(X.shape[1:]))
    xp, keep = _as_input(X, np.float32)
    k = _kernel(kind, sigma, n_atoms)
    opt = kkm_options()
    lib.kkm_options_default(ctypes.byref(opt))
    opt.precision = int(precision)
    opt.sampling = SAMPLING[sampling] if isinstance(sampling, str) else int(sampling)
    opt.early_stop = 1 if early_stop else 0
    opt.pipeline = PIPELINE[pipeline] if isinstance(pipeline, str) else int(pipeline)
    opt.iteration = ITERATION[iteration] if isinstance(iteration, str) else int(iteration)
    init_arr = None
    if init_medoids is not None:
        init_arr = np.ascontiguousarray(init_medoids, dtype=np.int64)
        opt.init_medoids = init_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    opt.stream = stream if stream is not None else _stream_of(X)
    lab_p, lab = _out_like(X, N, np.int32) if labels else (None, None)
    h = ctypes.c_void_p()
    _check(lib.kkm_fit(xp, N, d, int(C), int(B), float(s), ctypes.byref(k), int(iters),
                       int(seed) & ((1 << 64) - 1), ctypes.byref(opt), lab_p, ctypes.byref(h)))
    del keep, init_arr
    return lab, Model(h)


class Checkpoint:
    """The state of a fit between two mini-batches (owns the C handle)."""

    def __init__(self, handle):
        self._h = handle

    @property
    def handle(self):
        return self._h

    def __del__(self):
        if getattr(self, "_h", None) and _lib is not None:
            _lib.kkm_checkpoint_free(self._h)
            self._h = None

    def info(self):
        nb, B, C, sig = _I32(), _I32(), _I32(), _F32()
        _check(load().kkm_checkpoint_info(self._h, ctypes.byref(nb), ctypes.byref(B), ctypes.byref(C),
                                          ctypes.byref(sig), None))
        return {"next_batch": nb.value, "B": B.value, "C": C.value, "sigma": sig.value}

    def medoids(self):
        """The global medoids (sample indices) after the last mini-batch run."""
        med = np.empty(self.info()["C"], np.int64)
        _check(load().kkm_checkpoint_info(self._h, None, None, None, None, med.ctypes.data))
        return med

    def save(self, path):
        """kkm_checkpoint_save of the C ABI."""
        _check(load().kkm_checkpoint_save(self._h, os.fsencode(path)))

    @staticmethod
    def load(path):
        """kkm_checkpoint_load of the C ABI."""
        h = ctypes.c_void_p()
        _check(load().kkm_checkpoint_load(os.fsencode(path), ctypes.byref(h)))
        return Checkpoint(h)


def kkm_fit_range(X, C, B, s, kind="rbf", sigma=0.0, n_atoms=0, iters=20, seed=0, *, stop,
                  checkpoint=None, precision=KKM_FP32, sampling="stride", early_stop=True, init_medoids=None,
                  labels=True, model=False, stream=None, pipeline="auto", iteration="auto"):
    """kkm_fit_range of the C ABI: the mini-batches [start, stop), start = 0
    or the checkpoint's next mini-batch.  `labels` is True (a new [N] buffer,
    -1 in rows outside the range), an existing int32 buffer to continue, or
    False.  Returns (labels or None, Model or None, Checkpoint)."""
    lib = load()
    N, d = int(X.shape[0]), int(np.prod(X.shape[1:]))
    xp, keep = _as_input(X, np.float32)
    k = _kernel(kind, sigma, n_atoms)
    st = stream if stream is not None else _stream_of(X)
    opt = _options(precision, sampling, early_stop, pipeline, iteration, st)
    init_arr = None
    if init_medoids is not None:
        init_arr = np.ascontiguousarray(init_medoids, dtype=np.int64)
        opt.init_medoids = init_arr.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    if labels is True:
        lp, lab = _out_like(X, N, np.int32)
        lab[:] = -1
    elif labels is False or labels is None:
        lp, lab = None, None
    else:
        lab = labels
        is_int32 = lab.dtype == (_torch().int32 if hasattr(lab, "data_ptr") else np.int32)
        if not is_int32 or int(np.prod(lab.shape)) != N:
            raise ValueError("labels must be an int32 buffer of N entries")
        if hasattr(lab, "data_ptr"):
            if not lab.is_contiguous():
                raise ValueError("labels must be contiguous")
            lp = ctypes.c_void_p(lab.data_ptr())
        else:
            if not lab.flags["C_CONTIGUOUS"]:
                raise ValueError("labels must be contiguous")
            lp = ctypes.c_void_p(lab.ctypes.data)
    h = ctypes.c_void_p()
    ck = ctypes.c_void_p()
    _check(lib.kkm_fit_range(xp, N, d, int(C), int(B), float(s), ctypes.byref(k), int(iters),
                             int(seed) & ((1 << 64) - 1), ctypes.byref(opt),
                             checkpoint.handle if checkpoint is not None else None, int(stop), lp,
                             ctypes.byref(h) if model else None, ctypes.byref(ck)))
    del keep, init_arr
    return lab, (Model(h) if model else None), Checkpoint(ck)


def _options(precision, sampling, early_stop, pipeline, iteration, stream):
    opt = kkm_options()
    load().kkm_options_default(ctypes.byref(opt))
    opt.precision = int(precision)
    opt.sampling = SAMPLING[sampling] if isinstance(sampling, str) else int(sampling)
    opt.early_stop = int(bool(early_stop))
    opt.pipeline = PIPELINE[pipeline] if isinstance(pipeline, str) else int(pipeline)
    opt.iteration = ITERATION[iteration] if isinstance(iteration, str) else int(iteration)
    opt.stream = stream
    return opt


def kkm_fit_restarts(X, C, B, s, kind="rbf", sigma=0.0, n_atoms=0, iters=20, seed=0, n_restarts=5, *,
                     precision=KKM_FP32, sampling="stride", early_stop=True, labels=True, stream=None,
                     pipeline="auto", iteration="auto"):
    """kkm_fit_restarts of the C ABI.  Returns (labels or None, Model of the
    best restart, every restart's cost, the best restart's index)."""
    lib = load()
    N, d = int(X.shape[0]), int(np.prod(X.shape[1:]))
    xp, keep = _as_input(X, np.float32)
    k = _kernel(kind, sigma, n_atoms)
    st = stream if stream is not None else _stream_of(X)
    opt = _options(precision, sampling, early_stop, pipeline, iteration, st)
    lp, lab = _out_like(X, N, np.int32) if labels else (None, None)
    costs = np.empty(int(n_restarts), np.float64)
    best = _I32()
    h = ctypes.c_void_p()
    _check(lib.kkm_fit_restarts(xp, N, d, int(C), int(B), float(s), ctypes.byref(k), int(iters),
                                int(seed) & ((1 << 64) - 1), int(n_restarts), ctypes.byref(opt), lp,
                                ctypes.byref(h), costs.ctypes.data, ctypes.byref(best)))
    del keep
    return lab, Model(h), costs, best.value


def kkm_elbow(X, C_lo, C_hi, B, s, kind="rbf", sigma=0.0, n_atoms=0, iters=20, seed=0, n_restarts=1, *,
              precision=KKM_FP32, sampling="stride", early_stop=True, stream=None, pipeline="auto",
              iteration="auto"):
    """kkm_elbow of the C ABI.  Returns (the minimum cost of every C in
    [C_lo, C_hi], the elbow C)."""
    lib = load()
    N, d = int(X.shape[0]), int(np.prod(X.shape[1:]))
    xp, keep = _as_input(X, np.float32)
    k = _kernel(kind, sigma, n_atoms)
    st = stream if stream is not None else _stream_of(X)
    opt = _options(precision, sampling, early_stop, pipeline, iteration, st)
    costs = np.empty(int(C_hi) - int(C_lo) + 1, np.float64)
    c_out = _I32()
    _check(lib.kkm_elbow(xp, N, d, int(C_lo), int(C_hi), int(B), float(s), ctypes.byref(k), int(iters),
                         int(seed) & ((1 << 64) - 1), int(n_restarts), ctypes.byref(opt), costs.ctypes.data,
                         ctypes.byref(c_out)))
    del keep
    return costs, c_out.value


def kkm_fit_batch(problems, n_streams=0, stream=None, check=True):
    """kkm_fit_batch of the C ABI.  `problems` is a list of dicts with the
    kkm_fit arguments (X, C, B, s and optionally kind, sigma, n_atoms, iters,
    seed, precision, sampling, early_stop, init_medoids, labels, pipeline, iteration).  Returns a
    list of (labels or None, Model or None, status) in problem order; with
    check=True a failed problem raises KKMError instead."""
    lib = load()
    n = len(problems)
    arr = (kkm_problem * max(n, 1))()
    keep, outs = [], []
    for i, p in enumerate(problems):
        outs.append(_fill_problem(arr[i], p, keep))
    models = (ctypes.c_void_p * max(n, 1))()
    status = (ctypes.c_int32 * max(n, 1))()
    if stream is None:
        stream = _stream_of(problems[0]["X"]) if n else ctypes.c_void_p(0)
    rc = lib.kkm_fit_batch(arr, n, int(n_streams), models, status, stream)
    if check:
        _check(rc)
    del keep
    return [(outs[i], Model(ctypes.c_void_p(models[i])) if models[i] else None, status[i]) for i in range(n)]


def _fill_problem(q, p, keep):
    """Fills a kkm_problem from a dict; returns the labels buffer (or None)."""
    lib = load()
    X = p["X"]
    xp, kx = _as_input(X, np.float32)
    keep.append(kx)
    q.X = xp
    q.N = int(X.shape[0])
    q.d = int(np.prod(X.shape[1:]))
    q.C, q.B, q.s = int(p["C"]), int(p["B"]), float(p["s"])
    q.kernel = _kernel(p.get("kind", "rbf"), p.get("sigma", 0.0), p.get("n_atoms", 0))
    q.iters = int(p.get("iters", 20))
    q.seed = int(p.get("seed", 0)) & ((1 << 64) - 1)
    lib.kkm_options_default(ctypes.byref(q.opt))
    q.opt.precision = int(p.get("precision", KKM_FP32))
    smp = p.get("sampling", "stride")
    q.opt.sampling = SAMPLING[smp] if isinstance(smp, str) else int(smp)
    q.opt.early_stop = 1 if p.get("early_stop", True) else 0
    pl = p.get("pipeline", "auto")
    q.opt.pipeline = PIPELINE[pl] if isinstance(pl, str) else int(pl)
    it = p.get("iteration", "auto")
    q.opt.iteration = ITERATION[it] if isinstance(it, str) else int(it)
    if p.get("init_medoids") is not None:
        ia = np.ascontiguousarray(p["init_medoids"], dtype=np.int64)
        keep.append(ia)
        q.opt.init_medoids = ia.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))
    if p.get("labels", True):
        lp, lab = _out_like(X, q.N, np.int32)
        q.labels_out = lp
        keep.append(lab)
    else:
        lab = None
    return lab


class Server:
    """kkm_server of the C ABI: a request loop for fit and assign jobs.

    submit_fit / submit_assign return a ticket; wait(ticket) returns the
    job's outputs.  Inputs may be host arrays or CUDA tensors and must not be
    modified before the job is collected."""

    def __init__(self, budget_bytes, n_workers=0, max_batch_rows=0):
        lib = load()
        cfg = kkm_server_config(int(budget_bytes), int(n_workers), 0, int(max_batch_rows))
        h = ctypes.c_void_p()
        _check(lib.kkm_server_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._pending = {}

    def close(self):
        if getattr(self, "_h", None):
            load().kkm_server_destroy(self._h)
            self._h = None

    def __del__(self):
        if _lib is not None:
            self.close()

    def add_model(self, model):
        mid = _I32()
        _check(load().kkm_server_add_model(self._h, model.handle, ctypes.byref(mid)))
        model.release()
        return mid.value

    def remove_model(self, model_id):
        _check(load().kkm_server_remove_model(self._h, int(model_id)))

    def submit_fit(self, problem, keep_model=False):
        keep = []
        q = kkm_problem()
        lab = _fill_problem(q, problem, keep)
        t = _U64()
        _check(load().kkm_server_submit_fit(self._h, ctypes.byref(q), 1 if keep_model else 0, ctypes.byref(t)))
        self._pending[t.value] = (keep, lab)
        return t.value

    def submit_assign(self, model_id, X, mode="supports"):
        M = int(X.shape[0])
        xp, kx = _as_input(X, np.float32)
        lp, lab = _out_like(X, M, np.int32)
        dp, dist = _out_like(X, M, np.float32)
        t = _U64()
        _check(load().kkm_server_submit_assign(self._h, int(model_id), xp, M,
                                               MODE[mode] if isinstance(mode, str) else int(mode), lp, dp,
                                               ctypes.byref(t)))
        self._pending[t.value] = ([kx, lab, dist], (lab, dist))
        return t.value

    def wait(self, ticket, timeout_ms=-1):
        """Returns (status, outputs, model id): outputs are the labels of a
        fit, or (labels, squared distances) of an assign.  Raises KKMError
        with KKM_ETIMEOUT if the job is not done within timeout_ms."""
        st, mid = _I32(), _I32()
        _check(load().kkm_server_wait(self._h, int(ticket), int(timeout_ms), ctypes.byref(st), ctypes.byref(mid)))
        err = last_error() if st.value != 0 else ""
        keep, out = self._pending.pop(ticket)
        return st.value, out, mid.value, err

    def stats(self):
        s = kkm_serving_stats()
        _check(load().kkm_server_stats(self._h, ctypes.byref(s)))
        return {k: getattr(s, k) for k, _ in kkm_serving_stats._fields_}

    def reset_stats(self):
        _check(load().kkm_server_reset_stats(self._h))


def kkm_assign(model, Xnew, mode="supports", stream=None):
    """kkm_assign of the C ABI.  Returns (labels, squared distances)."""
    lib = load()
    M = int(Xnew.shape[0])
    xp, keep = _as_input(Xnew, np.float32)
    lab_p, lab = _out_like(Xnew, M, np.int32)
    dist_p, dist = _out_like(Xnew, M, np.float32)
    st = stream if stream is not None else _stream_of(Xnew)
    _check(lib.kkm_assign(model.handle, xp, M, MODE[mode] if isinstance(mode, str) else int(mode),
                          lab_p, dist_p, st))
    del keep
    return lab, dist


def _check_noalloc_args(d, Xnew, labels_out, dist_out):
    """Argument checks of kkm_assign_noalloc.  The C entry point receives bare
    device pointers and no row length, so it cannot see a wrong dtype, a
    strided view, a short output or a tensor on another device; a wrong one
    would be read or written past its end.  Raises ValueError."""
    torch = _torch()
    if not _is_cuda(Xnew):
        raise ValueError("kkm_assign_noalloc: Xnew must be a CUDA tensor")
    if Xnew.dtype != torch.float32 or not Xnew.is_contiguous():
        raise ValueError("kkm_assign_noalloc: Xnew must be contiguous float32")
    if Xnew.dim() < 2 or int(np.prod(Xnew.shape[1:])) != d:
        raise ValueError(f"kkm_assign_noalloc: Xnew must be [M][{d}] (rows of the model's length)")
    M = int(Xnew.shape[0])
    outs = [("labels_out", labels_out, torch.int32)]
    if dist_out is not None:
        outs.append(("dist_out", dist_out, torch.float32))
    for name, t, dt in outs:
        if not _is_cuda(t) or t.dtype != dt or not t.is_contiguous():
            raise ValueError(f"kkm_assign_noalloc: {name} must be a contiguous CUDA {dt} tensor")
        if t.numel() < M:
            raise ValueError(f"kkm_assign_noalloc: {name} holds {t.numel()} elements, needs {M}")
        if t.device != Xnew.device:
            raise ValueError(f"kkm_assign_noalloc: {name} is on {t.device}, Xnew on {Xnew.device}")
    return M


def kkm_assign_noalloc(model, Xnew, labels_out, dist_out=None, mode="supports", stream=None):
    """kkm_assign_noalloc of the C ABI: labels (and squared distances) of at
    most KKM_NOALLOC_MAX_ROWS new samples written into the caller's CUDA
    tensors; neither this function nor the library allocates.  Xnew is a
    contiguous float32 CUDA tensor [M][d] (d the model's row length),
    labels_out an int32 and dist_out (optional) a float32 CUDA tensor of at
    least M elements, all on the model's device."""
    lib = load()
    M = _check_noalloc_args(model.info()["d"], Xnew, labels_out, dist_out)
    st = stream if stream is not None else _stream_of(Xnew)
    _check(lib.kkm_assign_noalloc(model.handle, ctypes.c_void_p(Xnew.data_ptr()), M,
                                  MODE[mode] if isinstance(mode, str) else int(mode),
                                  ctypes.c_void_p(labels_out.data_ptr()),
                                  ctypes.c_void_p(dist_out.data_ptr()) if dist_out is not None else None,
                                  st))


def kkm_cost(model, X, mode="supports", stream=None):
    """kkm_cost of the C ABI (Eq. 1, FP64)."""
    lib = load()
    N = int(X.shape[0])
    xp, keep = _as_input(X, np.float32)
    out = _F64()
    st = stream if stream is not None else _stream_of(X)
    _check(lib.kkm_cost(model.handle, xp, N, MODE[mode] if isinstance(mode, str) else int(mode),
                        ctypes.byref(out), st))
    del keep
    return out.value


def kkm_kernel_matrix(A, B, kind="rbf", sigma=1.0, n_atoms=0, precision=KKM_FP32, stream=None):
    """kkm_kernel_matrix of the C ABI: K(A, B) as [len(A)][len(B)] float32."""
    lib = load()
    nA, nB = int(A.shape[0]), int(B.shape[0])
    d = int(np.prod(A.shape[1:]))
    ap, ka = _as_input(A, np.float32)
    bp, kb = _as_input(B, np.float32)
    if _is_cuda(A):
        torch = _torch()
        out = torch.empty((nA, nB), dtype=torch.float32, device=A.device)
        op = ctypes.c_void_p(out.data_ptr())
    else:
        out = np.empty((nA, nB), np.float32)
        op = ctypes.c_void_p(out.ctypes.data)
    k = _kernel(kind, sigma, n_atoms)
    st = stream if stream is not None else _stream_of(A)
    _check(lib.kkm_kernel_matrix(ap, nA, bp, nB, d, ctypes.byref(k), int(precision), op, st))
    del ka, kb
    return out


def kkm_median_bandwidth(X, kind="rbf", n_atoms=0, seed=0):
    lib = load()
    N, d = int(X.shape[0]), int(np.prod(X.shape[1:]))
    xp, keep = _as_input(X, np.float32)
    k = _kernel(kind, 0.0, n_atoms)
    out = _F32()
    _check(lib.kkm_median_bandwidth(xp, N, d, ctypes.byref(k), int(seed) & ((1 << 64) - 1),
                                    ctypes.byref(out)))
    del keep
    return out.value


def kkm_debug_step(Xb, L, u, C, kind="rbf", sigma=1.0, n_atoms=0, stream=None, precision=KKM_FP32,
                   iteration="auto"):
    """kkm_debug_step of the C ABI: one teacher-forced inner iteration."""
    lib = load()
    Ni, d = int(Xb.shape[0]), int(np.prod(Xb.shape[1:]))
    xp, keep = _as_input(Xb, np.float32)
    L = np.ascontiguousarray(L, np.int32)
    u = np.ascontiguousarray(u, np.int32)
    out = {"u": np.empty(Ni, np.int32), "fhat": np.empty((Ni, C), np.float32),
           "margin": np.empty(Ni, np.float32), "ghat": np.empty(C, np.float64),
           "n": np.empty(C, np.int32)}
    om, ch = _F64(), _I32()
    k = _kernel(kind, sigma, n_atoms)
    st = stream if stream is not None else _stream_of(Xb)
    it = ITERATION[iteration] if isinstance(iteration, str) else int(iteration)
    _check(lib.kkm_debug_step(xp, Ni, d, L.ctypes.data, len(L), ctypes.byref(k), int(C), int(precision), it,
                              u.ctypes.data,
                              out["u"].ctypes.data, out["fhat"].ctypes.data, out["margin"].ctypes.data,
                              out["ghat"].ctypes.data, out["n"].ctypes.data, ctypes.byref(om),
                              ctypes.byref(ch), st))
    out["omega"] = om.value
    out["changed"] = ch.value
    del keep
    return out


def kkm_debug_kmeanspp(X0, C, seed, kind="rbf", sigma=1.0, n_atoms=0, stream=None):
    lib = load()
    N0, d = int(X0.shape[0]), int(np.prod(X0.shape[1:]))
    xp, keep = _as_input(X0, np.float32)
    picks = np.empty(C, np.int64)
    k = _kernel(kind, sigma, n_atoms)
    st = stream if stream is not None else _stream_of(X0)
    _check(lib.kkm_debug_kmeanspp(xp, N0, d, ctypes.byref(k), int(C), int(seed) & ((1 << 64) - 1),
                                  picks.ctypes.data, st))
    del keep
    return picks


def kkm_minibatch_plan(N, B, s, seed, batch, sampling="stride"):
    """Host-only: (global indices of mini-batch `batch`, its sorted landmarks)."""
    lib = load()
    smp = SAMPLING[sampling] if isinstance(sampling, str) else int(sampling)
    start, step, n, nl = _I64(), _I64(), _I64(), _I64()
    args = (int(N), int(B), smp, float(s), int(seed) & ((1 << 64) - 1), int(batch))
    _check(lib.kkm_minibatch_plan(*args, ctypes.byref(start), ctypes.byref(step), ctypes.byref(n), None,
                                  ctypes.byref(nl)))
    L = np.empty(nl.value, np.int32)
    _check(lib.kkm_minibatch_plan(*args, ctypes.byref(start), ctypes.byref(step), ctypes.byref(n),
                                  L.ctypes.data, ctypes.byref(nl)))
    gidx = start.value + step.value * np.arange(n.value, dtype=np.int64)
    return gidx, L


# ------------------------------------------------------------- profiling
def prof_enable(on=True):
    """True/1: time every launch; 2: count every launch, time the heavy kernels."""
    load().kkm_prof_enable(int(on) if not isinstance(on, bool) else (1 if on else 0))


def prof_reset():
    load().kkm_prof_reset()


def prof_read(name):
    n, ms = _I64(), _F64()
    load().kkm_prof_read(name.encode(), ctypes.byref(n), ctypes.byref(ms))
    return n.value, ms.value


def prof_work(name):
    """Work units a data-dependent kernel reported while profiling was on."""
    return load().kkm_prof_work(name.encode())


def prof_names():
    lib = load()
    size = lib.kkm_prof_names(None, 0)
    buf = ctypes.create_string_buffer(size + 1)
    lib.kkm_prof_names(buf, size + 1)
    return [s for s in buf.value.decode().split(",") if s]
