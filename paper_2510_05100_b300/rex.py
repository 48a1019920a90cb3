"""Python binding of the C ABI in include/rex.h (argument marshalling only).

Every step of the computation runs in the CUDA kernels of librex_b300.so; this
module converts torch tensors / numpy arrays to pointers and error codes to
exceptions.  Importing it fails loudly when the shared library is missing:
there is no CPU fallback.

    import torch
    from paper_2510_05100_b300 import rex
    proc = rex.Process("gg_ttxg", precision=rex.FP64)
    proc.set_params(mt=173.0, alphas=0.118)
    w_out = proc.reweight(momenta_cuda, w_in_cuda, [dict(mt=171.0, alphas=0.118), ...])
"""
from __future__ import annotations

import ctypes
import os
from typing import Iterable, Sequence

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "librex_b300.so")
TOOLING_LIB_PATH = os.path.join(HERE, "librex_tooling_b300.so")
TOOLING_EXPORTS = ("rex_probe_fma", "rex_probe_convert")

REX_OK = 0
REX_EINVAL = -1
REX_ENOTINIT = -2
REX_ECUDA = -3
REX_ENOMEM = -4
REX_EUNSUPPORTED = -5
FP64 = 0
MIXED = 1
DF64 = 2          # double-float amplitudes (gg_ttx, gg_ttxg)
FLAG_NO_DEDUPE = 1
MULTI_PERSISTENT = 0
MULTI_STREAMS = 1
SURROGATE_FUSED = 0
SURROGATE_LAYERED = 1

# symbols declared in include/rex.h
EXPORTS = (
    "rex_init_process", "rex_process_npart", "rex_set_flags", "rex_set_params", "rex_reweight_helicity",
    "rex_reweight", "rex_reweight_host", "rex_me2", "rex_free_process",
    "rex_last_error", "rex_version", "rex_num_variants", "rex_get_variant",
    "rex_set_variant", "rex_autotune", "rex_multi_create", "rex_reweight_multi", "rex_multi_capture",
    "rex_multi_replay", "rex_multi_free", "rex_reweight_multi_noalloc", "rex_multi_set_mode",
    "rex_multi_set_slot_groups", "rex_multi_get_slot_groups", "rex_multi_autotune",
    "rex_multi_get_tile_cost", "rex_multi_set_tile_cost",
    "rex_surrogate_num_params", "rex_surrogate_last_error", "rex_surrogate_create",
    "rex_surrogate_set_weights", "rex_surrogate_get_weights", "rex_surrogate_loss_grad",
    "rex_surrogate_train", "rex_surrogate_reweight", "rex_surrogate_set_exact_alphas", "rex_surrogate_set_kernel",
    "rex_surrogate_set_guard", "rex_surrogate_calibrate",
    "rex_surrogate_save", "rex_surrogate_load",
    "rex_surrogate_free",
    "rex_xsec_last_error", "rex_xsec_create", "rex_xsec_reset", "rex_xsec_accumulate", "rex_xsec_result",
    "rex_xsec_free", "rex_xsec_get_state", "rex_xsec_set_state", "rex_xsec_merge_states",
    "rex_lhe_last_error", "rex_lhe_read", "rex_lhe_num_events", "rex_lhe_extract", "rex_lhe_extract_helicities", "rex_lhe_set_weights",
    "rex_lhe_write", "rex_lhe_free",
)


class RexError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"rex error {code}: {msg}")
        self.code = code


class Batch(ctypes.Structure):
    _fields_ = [("proc", ctypes.c_void_p), ("momenta", ctypes.c_void_p), ("w_in", ctypes.c_void_p),
                ("nev", ctypes.c_int64), ("w_out", ctypes.c_void_p)]


class Params(ctypes.Structure):
    _fields_ = [("mt", ctypes.c_double), ("wt", ctypes.c_double), ("alphas", ctypes.c_double),
                ("mz", ctypes.c_double), ("wz", ctypes.c_double), ("sw2", ctypes.c_double),
                ("alpha", ctypes.c_double)]


def params(d: dict) -> Params:
    return Params(d.get("mt", 0.0), d.get("wt", 0.0), d.get("alphas", 0.0),
                  d.get("mz", 0.0), d.get("wz", 0.0), d.get("sw2", 0.0), d.get("alpha", 0.0))


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load librex_b300.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_2510_05100_b300.build`")
    lib = ctypes.CDLL(path)
    vp, i64, dp = ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(ctypes.c_double)
    pp = ctypes.POINTER(Params)
    lib.rex_init_process.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(vp)]
    lib.rex_init_process.restype = ctypes.c_int
    lib.rex_process_npart.argtypes = [vp]
    lib.rex_process_npart.restype = ctypes.c_int
    lib.rex_set_flags.argtypes = [vp, ctypes.c_uint]
    lib.rex_set_flags.restype = ctypes.c_int
    lib.rex_set_params.argtypes = [vp, pp]
    lib.rex_set_params.restype = ctypes.c_int
    lib.rex_reweight.argtypes = [vp, vp, vp, i64, pp, ctypes.c_int, vp, vp]
    lib.rex_reweight.restype = ctypes.c_int
    lib.rex_reweight_helicity.argtypes = [vp, vp, vp, vp, i64, pp, ctypes.c_int, vp, vp]
    lib.rex_reweight_helicity.restype = ctypes.c_int
    lib.rex_reweight_host.argtypes = [vp, vp, vp, i64, pp, ctypes.c_int, vp, vp]
    lib.rex_reweight_host.restype = ctypes.c_int
    lib.rex_me2.argtypes = [vp, vp, i64, pp, vp, vp]
    lib.rex_me2.restype = ctypes.c_int
    lib.rex_free_process.argtypes = [vp]
    lib.rex_free_process.restype = None
    lib.rex_last_error.argtypes = []
    lib.rex_last_error.restype = ctypes.c_char_p
    lib.rex_num_variants.argtypes = [vp]
    lib.rex_num_variants.restype = ctypes.c_int
    lib.rex_get_variant.argtypes = [vp]
    lib.rex_get_variant.restype = ctypes.c_int
    lib.rex_set_variant.argtypes = [vp, ctypes.c_int]
    lib.rex_set_variant.restype = ctypes.c_int
    lib.rex_autotune.argtypes = [vp, vp, vp, i64, pp, ctypes.c_int, vp, vp, ctypes.POINTER(ctypes.c_float)]
    lib.rex_autotune.restype = ctypes.c_int
    bp = ctypes.POINTER(Batch)
    lib.rex_multi_create.argtypes = [ctypes.c_int, ctypes.POINTER(vp)]
    lib.rex_multi_create.restype = ctypes.c_int
    lib.rex_reweight_multi.argtypes = [vp, bp, ctypes.c_int, pp, ctypes.c_int, vp]
    lib.rex_reweight_multi.restype = ctypes.c_int
    lib.rex_multi_capture.argtypes = [vp, bp, ctypes.c_int, pp, ctypes.c_int]
    lib.rex_multi_capture.restype = ctypes.c_int
    lib.rex_multi_replay.argtypes = [vp, vp]
    lib.rex_multi_replay.restype = ctypes.c_int
    lib.rex_multi_free.argtypes = [vp]
    lib.rex_multi_free.restype = None
    lib.rex_multi_set_mode.argtypes = [vp, ctypes.c_int]
    lib.rex_multi_set_mode.restype = ctypes.c_int
    lib.rex_reweight_multi_noalloc.argtypes = [bp, ctypes.c_int, pp, ctypes.c_int, ctypes.c_int, vp]
    lib.rex_reweight_multi_noalloc.restype = ctypes.c_int
    lib.rex_multi_set_slot_groups.argtypes = [vp, ctypes.c_int]
    lib.rex_multi_set_slot_groups.restype = ctypes.c_int
    lib.rex_multi_get_slot_groups.argtypes = [vp]
    lib.rex_multi_get_slot_groups.restype = ctypes.c_int
    lib.rex_multi_autotune.argtypes = [vp, bp, ctypes.c_int, pp, ctypes.c_int, vp, ctypes.POINTER(ctypes.c_float)]
    lib.rex_multi_autotune.restype = ctypes.c_int
    lib.rex_multi_get_tile_cost.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_double)]
    lib.rex_multi_get_tile_cost.restype = ctypes.c_int
    lib.rex_multi_set_tile_cost.argtypes = [vp, vp, ctypes.c_double]
    lib.rex_multi_set_tile_cost.restype = ctypes.c_int
    fp = ctypes.POINTER(ctypes.c_float)
    lib.rex_surrogate_num_params.argtypes = []
    lib.rex_surrogate_num_params.restype = ctypes.c_int64
    lib.rex_surrogate_last_error.argtypes = []
    lib.rex_surrogate_last_error.restype = ctypes.c_char_p
    lib.rex_surrogate_create.argtypes = [ctypes.c_ulonglong, ctypes.POINTER(vp)]
    lib.rex_surrogate_create.restype = ctypes.c_int
    lib.rex_surrogate_set_weights.argtypes = [vp, vp, i64]
    lib.rex_surrogate_set_weights.restype = ctypes.c_int
    lib.rex_surrogate_get_weights.argtypes = [vp, vp, i64]
    lib.rex_surrogate_get_weights.restype = ctypes.c_int
    lib.rex_surrogate_loss_grad.argtypes = [vp, vp, vp, vp, vp, i64, fp, vp, vp]
    lib.rex_surrogate_loss_grad.restype = ctypes.c_int
    lib.rex_surrogate_train.argtypes = [vp, vp, vp, i64, pp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_float, ctypes.c_ulonglong, vp, vp]
    lib.rex_surrogate_train.restype = ctypes.c_int
    lib.rex_surrogate_reweight.argtypes = [vp, vp, vp, vp, i64, pp, ctypes.c_int, ctypes.c_float, vp, vp, vp,
                                           ctypes.POINTER(ctypes.c_int64), vp]
    lib.rex_surrogate_reweight.restype = ctypes.c_int
    lib.rex_surrogate_set_exact_alphas.argtypes = [vp, ctypes.c_double, ctypes.c_int]
    lib.rex_surrogate_set_exact_alphas.restype = ctypes.c_int
    lib.rex_surrogate_save.argtypes = [vp, ctypes.c_char_p]
    lib.rex_surrogate_save.restype = ctypes.c_int
    lib.rex_surrogate_load.argtypes = [vp, ctypes.c_char_p]
    lib.rex_surrogate_load.restype = ctypes.c_int
    lib.rex_surrogate_set_kernel.argtypes = [vp, ctypes.c_int]
    lib.rex_surrogate_set_kernel.restype = ctypes.c_int
    lib.rex_surrogate_set_guard.argtypes = [vp, ctypes.c_double]
    lib.rex_surrogate_set_guard.restype = ctypes.c_int
    lib.rex_surrogate_calibrate.argtypes = [vp, vp, vp, i64, pp, ctypes.c_int, ctypes.c_double, ctypes.c_double,
                                            fp, dp, dp, dp, vp]
    lib.rex_surrogate_calibrate.restype = ctypes.c_int
    lib.rex_xsec_last_error.argtypes = []
    lib.rex_xsec_last_error.restype = ctypes.c_char_p
    lib.rex_xsec_create.argtypes = [ctypes.c_int, ctypes.POINTER(vp)]
    lib.rex_xsec_create.restype = ctypes.c_int
    lib.rex_xsec_reset.argtypes = [vp, vp]
    lib.rex_xsec_reset.restype = ctypes.c_int
    lib.rex_xsec_accumulate.argtypes = [vp, vp, vp, i64, vp]
    lib.rex_xsec_accumulate.restype = ctypes.c_int
    lib.rex_xsec_result.argtypes = [vp, ctypes.c_double, ctypes.c_double, vp, vp, vp, vp]
    lib.rex_xsec_result.restype = ctypes.c_int
    lib.rex_lhe_last_error.argtypes = []
    lib.rex_lhe_last_error.restype = ctypes.c_char_p
    lib.rex_lhe_read.argtypes = [ctypes.c_char_p, ctypes.c_int, ctypes.POINTER(vp)]
    lib.rex_lhe_read.restype = ctypes.c_int
    lib.rex_lhe_num_events.argtypes = [vp]
    lib.rex_lhe_num_events.restype = i64
    lib.rex_lhe_extract.argtypes = [vp, vp, ctypes.c_int, vp, ctypes.c_int, ctypes.POINTER(i64), vp, vp, vp]
    lib.rex_lhe_extract.restype = ctypes.c_int
    lib.rex_lhe_extract_helicities.argtypes = [vp, vp, ctypes.c_int, vp, ctypes.c_int, ctypes.POINTER(i64), vp]
    lib.rex_lhe_extract_helicities.restype = ctypes.c_int
    lib.rex_lhe_set_weights.argtypes = [vp, ctypes.c_char_p, vp, vp, i64]
    lib.rex_lhe_set_weights.restype = ctypes.c_int
    lib.rex_lhe_write.argtypes = [vp, ctypes.c_char_p]
    lib.rex_lhe_write.restype = ctypes.c_int
    lib.rex_lhe_free.argtypes = [vp]
    lib.rex_lhe_free.restype = None
    lib.rex_xsec_get_state.argtypes = [vp, vp, vp]
    lib.rex_xsec_get_state.restype = ctypes.c_int
    lib.rex_xsec_set_state.argtypes = [vp, vp, vp]
    lib.rex_xsec_set_state.restype = ctypes.c_int
    lib.rex_xsec_merge_states.argtypes = [vp, vp, ctypes.c_int, vp]
    lib.rex_xsec_merge_states.restype = ctypes.c_int
    lib.rex_xsec_free.argtypes = [vp]
    lib.rex_xsec_free.restype = None
    lib.rex_surrogate_free.argtypes = [vp]
    lib.rex_surrogate_free.restype = None
    lib.rex_version.argtypes = []
    lib.rex_version.restype = ctypes.c_char_p
    _lib = lib
    return lib


def _check(rc: int) -> None:
    if rc != REX_OK:
        raise RexError(rc, load().rex_last_error().decode())


def _ptr(t) -> int:
    """Device or host address of a torch tensor / numpy array (contiguous float64)."""
    if t is None:
        return 0
    if hasattr(t, "data_ptr"):
        if not t.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return t.data_ptr()
    if not t.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return t.ctypes.data


def _stream_ptr(stream) -> int:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if hasattr(stream, "cuda_stream"):
        return stream.cuda_stream
    return int(stream)


def _param_array(points: Sequence[dict]):
    arr = (Params * max(1, len(points)))()
    for i, d in enumerate(points):
        arr[i] = params(d)
    return arr


class Process:
    """One subprocess handle (rex_init_process / rex_free_process)."""

    def __init__(self, name: str, precision: int = FP64):
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.rex_init_process(name.encode(), precision, ctypes.byref(h)))
        self._h = h
        self.name = name
        self.precision = precision
        self.npart = lib.rex_process_npart(h)

    def close(self):
        if getattr(self, "_h", None):
            load().rex_free_process(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_flags(self, flags: int) -> None:
        _check(load().rex_set_flags(self._h, flags))

    def set_params(self, point: dict | None = None, **kw) -> None:
        d = dict(point or {})
        d.update(kw)
        p = params(d)
        _check(load().rex_set_params(self._h, ctypes.byref(p)))

    def reweight(self, momenta, w_in, points: Sequence[dict], w_out=None, stream=None):
        """Device tensors in, device tensor [nev, k] out (enqueued on ``stream``)."""
        import torch
        nev = momenta.shape[0]
        k = len(points)
        if w_out is None:
            w_out = torch.empty((nev, k), dtype=torch.float64, device=momenta.device)
        arr = _param_array(points)
        _check(load().rex_reweight(self._h, _ptr(momenta), _ptr(w_in), nev, arr, k,
                                   _ptr(w_out), _stream_ptr(stream)))
        return w_out

    def reweight_helicity(self, momenta, helicities, w_in, points: Sequence[dict], w_out=None, stream=None):
        """Helicity-exclusive reweighting: helicities is a device int8 tensor [nev, npart] of
        +1/-1 (the events' own configurations); otherwise as reweight."""
        import torch
        nev = momenta.shape[0]
        k = len(points)
        if helicities.dtype != torch.int8 or not helicities.is_contiguous():
            raise ValueError("helicities must be a contiguous int8 tensor [nev, npart]")
        if w_out is None:
            w_out = torch.empty((nev, k), dtype=torch.float64, device=momenta.device)
        arr = _param_array(points)
        _check(load().rex_reweight_helicity(self._h, _ptr(momenta), _ptr(helicities), _ptr(w_in), nev, arr, k,
                                            _ptr(w_out), _stream_ptr(stream)))
        return w_out

    def reweight_host(self, momenta, w_in, points: Sequence[dict], w_out, stream=None) -> None:
        """Host arrays in and out (copies inside the call; blocks until w_out is written)."""
        arr = _param_array(points)
        _check(load().rex_reweight_host(self._h, _ptr(momenta), _ptr(w_in), momenta.shape[0], arr,
                                        len(points), _ptr(w_out), _stream_ptr(stream)))

    @property
    def num_variants(self) -> int:
        return load().rex_num_variants(self._h)

    @property
    def variant(self) -> int:
        return load().rex_get_variant(self._h)

    @variant.setter
    def variant(self, v: int) -> None:
        _check(load().rex_set_variant(self._h, v))

    def autotune(self, momenta, w_in, points: Sequence[dict], w_out, stream=None) -> list:
        """Time every kernel variant on these device buffers, keep the fastest; returns ms per variant."""
        n = max(1, self.num_variants)
        ms = (ctypes.c_float * n)()
        arr = _param_array(points)
        _check(load().rex_autotune(self._h, _ptr(momenta), _ptr(w_in), momenta.shape[0], arr, len(points),
                                   _ptr(w_out), _stream_ptr(stream), ms))
        return list(ms)

    def me2(self, momenta, point: dict, out=None, stream=None):
        import torch
        nev = momenta.shape[0]
        if out is None:
            out = torch.empty((nev,), dtype=torch.float64, device=momenta.device)
        p = params(point)
        _check(load().rex_me2(self._h, _ptr(momenta), nev, ctypes.byref(p), _ptr(out),
                              _stream_ptr(stream)))
        return out


class Multi:
    """Several subprocess batches in one persistent launch (rex_multi_*)."""

    def __init__(self, precision: int = FP64, mode: int = MULTI_PERSISTENT):
        h = ctypes.c_void_p()
        _check(load().rex_multi_create(precision, ctypes.byref(h)))
        self._h = h
        self.precision = precision
        if mode != MULTI_PERSISTENT:
            self.set_mode(mode)

    def set_mode(self, mode: int) -> None:
        _check(load().rex_multi_set_mode(self._h, mode))

    @property
    def slot_groups(self) -> int:
        return load().rex_multi_get_slot_groups(self._h)

    @slot_groups.setter
    def slot_groups(self, groups: int) -> None:
        _check(load().rex_multi_set_slot_groups(self._h, int(groups)))

    def tile_cost(self, proc) -> float:
        """rex_multi_get_tile_cost: measured microseconds of one tile of proc's kind (0: none)."""
        us = ctypes.c_double()
        _check(load().rex_multi_get_tile_cost(self._h, proc._h, ctypes.byref(us)))
        return us.value

    def set_tile_cost(self, proc, us: float) -> None:
        """rex_multi_set_tile_cost (0 clears the measured cost)."""
        _check(load().rex_multi_set_tile_cost(self._h, proc._h, float(us)))

    def autotune(self, batches, points: Sequence[dict], stream=None) -> list:
        """rex_multi_autotune: measure each tile kind's cost, then time 1, 2, 3, 4, 6, 8
        slot groups on these batches and keep the fastest; returns the mean ms per
        launch of each."""
        arr = self._batches(batches)
        ms = (ctypes.c_float * 6)()
        _check(load().rex_multi_autotune(self._h, arr, len(batches), _param_array(points), len(points),
                                         _stream_ptr(stream), ms))
        return list(ms)

    def close(self):
        if getattr(self, "_h", None):
            load().rex_multi_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _batches(batches):
        arr = (Batch * len(batches))()
        for i, (proc, mom, w_in, w_out) in enumerate(batches):
            arr[i] = Batch(proc._h.value if isinstance(proc._h, ctypes.c_void_p) else proc._h,
                           _ptr(mom), _ptr(w_in), mom.shape[0], _ptr(w_out))
        return arr

    def reweight(self, batches, points: Sequence[dict], stream=None) -> None:
        """batches: [(Process, momenta, w_in, w_out)] device tensors; enqueued on stream."""
        arr = self._batches(batches)
        _check(load().rex_reweight_multi(self._h, arr, len(batches), _param_array(points), len(points),
                                         _stream_ptr(stream)))

    def capture(self, batches, points: Sequence[dict]) -> None:
        arr = self._batches(batches)
        _check(load().rex_multi_capture(self._h, arr, len(batches), _param_array(points), len(points)))

    def replay(self, stream=None) -> None:
        _check(load().rex_multi_replay(self._h, _stream_ptr(stream)))


def reweight_multi_noalloc(batches, points: Sequence[dict], precision: int = FP64, stream=None) -> None:
    """rex_reweight_multi_noalloc: the multi-process launch without any library
    allocation, for callers that cannot allocate device memory (at most 64 points).

    batches: [(Process, momenta, w_in, w_out)] device tensors; enqueued on stream.
    """
    arr = Multi._batches(batches)
    _check(load().rex_reweight_multi_noalloc(arr, len(batches), _param_array(points), len(points),
                                             precision, _stream_ptr(stream)))


def _scheck(rc: int) -> None:
    if rc != REX_OK:
        raise RexError(rc, load().rex_surrogate_last_error().decode())


class Surrogate:
    """MLP surrogate of the log weight ratio (rex_surrogate_*); g g -> t t~ g events."""

    def __init__(self, seed: int = 0):
        h = ctypes.c_void_p()
        _scheck(load().rex_surrogate_create(seed, ctypes.byref(h)))
        self._h = h
        self.nparam = load().rex_surrogate_num_params()

    def close(self):
        if getattr(self, "_h", None):
            load().rex_surrogate_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_weights(self):
        import numpy as np
        out = np.empty(self.nparam, dtype=np.float32)
        _scheck(load().rex_surrogate_get_weights(self._h, out.ctypes.data, self.nparam))
        return out

    def set_weights(self, w) -> None:
        import numpy as np
        w = np.ascontiguousarray(w, dtype=np.float32)
        _scheck(load().rex_surrogate_set_weights(self._h, w.ctypes.data, w.size))

    def set_exact_alphas(self, alphas0: float, power: int) -> None:
        """Make the alphas^power dependence of |M|^2 exact; the network learns the rest."""
        _scheck(load().rex_surrogate_set_exact_alphas(self._h, float(alphas0), int(power)))

    def set_guard(self, y_min: float) -> None:
        """Always recompute exactly the events whose final-gluon invariant
        min_i 2 k.p_i / s_hat is below y_min (0 turns the guard off)."""
        _scheck(load().rex_surrogate_set_guard(self._h, float(y_min)))

    def calibrate(self, exact: "Process", momenta, points: Sequence[dict], bound: float, max_escape: float,
                  stream=None) -> dict:
        """rex_surrogate_calibrate on held-out device momenta: picks tau and the guard that keep
        the most events with at most max_escape of the kept pairs off by more than bound in
        log weight; sets the guard and returns {tau, guard, fallback_rate, escape_rate}."""
        tau = ctypes.c_float()
        guard, fb, esc = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        _scheck(load().rex_surrogate_calibrate(self._h, exact._h, _ptr(momenta), momenta.shape[0],
                                               _param_array(points), len(points), float(bound), float(max_escape),
                                               ctypes.byref(tau), ctypes.byref(guard), ctypes.byref(fb),
                                               ctypes.byref(esc), _stream_ptr(stream)))
        return {"tau": tau.value, "guard": guard.value, "fallback_rate": fb.value, "escape_rate": esc.value}

    def save(self, path: str) -> None:
        _scheck(load().rex_surrogate_save(self._h, os.fsencode(path)))

    def load(self, path: str) -> None:
        _scheck(load().rex_surrogate_load(self._h, os.fsencode(path)))

    def set_kernel(self, kind: int) -> None:
        """Inference kernel: SURROGATE_FUSED (tcgen05, default) or SURROGATE_LAYERED (mma.sync GEMMs)."""
        _scheck(load().rex_surrogate_set_kernel(self._h, int(kind)))

    def loss_grad(self, momenta, ratio, mt, alphas, stream=None):
        import numpy as np
        loss = ctypes.c_float()
        grad = np.empty(self.nparam, dtype=np.float32)
        _scheck(load().rex_surrogate_loss_grad(self._h, _ptr(momenta), _ptr(ratio), _ptr(mt), _ptr(alphas),
                                               momenta.shape[0], ctypes.byref(loss), grad.ctypes.data,
                                               _stream_ptr(stream)))
        return loss.value, grad

    def train(self, momenta, ratio, points, steps, batch=8192, lr=1e-3, seed=0, stream=None):
        import numpy as np
        losses = np.empty(max(1, steps), dtype=np.float32)
        _scheck(load().rex_surrogate_train(self._h, _ptr(momenta), _ptr(ratio), momenta.shape[0],
                                           _param_array(points), len(points), steps, batch, lr, seed,
                                           losses.ctypes.data, _stream_ptr(stream)))
        return losses[:steps]

    def reweight(self, momenta, w_in, points, tau=float("inf"), exact=None, w_out=None, pred=None, err=None,
                 stream=None) -> int:
        nfb = ctypes.c_int64(0)
        _scheck(load().rex_surrogate_reweight(self._h, exact._h if exact is not None else None, _ptr(momenta),
                                              _ptr(w_in), momenta.shape[0], _param_array(points), len(points),
                                              tau, _ptr(w_out), _ptr(pred), _ptr(err), ctypes.byref(nfb),
                                              _stream_ptr(stream)))
        return nfb.value


def _xcheck(rc: int) -> None:
    if rc != 0:
        raise RexError(rc, load().rex_xsec_last_error().decode())


class XSec:
    """Reweighted cross sections and errors (rex_xsec_*), accumulated over calls."""

    def __init__(self, k: int):
        h = ctypes.c_void_p()
        _xcheck(load().rex_xsec_create(int(k), ctypes.byref(h)))
        self._h = h
        self.k = int(k)

    def close(self):
        if getattr(self, "_h", None):
            load().rex_xsec_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def reset(self, stream=None) -> None:
        _xcheck(load().rex_xsec_reset(self._h, _stream_ptr(stream)))

    def accumulate(self, w_in, w_out, stream=None) -> None:
        _xcheck(load().rex_xsec_accumulate(self._h, _ptr(w_in), _ptr(w_out), w_in.shape[0], _stream_ptr(stream)))

    def get_state(self, stream=None):
        """The accumulated statistics, 5k + 3 doubles (see rex_xsec_get_state)."""
        import numpy as np
        st = np.empty(5 * self.k + 3)
        _xcheck(load().rex_xsec_get_state(self._h, st.ctypes.data, _stream_ptr(stream)))
        return st

    def set_state(self, state, stream=None) -> None:
        import numpy as np
        st = np.ascontiguousarray(state, dtype=np.float64)
        if st.size != 5 * self.k + 3:
            raise ValueError(f"state must hold {5 * self.k + 3} doubles")
        _xcheck(load().rex_xsec_set_state(self._h, st.ctypes.data, _stream_ptr(stream)))

    def result(self, sigma: float, dsigma: float, stream=None):
        """(sigma' [k], dsigma' [k], fallback [k] bool) as numpy arrays."""
        import numpy as np
        s = np.empty(self.k)
        ds = np.empty(self.k)
        fb = np.empty(self.k, dtype=np.int32)
        _xcheck(load().rex_xsec_result(self._h, float(sigma), float(dsigma), s.ctypes.data, ds.ctypes.data,
                                       fb.ctypes.data, _stream_ptr(stream)))
        return s, ds, fb.astype(bool)


def _lcheck(rc: int) -> None:
    if rc != 0:
        raise RexError(rc, load().rex_lhe_last_error().decode())


class Lhe:
    """An LHE v3 file: process extraction and weight writing (rex_lhe_*; host only)."""

    def __init__(self, path: str, nthreads: int = 0):
        h = ctypes.c_void_p()
        _lcheck(load().rex_lhe_read(os.fsencode(path), int(nthreads), ctypes.byref(h)))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().rex_lhe_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def num_events(self) -> int:
        return load().rex_lhe_num_events(self._h)

    def extract(self, pdg_in, pdg_out):
        """(momenta [n][npart][4] (E, px, py, pz), weights [n], file positions [n]) as numpy arrays."""
        import numpy as np
        a = np.ascontiguousarray(pdg_in, dtype=np.int32)
        b = np.ascontiguousarray(pdg_out, dtype=np.int32)
        n = ctypes.c_int64()
        _lcheck(load().rex_lhe_extract(self._h, a.ctypes.data, a.size, b.ctypes.data, b.size, ctypes.byref(n),
                                       None, None, None))
        mom = np.empty((n.value, a.size + b.size, 4))
        w = np.empty(n.value)
        idx = np.empty(n.value, dtype=np.int64)
        _lcheck(load().rex_lhe_extract(self._h, a.ctypes.data, a.size, b.ctypes.data, b.size, ctypes.byref(n),
                                       mom.ctypes.data, w.ctypes.data, idx.ctypes.data))
        return mom, w, idx

    def extract_helicities(self, pdg_in, pdg_out):
        """The SPINUP values of the same events and particle order as extract, int8 [n][npart]
        (+1 / -1 helicities, 9 unknown)."""
        import numpy as np
        a = np.ascontiguousarray(pdg_in, dtype=np.int32)
        b = np.ascontiguousarray(pdg_out, dtype=np.int32)
        n = ctypes.c_int64()
        _lcheck(load().rex_lhe_extract_helicities(self._h, a.ctypes.data, a.size, b.ctypes.data, b.size,
                                                  ctypes.byref(n), None))
        hel = np.empty((n.value, a.size + b.size), dtype=np.int8)
        _lcheck(load().rex_lhe_extract_helicities(self._h, a.ctypes.data, a.size, b.ctypes.data, b.size,
                                                  ctypes.byref(n), hel.ctypes.data))
        return hel

    def set_weights(self, wid: str, index, values) -> None:
        import numpy as np
        i = np.ascontiguousarray(index, dtype=np.int64)
        v = np.ascontiguousarray(values, dtype=np.float64)
        if i.size != v.size:
            raise ValueError("index and values differ in length")
        _lcheck(load().rex_lhe_set_weights(self._h, wid.encode(), i.ctypes.data, v.ctypes.data, i.size))

    def write(self, path: str) -> None:
        _lcheck(load().rex_lhe_write(self._h, os.fsencode(path)))


def xsec_merge_states(a, b, k: int):
    """State a merged with state b (host only; rex_xsec_merge_states)."""
    import numpy as np
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    out = np.empty_like(a)
    _xcheck(load().rex_xsec_merge_states(a.ctypes.data, b.ctypes.data, int(k), out.ctypes.data))
    return out


_tooling = None


def load_tooling(path: str = TOOLING_LIB_PATH) -> ctypes.CDLL:
    """Load librex_tooling_b300.so, the measurement and test probes (include/rex_tooling.h)."""
    global _tooling
    if _tooling is not None:
        return _tooling
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_2510_05100_b300.build`")
    lib = ctypes.CDLL(path)
    vp, i64 = ctypes.c_void_p, ctypes.c_int64
    lib.rex_probe_fma.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_double), vp]
    lib.rex_probe_fma.restype = ctypes.c_int
    lib.rex_probe_convert.argtypes = [vp, i64, vp, vp, vp, vp]
    lib.rex_probe_convert.restype = ctypes.c_int
    _tooling = lib
    return lib


def _tcheck(rc: int, what: str) -> None:
    if rc != 0:
        raise RexError(rc, f"{what} failed")


def probe_fma(fp64: bool, stream=None) -> float:
    """Measured FMA-pipe rate of the current device in flop/s (FP64 or FP32)."""
    out = ctypes.c_double()
    _tcheck(load_tooling().rex_probe_fma(1 if fp64 else 0, ctypes.byref(out), _stream_ptr(stream)), "rex_probe_fma")
    return out.value


def probe_convert(values, stream=None):
    """The integer-ALU FP64 -> FP32 -> FP64 conversions of the mixed q q~ -> t t~ kernel on a
    device FP64 tensor; returns (FP32, FP64 round trip, FP32 by the momentum conversion)."""
    import torch
    f32 = torch.empty(values.shape, dtype=torch.float32, device=values.device)
    f64 = torch.empty(values.shape, dtype=torch.float64, device=values.device)
    fin = torch.empty(values.shape, dtype=torch.float32, device=values.device)
    _tcheck(load_tooling().rex_probe_convert(_ptr(values), values.numel(), _ptr(f32), _ptr(f64), _ptr(fin),
                                             _stream_ptr(stream)), "rex_probe_convert")
    return f32, f64, fin


def version() -> str:
    return load().rex_version().decode()
