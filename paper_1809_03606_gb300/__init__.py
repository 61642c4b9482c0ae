"""polarscs: batched SCS decoding of polar codes on GB300 (sm_103a).

Thin ctypes binding of ``include/polarscs.h``: the functions below carry the
C names and only marshal arguments (tensor pointers, the current CUDA stream,
output allocation).  Every encode and decode step runs in the CUDA kernels
of ``csrc/``; there is no CPU fallback -- importing the compute entry points
without the built library raises.

PyTorch is used for device memory and streams only.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _build

POLAR_OK, POLAR_CRC_FAIL, POLAR_TIMEOUT, POLAR_DEBUG_FAIL = 0, 1, 2, 4
POLAR_EINVAL, POLAR_ENOMEM, POLAR_ECUDA, POLAR_ELIMIT, POLAR_ESCRATCH, POLAR_ETIMEOUT = -1, -2, -3, -4, -5, -6
MAX_N_GPU, MAX_D_GPU, MAX_L_GPU = 8192, 64, 255
MAX_D_GPU_DEEP = 65536  # scs_decode_batch of min-sum plans (memory stack)
OP_NAMES = {0: "alpha", 1: "beta", 2: "R0", 3: "R1", 4: "REP", 5: "SPC", 6: "leaf0", 7: "leaf1"}

EXPORTED = (
    "polar_construct", "polar_plan_create", "polar_plan_destroy", "polar_plan_schedule", "polar_encode_batch",
    "polar_encode", "scs_decode_batch", "scs_decode", "polar_device_info", "scs_decode_batch_noalloc",
    "polar_plan_set_create", "polar_plan_set_destroy", "scs_decode_mixed", "scs_tune_mixed",
    "gsc_loss", "gsc_loss_grad", "gsc_loss_f64", "gsc_loss_grad_f64", "polar_plan_set_scales", "polar_mixed_order",
    "polar_serve", "polar_serve_baseline", "polar_plan_set_systematic", "polar_plan_set_exact",
    "polar_mixed_split_order", "scs_decode_mixed_split", "polar_plan_set_tuning", "polar_plan_set_get_tuning",
)

_lock = threading.Lock()
_lib = None


class PolarError(RuntimeError):
    def __init__(self, fn: str, rc: int):
        names = {-1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ELIMIT", -5: "ESCRATCH", -6: "ETIMEOUT"}
        super().__init__(f"{fn} failed: {names.get(rc, rc)}")
        self.rc = rc


def lib_path() -> str:
    """The library this process loads: $POLARSCS_LIB if set, else the in-tree build."""
    return os.environ.get("POLARSCS_LIB") or _build.LIB


def load(build_if_missing: bool = False):
    """Load libpolarscs.so (building the in-tree library first only if asked)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = lib_path()
        if build_if_missing and path == _build.LIB:
            _build.build()
        if not os.path.exists(path):
            raise ImportError(f"libpolarscs.so is not built ({path}); run __graft_entry__.build()")
        lib = C.CDLL(path)
        vp, i32, f32 = C.c_void_p, C.c_int, C.c_float
        lib.polar_construct.argtypes = [i32, i32, f32, vp]
        lib.polar_plan_create.argtypes = [i32, i32, vp, i32, i32, C.POINTER(vp)]
        lib.polar_plan_destroy.argtypes = [vp]
        lib.polar_plan_destroy.restype = None
        lib.polar_plan_schedule.argtypes = [vp, vp, i32]
        lib.polar_plan_set_scales.argtypes = [vp, vp]
        lib.polar_plan_set_systematic.argtypes = [vp, i32]
        lib.polar_plan_set_exact.argtypes = [vp, i32]
        lib.polar_encode_batch.argtypes = [vp, vp, i32, vp, vp]
        lib.polar_encode.argtypes = [vp, i32, i32, vp, i32, vp]
        lib.scs_decode_batch.argtypes = [vp, vp, i32, i32, i32, vp, vp, vp, vp, vp]
        lib.scs_decode.argtypes = [vp, i32, i32, vp, i32, i32, i32, vp, vp]
        lib.scs_decode_batch_noalloc.argtypes = [vp, vp, i32, i32, i32, vp, vp, vp, vp, vp]
        lib.polar_device_info.argtypes = [vp, vp, vp]
        lib.polar_plan_set_create.argtypes = [vp, i32, C.POINTER(vp)]
        lib.polar_plan_set_destroy.argtypes = [vp]
        lib.polar_plan_set_destroy.restype = None
        lib.scs_decode_mixed.argtypes = [vp, vp, vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp]
        lib.scs_tune_mixed.argtypes = [vp, vp, vp, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp]
        lib.polar_plan_set_tuning.argtypes = [vp, i32, i32]
        lib.polar_plan_set_get_tuning.argtypes = [vp, vp, vp]
        lib.polar_mixed_order.argtypes = [vp, vp, i32, vp]
        lib.polar_mixed_split_order.argtypes = [vp, vp, i32, vp, vp]
        lib.scs_decode_mixed_split.argtypes = [vp, vp, vp, i32, i32, i32, vp, vp, vp, vp, vp, vp, vp, vp]
        i64, f64 = C.c_int64, C.c_double
        lib.polar_serve.argtypes = [vp, vp, vp, i32, vp, vp, i32, i64, f64, vp, vp, vp, vp, vp, vp, vp]
        lib.polar_serve_baseline.argtypes = [vp, vp, vp, i32, vp, vp, i32, i64, f64, f64, vp, vp, vp, vp]
        for fn in (lib.gsc_loss, lib.gsc_loss_f64):
            fn.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp]
        for fn in (lib.gsc_loss_grad, lib.gsc_loss_grad_f64):
            fn.argtypes = [vp, vp, vp, i32, vp, vp, vp, vp, vp]
        _lib = lib
        return lib


def _check(fn: str, rc: int) -> int:
    if rc < 0:
        raise PolarError(fn, rc)
    return rc


def _np_ptr(a: np.ndarray):
    return C.c_void_p(a.ctypes.data)


def _stream_ptr(stream) -> C.c_void_p:
    import torch

    s = torch.cuda.current_stream() if stream is None else stream
    return C.c_void_p(int(s.cuda_stream))


def _dev_ptr(t, dtype, name: str, shape=None):
    import torch

    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype or not t.is_contiguous():
        raise TypeError(f"{name} must be a contiguous {dtype} tensor")
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return C.c_void_p(t.data_ptr())


# ---------------------------------------------------------------- host calls
def polar_construct(N: int, K: int, design_snr_db: float) -> np.ndarray:
    fr = np.zeros(N, np.uint8)
    _check("polar_construct", load().polar_construct(N, K, float(design_snr_db), _np_ptr(fr)))
    return fr


class Plan:
    """Owner of a ``polar_plan*`` (the schedule of Fig. fsscsch plus tables)."""

    def __init__(self, N: int, K: int, frozen: np.ndarray, fast_nodes: bool = True, crc: int = 0,
                 systematic: bool = False, exact: bool = False):
        fr = np.ascontiguousarray(frozen, dtype=np.uint8)
        if fr.size != N:
            raise ValueError("frozen mask must have N entries")
        h = C.c_void_p()
        _check("polar_plan_create", load().polar_plan_create(N, K, _np_ptr(fr), int(bool(fast_nodes)), crc, C.byref(h)))
        self._h = h
        self.systematic = False
        self.exact = False
        if systematic:
            polar_plan_set_systematic(self, True)
        if exact:
            polar_plan_set_exact(self, True)
        self.N, self.K, self.crc, self.fast = N, K, crc, bool(fast_nodes)
        self.kmsg = K - crc
        self.frozen = fr.copy()
        self.words = max(1, N // 32)
        self.msg_words = (self.kmsg + 31) // 32

    @property
    def handle(self) -> C.c_void_p:
        return self._h

    def schedule(self) -> list[tuple[str, int, int]]:
        return polar_plan_schedule(self)

    def set_scales(self, scales) -> None:
        """Per-stage min-sum scales for decoding (None: plain min-sum)."""
        polar_plan_set_scales(self, scales)

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            load().polar_plan_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def polar_plan_create(N: int, K: int, frozen: np.ndarray, fast_nodes: bool = True, crc: int = 0,
                      systematic: bool = False) -> Plan:
    return Plan(N, K, frozen, fast_nodes, crc, systematic)


def polar_plan_set_exact(plan: Plan, on: bool) -> None:
    """Exact-f decoding for a bit-level plan (before its first GPU use)."""
    _check("polar_plan_set_exact", load().polar_plan_set_exact(plan.handle, int(bool(on))))
    plan.exact = bool(on)


def polar_plan_set_systematic(plan: Plan, on: bool) -> None:
    """Systematic encoding and decoding for the plan (before its first GPU use)."""
    _check("polar_plan_set_systematic", load().polar_plan_set_systematic(plan.handle, int(bool(on))))
    plan.systematic = bool(on)


def polar_plan_destroy(plan: Plan) -> None:
    plan.close()


def polar_plan_set_scales(plan: Plan, scales) -> None:
    if scales is None:
        _check("polar_plan_set_scales", load().polar_plan_set_scales(plan.handle, None))
        plan.scales = None
        return
    sc = np.ascontiguousarray(scales, dtype=np.float32)
    if sc.size != int(np.log2(plan.N)):
        raise ValueError("one scale per stage (log2 N values)")
    _check("polar_plan_set_scales", load().polar_plan_set_scales(plan.handle, _np_ptr(sc)))
    plan.scales = sc.copy()


def polar_plan_schedule(plan: Plan) -> list[tuple[str, int, int]]:
    n = _check("polar_plan_schedule", load().polar_plan_schedule(plan.handle, None, 0))
    buf = np.zeros(3 * max(n, 1), np.int32)
    _check("polar_plan_schedule", load().polar_plan_schedule(plan.handle, _np_ptr(buf), n))
    t = buf[: 3 * n].reshape(n, 3)
    return [(OP_NAMES[int(a)], int(b), int(c)) for a, b, c in t]


# -------------------------------------------------------------- GPU calls
def polar_encode_batch(plan: Plan, msg_words, codeword_words, stream=None) -> None:
    """Encode B packed messages [B, ceil(kmsg/32)] int32 into packed codewords [B, N/32]."""
    import torch

    B = msg_words.shape[0]
    _check("polar_encode_batch", load().polar_encode_batch(
        plan.handle, _dev_ptr(msg_words, torch.int32, "msg_words", (B, plan.msg_words)), B,
        _dev_ptr(codeword_words, torch.int32, "codeword_words", (B, plan.words)), _stream_ptr(stream)))


def polar_encode(msg: np.ndarray, N: int, K: int, frozen: np.ndarray, crc: int = 0) -> np.ndarray:
    m = np.ascontiguousarray(msg, dtype=np.uint8)
    fr = np.ascontiguousarray(frozen, dtype=np.uint8)
    cw = np.zeros(N, np.uint8)
    _check("polar_encode", load().polar_encode(_np_ptr(m), N, K, _np_ptr(fr), crc, _np_ptr(cw)))
    return cw


def scs_decode_batch(plan: Plan, llr, D: int, L: int, info_words, pm, status, stats=None, stream=None) -> None:
    """Decode B frames of float32 LLRs [B, N] (CUDA tensors) into the given outputs."""
    import torch

    B = llr.shape[0]
    _check("scs_decode_batch", load().scs_decode_batch(
        plan.handle, _dev_ptr(llr, torch.float32, "llr", (B, plan.N)), B, D, L,
        _dev_ptr(info_words, torch.int32, "info_words", (B, plan.msg_words)),
        _dev_ptr(pm, torch.float32, "pm", (B,)), _dev_ptr(status, torch.int8, "status", (B,)),
        None if stats is None else _dev_ptr(stats, torch.int32, "stats", (B, 4)), _stream_ptr(stream)))


def scs_decode_batch_noalloc(plan: Plan, llr, D: int, L: int, info_words, pm, status, stats=None, stream=None) -> None:
    """scs_decode_batch with the library's fixed static scratch: no device
    allocation by the library (see include/polarscs.h for its limits and the
    rule that calls must not overlap on the GPU)."""
    import torch

    B = llr.shape[0]
    _check("scs_decode_batch_noalloc", load().scs_decode_batch_noalloc(
        plan.handle, _dev_ptr(llr, torch.float32, "llr", (B, plan.N)), B, D, L,
        _dev_ptr(info_words, torch.int32, "info_words", (B, plan.msg_words)),
        _dev_ptr(pm, torch.float32, "pm", (B,)), _dev_ptr(status, torch.int8, "status", (B,)),
        None if stats is None else _dev_ptr(stats, torch.int32, "stats", (B, 4)), _stream_ptr(stream)))


def decode(plan: Plan, llr, D: int, L: int, with_stats: bool = False, stream=None):
    """Allocate outputs and call scs_decode_batch.  Returns (info_words, pm, status[, stats])."""
    import torch

    B = llr.shape[0]
    dev = llr.device
    info = torch.empty((B, plan.msg_words), dtype=torch.int32, device=dev)
    pm = torch.empty(B, dtype=torch.float32, device=dev)
    status = torch.empty(B, dtype=torch.int8, device=dev)
    stats = torch.empty((B, 4), dtype=torch.int32, device=dev) if with_stats else None
    scs_decode_batch(plan, llr, D, L, info, pm, status, stats, stream)
    return (info, pm, status, stats) if with_stats else (info, pm, status)


# ------------------------------------------------------------- mixed batches
class PlanSet:
    """Owner of a ``polar_plan_set*``: plans decoded together by index."""

    def __init__(self, plans):
        self.plans = list(plans)  # kept alive: the set refers to them
        arr = (C.c_void_p * len(self.plans))(*[pl.handle.value for pl in self.plans])
        h = C.c_void_p()
        _check("polar_plan_set_create", load().polar_plan_set_create(C.cast(arr, C.c_void_p), len(self.plans), C.byref(h)))
        self._h = h

    @property
    def handle(self) -> C.c_void_p:
        return self._h

    def close(self) -> None:
        if getattr(self, "_h", None) and self._h.value:
            load().polar_plan_set_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def polar_plan_set_create(plans) -> PlanSet:
    return PlanSet(plans)


def polar_plan_set_destroy(pset: PlanSet) -> None:
    pset.close()


def _mixed_args(pset, frames, Dmax, llr, llr_off, info, info_off, pm, status, order=None):
    import torch

    B = frames.shape[0]
    return (pset.handle, _dev_ptr(frames, torch.int32, "frames", (B, 4)),
            None if order is None else _dev_ptr(order, torch.int32, "order", (B,)), B, int(Dmax),
            _dev_ptr(llr, torch.float32, "llr"), _dev_ptr(llr_off, torch.int64, "llr_off", (B,)),
            _dev_ptr(info, torch.int32, "info"), _dev_ptr(info_off, torch.int64, "info_off", (B,)),
            _dev_ptr(pm, torch.float32, "pm", (B,)), _dev_ptr(status, torch.int8, "status", (B,)))


def scs_decode_mixed(pset: PlanSet, frames, Dmax: int, llr, llr_off, info, info_off, pm, status, stats=None,
                     stream=None, order=None) -> None:
    """Decode a packed batch of frames of different codes in one launch (see polarscs.h)."""
    import torch

    B = frames.shape[0]
    _check("scs_decode_mixed", load().scs_decode_mixed(
        *_mixed_args(pset, frames, Dmax, llr, llr_off, info, info_off, pm, status, order),
        None if stats is None else _dev_ptr(stats, torch.int32, "stats", (B, 4)), _stream_ptr(stream)))


def scs_tune_mixed(pset: PlanSet, frames, Dmax: int, llr, llr_off, info, info_off, pm, status, stream=None,
                   order=None):
    """Run the native autotuner on this batch; returns (warps per block, frames per claim)."""
    w, c = C.c_int(0), C.c_int(0)
    _check("scs_tune_mixed", load().scs_tune_mixed(
        *_mixed_args(pset, frames, Dmax, llr, llr_off, info, info_off, pm, status, order), _stream_ptr(stream),
        C.byref(w), C.byref(c)))
    return w.value, c.value


def polar_plan_set_tuning(pset: PlanSet, warps_per_block: int, frames_per_claim: int) -> None:
    """Set the set's mixed-batch launch shape (both 0: the defaults)."""
    _check("polar_plan_set_tuning", load().polar_plan_set_tuning(pset.handle, int(warps_per_block),
                                                                 int(frames_per_claim)))


def polar_plan_set_get_tuning(pset: PlanSet):
    """The set's mixed-batch launch shape: (warps per block, frames per claim), (0, 0) if unset."""
    w, c = C.c_int(0), C.c_int(0)
    _check("polar_plan_set_get_tuning", load().polar_plan_set_get_tuning(pset.handle, C.byref(w), C.byref(c)))
    return w.value, c.value


def tuning_key(pset: PlanSet, Dmax: int, device: str) -> str:
    """Key of a tuning result: the GPU, the largest D and, per code, N, K, CRC
    length, fast nodes, systematic form and a digest of the frozen set."""
    import hashlib

    codes = []
    for pl in pset.plans:
        fz = hashlib.sha256(np.ascontiguousarray(pl.frozen, dtype=np.uint8).tobytes()).hexdigest()[:12]
        codes.append(f"{pl.N}/{pl.K}/{pl.crc}/{int(pl.fast)}/{int(pl.systematic)}/{fz}")
    return f"{device}|D{int(Dmax)}|" + ";".join(codes)


class TuningCache:
    """Autotuner results kept in a JSON file between runs, so that a process
    restores the launch shape of a known (GPU, codes, D) instead of timing
    the nine shapes again.  The file maps tuning_key() to [warps per block,
    frames per claim]; it is rewritten whole (through a temporary file) on
    every store."""

    def __init__(self, path: str):
        self.path = path

    def _read(self) -> dict:
        import json

        try:
            with open(self.path) as f:
                data = json.load(f)
        except FileNotFoundError:
            return {}
        if not isinstance(data, dict):
            raise ValueError(f"{self.path}: not a tuning cache")
        return data

    def lookup(self, key: str):
        v = self._read().get(key)
        return None if v is None else (int(v[0]), int(v[1]))

    def store(self, key: str, warps_per_block: int, frames_per_claim: int) -> None:
        import json

        data = self._read()
        data[key] = [int(warps_per_block), int(frames_per_claim)]
        tmp = f"{self.path}.{os.getpid()}.tmp"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, self.path)


def tune_mixed_cached(cache: TuningCache, pset: PlanSet, frames, Dmax: int, llr, llr_off, info, info_off, pm,
                      status, stream=None, order=None, device: str | None = None, tuner=None):
    """scs_tune_mixed through a TuningCache: a known key sets the stored shape
    on the set (no device work); otherwise the native autotuner runs on this
    batch and its result is stored.  Returns (warps per block, frames per
    claim, True if it came from the cache).  ``tuner`` replaces
    scs_tune_mixed (same arguments), e.g. in tests without a GPU."""
    if device is None:
        import torch

        device = torch.cuda.get_device_name(torch.cuda.current_device())
    key = tuning_key(pset, Dmax, device)
    hit = cache.lookup(key)
    if hit is not None:
        polar_plan_set_tuning(pset, *hit)
        return hit[0], hit[1], True
    w, c = (tuner or scs_tune_mixed)(pset, frames, Dmax, llr, llr_off, info, info_off, pm, status, stream=stream,
                                     order=order)
    polar_plan_set_tuning(pset, w, c)
    cache.store(key, w, c)
    return w, c, False


def save_scales(path: str, scales) -> None:
    """Write learned per-stage scales (float32) to a JSON file; every float32
    value is exact as a JSON number."""
    import json

    sc = np.ascontiguousarray(scales, dtype=np.float32)
    with open(path, "w") as f:
        json.dump({"stages": int(sc.size), "scales": [float(x) for x in sc]}, f)


def load_scales(path: str) -> np.ndarray:
    """Read scales written by save_scales (float32, one per stage)."""
    import json

    with open(path) as f:
        data = json.load(f)
    sc = np.asarray(data["scales"], dtype=np.float32)
    if sc.size != int(data["stages"]):
        raise ValueError(f"{path}: {sc.size} scales for {data['stages']} stages")
    return sc


def polar_mixed_split_order(pset: PlanSet, frames_host: np.ndarray):
    """Claim order for scs_decode_mixed_split (host): (order, n_two), the
    frames needing two stack rows (D > 32) first."""
    fr = np.ascontiguousarray(frames_host, dtype=np.int32)
    out = np.zeros(fr.shape[0], np.int32)
    n_two = C.c_int(0)
    _check("polar_mixed_split_order", load().polar_mixed_split_order(pset.handle, _np_ptr(fr), fr.shape[0],
                                                                     _np_ptr(out), C.byref(n_two)))
    return out, n_two.value


def scs_decode_mixed_split(pset: PlanSet, frames, order, n_two: int, Dmax: int, llr, llr_off, info, info_off, pm,
                           status, stats=None, stream=None) -> None:
    """The mixed batch in two launches split by stack rows (see polarscs.h);
    ``order`` and ``n_two`` come from polar_mixed_split_order."""
    import torch

    B = frames.shape[0]
    args = _mixed_args(pset, frames, Dmax, llr, llr_off, info, info_off, pm, status, order)
    # _mixed_args gives (set, frames, order, B, Dmax, llr, llr_off, info, info_off, pm, status)
    _check("scs_decode_mixed_split", load().scs_decode_mixed_split(
        args[0], args[1], args[2], args[3], int(n_two), *args[4:],
        None if stats is None else _dev_ptr(stats, torch.int32, "stats", (B, 4)), _stream_ptr(stream)))


def polar_mixed_order(pset: PlanSet, frames_host: np.ndarray) -> np.ndarray:
    """Longest-first claim order (host) for a [B, 4] int32 descriptor array."""
    fr = np.ascontiguousarray(frames_host, dtype=np.int32)
    out = np.zeros(fr.shape[0], np.int32)
    _check("polar_mixed_order", load().polar_mixed_order(pset.handle, _np_ptr(fr), fr.shape[0], _np_ptr(out)))
    return out


class MixedBatch:
    """Device buffers of a mixed batch: frames (plan index, D, L) with their
    packed LLRs and output slots.  Built from host arrays (marshalling only)."""

    def __init__(self, pset: PlanSet, plan_idx, D, L, llr_rows, device="cuda"):
        import torch

        plan_idx = np.asarray(plan_idx, np.int32)
        B = plan_idx.size
        Ns = np.array([pset.plans[i].N for i in plan_idx], np.int64)
        words = np.array([pset.plans[i].msg_words for i in plan_idx], np.int64)
        self.B = B
        self.llr_off_np = np.concatenate([[0], np.cumsum(Ns)[:-1]]).astype(np.int64)
        self.info_off_np = np.concatenate([[0], np.cumsum(words)[:-1]]).astype(np.int64)
        fr = np.zeros((B, 4), np.int32)
        fr[:, 0] = plan_idx
        fr[:, 1] = np.asarray(D, np.int32)
        fr[:, 2] = np.asarray(L, np.int32)
        self.Dmax = int(fr[:, 1].max()) if B else 1
        self.frames = torch.from_numpy(fr).to(device)
        self.order = torch.from_numpy(polar_mixed_order(pset, fr)).to(device) if B else None
        split, self.n_two = polar_mixed_split_order(pset, fr) if B else (np.zeros(0, np.int32), 0)
        self.split_order = torch.from_numpy(split).to(device) if B else None
        if isinstance(llr_rows, np.ndarray) and llr_rows.ndim == 1:
            flat = llr_rows.astype(np.float32, copy=False)
        else:
            flat = np.concatenate([np.asarray(r, np.float32) for r in llr_rows]) if B else np.zeros(0, np.float32)
        self.llr = torch.from_numpy(flat).to(device)
        self.llr_off = torch.from_numpy(self.llr_off_np).to(device)
        self.info_off = torch.from_numpy(self.info_off_np).to(device)
        self.info = torch.zeros(int(words.sum()) if B else 1, dtype=torch.int32, device=device)
        self.pm = torch.empty(B, dtype=torch.float32, device=device)
        self.status = torch.empty(B, dtype=torch.int8, device=device)
        self.words = words

    def decode(self, pset: PlanSet, stats=None, stream=None) -> None:
        scs_decode_mixed(pset, self.frames, self.Dmax, self.llr, self.llr_off, self.info, self.info_off, self.pm,
                         self.status, stats, stream, self.order)

    def decode_split(self, pset: PlanSet, stats=None, stream=None) -> None:
        """The same batch in two launches split by stack rows (scs_decode_mixed_split)."""
        scs_decode_mixed_split(pset, self.frames, self.split_order, self.n_two, self.Dmax, self.llr, self.llr_off,
                               self.info, self.info_off, self.pm, self.status, stats, stream)

    def tune(self, pset: PlanSet, stream=None):
        return scs_tune_mixed(pset, self.frames, self.Dmax, self.llr, self.llr_off, self.info, self.info_off, self.pm,
                              self.status, stream, self.order)

    def message_words(self, b: int) -> np.ndarray:
        lo = int(self.info_off_np[b])
        return self.info[lo:lo + int(self.words[b])].cpu().numpy()


# ---------------------------------------- genie-aided SC (differentiation)
def _gsc_fns(dtype):
    import torch

    if dtype == torch.float32:
        return load().gsc_loss, load().gsc_loss_grad
    if dtype == torch.float64:
        return load().gsc_loss_f64, load().gsc_loss_grad_f64
    raise TypeError("genie-aided SC runs in float32 or float64")


def gsc_loss(plan: Plan, llr, u_words, scales, leaf=None, stream=None):
    """Mean BCE of genie-aided SC leaf LLRs over information leaves (device scalar)."""
    import torch

    B = llr.shape[0]
    loss = torch.empty((), dtype=llr.dtype, device=llr.device)
    fn, _ = _gsc_fns(llr.dtype)
    _check("gsc_loss", fn(plan.handle, _dev_ptr(llr, llr.dtype, "llr", (B, plan.N)),
                          _dev_ptr(u_words, torch.int32, "u_words", (B, plan.words)), B,
                          _dev_ptr(scales, llr.dtype, "scales"), C.c_void_p(loss.data_ptr()),
                          None if leaf is None else _dev_ptr(leaf, llr.dtype, "leaf", (B, plan.N)), _stream_ptr(stream)))
    return loss


def gsc_loss_grad(plan: Plan, llr, u_words, scales, want_llr_grad: bool = False, stream=None):
    """(loss, d loss/d scales, d loss/d llr or None), from the reverse kernel."""
    import torch

    B = llr.shape[0]
    loss = torch.empty((), dtype=llr.dtype, device=llr.device)
    gs = torch.empty_like(scales)
    gl = torch.empty_like(llr) if want_llr_grad else None
    _, fn = _gsc_fns(llr.dtype)
    _check("gsc_loss_grad", fn(plan.handle, _dev_ptr(llr, llr.dtype, "llr", (B, plan.N)),
                               _dev_ptr(u_words, torch.int32, "u_words", (B, plan.words)), B,
                               _dev_ptr(scales, llr.dtype, "scales"), C.c_void_p(loss.data_ptr()),
                               C.c_void_p(gs.data_ptr()), None if gl is None else C.c_void_p(gl.data_ptr()),
                               _stream_ptr(stream)))
    return loss, gs, gl


def _make_genie_function():
    import torch

    class GenieSCLoss(torch.autograd.Function):
        """loss = GenieSCLoss.apply(llr, scales, u_words, plan).  The forward
        kernel computes the loss; backward runs the hand-written reverse kernel
        (which recomputes the tree) for d loss/d scales and d loss/d llr."""

        @staticmethod
        def forward(ctx, llr, scales, u_words, plan):
            llr_c, sc_c = llr.detach().contiguous(), scales.detach().contiguous()
            ctx.save_for_backward(llr_c, sc_c, u_words)
            ctx.plan = plan
            return gsc_loss(plan, llr_c, u_words, sc_c)

        @staticmethod
        def backward(ctx, gout):
            llr_c, sc_c, u_words = ctx.saved_tensors
            _, gs, gl = gsc_loss_grad(ctx.plan, llr_c, u_words, sc_c, want_llr_grad=ctx.needs_input_grad[0])
            return (None if gl is None else gl * gout), gs * gout, None, None

    return GenieSCLoss


_genie_cls = None


def genie_sc_loss(llr, scales, u_words, plan: Plan):
    """Differentiable genie-aided SC loss (see gsc_loss)."""
    global _genie_cls
    if _genie_cls is None:
        _genie_cls = _make_genie_function()
    return _genie_cls.apply(llr, scales, u_words, plan)


def u_from_messages(plan: Plan, msg_bits: np.ndarray) -> np.ndarray:
    """Packed transmitted u vectors [B, N/32] from message bits [B, K] (no CRC):
    the information set in increasing index order, frozen positions 0."""
    msg_bits = np.asarray(msg_bits, np.uint8)
    B = msg_bits.shape[0]
    u = np.zeros((B, plan.N), np.uint8)
    u[:, plan.frozen == 0] = msg_bits
    return pack_bits(u)


# ------------------------------------------------------------------ serving
_REPORT = ("seconds_to_last_completion", "arena_full_stalls", "error", "max_in_flight_or_launches", "completed",
           "arena_bytes")


def _serve_inputs(req, arrival_s, pool_llr, pool_off):
    req = np.ascontiguousarray(req, dtype=np.int32).reshape(-1, 4)
    arr = np.ascontiguousarray(arrival_s, dtype=np.float64)
    pool = np.ascontiguousarray(pool_llr, dtype=np.float32).reshape(-1)
    poff = np.ascontiguousarray(pool_off, dtype=np.int64)
    if arr.size != req.shape[0]:
        raise ValueError("one arrival time per request")
    return req, arr, pool, poff


def polar_serve(pset: PlanSet, req, arrival_s, pool_llr, pool_off, arena_floats: int, wait_s: float = 30.0,
                info_off=None) -> dict:
    """Continuous-batching engine (see polarscs.h).  Returns per-request pm,
    status, latency (s), service time (s, a warp's start to completion),
    optional message words, and the engine report."""
    req, arr, pool, poff = _serve_inputs(req, arrival_s, pool_llr, pool_off)
    R = req.shape[0]
    pm = np.zeros(R, np.float32)
    st = np.zeros(R, np.int8)
    lat = np.zeros(R, np.float64)
    svc = np.zeros(R, np.float64)
    rep = np.zeros(6, np.float64)
    info = ioff = None
    if info_off is not None:
        ioff = np.ascontiguousarray(info_off, dtype=np.int64)
        words = np.array([pset.plans[int(i)].msg_words for i in req[:, 0]], np.int64)
        info = np.zeros(int((ioff + words).max()), np.uint32)
    rc = load().polar_serve(pset.handle, _np_ptr(req), _np_ptr(arr), R, _np_ptr(pool), _np_ptr(poff), poff.size,
                            int(arena_floats), float(wait_s), _np_ptr(pm), _np_ptr(st),
                            None if info is None else _np_ptr(info), None if ioff is None else _np_ptr(ioff),
                            _np_ptr(lat), _np_ptr(svc), _np_ptr(rep))
    out = dict(rc=rc, pm=pm, status=st, latency=lat, service=svc, info=info, report=dict(zip(_REPORT, rep.tolist())))
    if rc < 0 and rc != POLAR_ETIMEOUT:
        raise PolarError("polar_serve", rc)
    return out


def polar_serve_baseline(pset: PlanSet, req, arrival_s, pool_llr, pool_off, arena_floats: int,
                         interval_s: float = 1e-3, wait_s: float = 30.0) -> dict:
    """One-size-per-launch baseline engine over the same request stream."""
    req, arr, pool, poff = _serve_inputs(req, arrival_s, pool_llr, pool_off)
    R = req.shape[0]
    pm = np.zeros(R, np.float32)
    st = np.zeros(R, np.int8)
    lat = np.zeros(R, np.float64)
    rep = np.zeros(6, np.float64)
    rc = load().polar_serve_baseline(pset.handle, _np_ptr(req), _np_ptr(arr), R, _np_ptr(pool), _np_ptr(poff),
                                     poff.size, int(arena_floats), float(interval_s), float(wait_s), _np_ptr(pm),
                                     _np_ptr(st), _np_ptr(lat), _np_ptr(rep))
    out = dict(rc=rc, pm=pm, status=st, latency=lat, report=dict(zip(_REPORT, rep.tolist())))
    if rc < 0 and rc != POLAR_ETIMEOUT:
        raise PolarError("polar_serve_baseline", rc)
    return out


def scs_decode(llr: np.ndarray, N: int, K: int, frozen: np.ndarray, D: int, L: int, crc: int = 0):
    """One frame from host memory (synchronous).  Returns (status, message bits, pm)."""
    x = np.ascontiguousarray(llr, dtype=np.float32)
    fr = np.ascontiguousarray(frozen, dtype=np.uint8)
    out = np.zeros(K - crc, np.uint8)
    pm = C.c_float(0.0)
    rc = _check("scs_decode", load().scs_decode(_np_ptr(x), N, K, _np_ptr(fr), D, L, crc, _np_ptr(out), C.byref(pm)))
    return rc, out, np.float32(pm.value)


def polar_device_info() -> dict:
    sm, ma, mi = C.c_int(0), C.c_int(0), C.c_int(0)
    _check("polar_device_info", load().polar_device_info(C.byref(sm), C.byref(ma), C.byref(mi)))
    return dict(sm_count=sm.value, cc=(ma.value, mi.value))


# ------------------------------------------------------- bit packing helpers
def pack_bits(bits: np.ndarray) -> np.ndarray:
    """[B, k] 0/1 bytes -> [B, ceil(k/32)] int32 words, bit j in word j/32 at j%32."""
    bits = np.ascontiguousarray(bits, dtype=np.uint8)
    B, k = bits.shape
    w = (k + 31) // 32
    pad = np.zeros((B, w * 32), np.uint8)
    pad[:, :k] = bits
    return np.packbits(pad, axis=1, bitorder="little").view(np.uint32).astype(np.uint32).view(np.int32).reshape(B, w)


def unpack_bits(words: np.ndarray, k: int) -> np.ndarray:
    """Inverse of pack_bits: [B, w] int32/uint32 words -> [B, k] 0/1 bytes."""
    words = np.ascontiguousarray(words).view(np.uint32)
    B = words.shape[0]
    by = words.reshape(B, -1).view(np.uint8)
    return np.unpackbits(by, axis=1, bitorder="little")[:, :k]
