"""CPU oracle for SCS decoding of polar codes (arXiv 1809.03606).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  The GPU library
(``paper_1809_03606_gb300``) never imports it, and the two share no code.

The arithmetic lives in ``polar_oracle.c`` (plain scalar C, built with
``-O2 -fno-fast-math -ffp-contract=off``); this module compiles it for the
host it runs on and wraps it with ctypes.  Every function cites the passage
of the paper it follows in the C source.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "polar_oracle.c")
_INC = os.path.join(_HERE, "polar_oracle_exact.inc")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

OK, CRC_FAIL, EINVAL, ENOMEM = 0, 1, -1, -2
# schedule op codes (Fig. fsscsch)
ALPHA, BETA, R0, R1, REP, SPC, LEAF0, LEAF1 = range(8)
OP_NAMES = {ALPHA: "alpha", BETA: "beta", R0: "R0", R1: "R1", REP: "REP", SPC: "SPC", LEAF0: "leaf0", LEAF1: "leaf1"}

_FLAGS = ["-O2", "-fno-fast-math", "-ffp-contract=off", "-std=c11", "-shared", "-fPIC"]


def build(force: bool = False) -> str:
    """Compile the oracle for this host (gcc, no architecture-specific flags)."""
    os.makedirs(_BUILD, exist_ok=True)
    newest = max(os.path.getmtime(_SRC), os.path.getmtime(_INC))
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < newest:
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", *_FLAGS, "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            u8p, f32p, f64p, i32p, u64p, i8p = (C.POINTER(t) for t in (C.c_uint8, C.c_float, C.c_double, C.c_int, C.c_uint64, C.c_int8))
            lib.or_construct.argtypes = [C.c_int, C.c_int, C.c_double, u8p]
            lib.or_encode.argtypes = [u8p, C.c_int, u8p]
            lib.or_encode.restype = None
            lib.or_crc.argtypes = [u8p, C.c_int, C.c_int]
            lib.or_crc.restype = C.c_uint32
            lib.or_encode_msg.argtypes = [u8p, C.c_int, C.c_int, u8p, C.c_int, u8p]
            lib.or_encode_sys.argtypes = [u8p, C.c_int, u8p, u8p]
            lib.or_encode_msg_sys.argtypes = [u8p, C.c_int, C.c_int, u8p, C.c_int, u8p]
            lib.or_schedule.argtypes = [C.c_int, u8p, C.c_int, i32p, C.c_int]
            lib.or_scs_decode.argtypes = [f32p, C.c_int, C.c_int, u8p, C.c_int, C.c_int, C.c_int, C.c_int, u8p, f32p, u8p, u64p]
            lib.or_scs_decode_batch.argtypes = [f32p, C.c_int, C.c_int, C.c_int, u8p, C.c_int, C.c_int, C.c_int, C.c_int, u8p, f32p, i8p, u64p]
            lib.or_scs_decode_s.argtypes = [f32p, C.c_int, C.c_int, u8p, C.c_int, C.c_int, C.c_int, C.c_int, f32p, u8p, f32p, u8p, u64p]
            lib.or_scs_decode_batch_s.argtypes = [f32p, C.c_int, C.c_int, C.c_int, u8p, C.c_int, C.c_int, C.c_int, C.c_int, f32p, u8p, f32p, i8p, u64p]
            lib.or_scs_decode_sx.argtypes = [f32p, C.c_int, C.c_int, u8p, C.c_int, C.c_int, C.c_int, C.c_int, f32p, C.c_int, u8p, f32p, u8p, u64p]
            lib.or_scs_decode_batch_sx.argtypes = [f32p, C.c_int, C.c_int, C.c_int, u8p, C.c_int, C.c_int, C.c_int, C.c_int, f32p, C.c_int, u8p, f32p, i8p, u64p]
            lib.or_scs_decode_trace.argtypes = [f32p, C.c_int, C.c_int, u8p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                                C.c_int, i32p, f32p, u8p, i32p, u8p, f32p, u8p, u64p]
            lib.or_scs_decode_exact.argtypes = [f64p, C.c_int, C.c_int, u8p, C.c_int, C.c_int, u8p, f64p]
            lib.or_scs_decode_exact_f32.argtypes = [f32p, C.c_int, C.c_int, u8p, C.c_int, C.c_int, u8p, f32p]
            lib.or_gsc_forward.argtypes = [f64p, u8p, C.c_int, f64p, f64p]
            lib.or_gsc_loss_grad.argtypes = [f64p, u8p, C.c_int, C.c_int, u8p, f64p, f64p, f64p]
            _lib = lib
    return _lib


def _p(a: np.ndarray, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def _u8(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint8)


def construct(N: int, K: int, design_snr_db: float) -> np.ndarray:
    """Frozen mask (1 = frozen) by Bhattacharyya construction (reading R13)."""
    fr = np.zeros(N, np.uint8)
    rc = _load().or_construct(N, K, float(design_snr_db), _p(fr, C.c_uint8))
    if rc:
        raise ValueError(f"or_construct({N}, {K}) -> {rc}")
    return fr


def encode(u: np.ndarray) -> np.ndarray:
    """c = u F^{(x)n} (Sec. 2.1) for one length-N vector."""
    u = _u8(u)
    x = np.zeros_like(u)
    _load().or_encode(_p(u, C.c_uint8), u.size, _p(x, C.c_uint8))
    return x


def crc(bits: np.ndarray, crc_len: int) -> int:
    bits = _u8(bits)
    return int(_load().or_crc(_p(bits, C.c_uint8), bits.size, crc_len))


def encode_sys(info: np.ndarray, N: int, frozen: np.ndarray) -> np.ndarray:
    """Systematic codeword: x = u F^{(x)n}, u frozen = 0, x on the information
    set = the K bits of ``info`` in increasing index order."""
    info, fr = _u8(info), _u8(frozen)
    x = np.zeros(N, np.uint8)
    rc = _load().or_encode_sys(_p(info, C.c_uint8), N, _p(fr, C.c_uint8), _p(x, C.c_uint8))
    if rc:
        raise ValueError(f"or_encode_sys -> {rc}")
    return x


def encode_msg(msg: np.ndarray, N: int, K: int, frozen: np.ndarray, crc_len: int = 0,
               systematic: bool = False) -> np.ndarray:
    """Codeword for one message of K - crc bits (CRC appended MSB first)."""
    msg, fr = _u8(msg), _u8(frozen)
    cw = np.zeros(N, np.uint8)
    fn = _load().or_encode_msg_sys if systematic else _load().or_encode_msg
    rc = fn(_p(msg, C.c_uint8), N, K, _p(fr, C.c_uint8), crc_len, _p(cw, C.c_uint8))
    if rc:
        raise ValueError(f"or_encode_msg -> {rc}")
    return cw


def encode_batch(msgs: np.ndarray, N: int, K: int, frozen: np.ndarray, crc_len: int = 0,
                 systematic: bool = False) -> np.ndarray:
    msgs = _u8(msgs)
    out = np.zeros((msgs.shape[0], N), np.uint8)
    for b in range(msgs.shape[0]):
        out[b] = encode_msg(msgs[b], N, K, frozen, crc_len, systematic)
    return out


def schedule(N: int, frozen: np.ndarray, fast: bool) -> list[tuple[str, int, int]]:
    """The FSSC (or bit-level) schedule as (op, lambda, phi) triples."""
    fr = _u8(frozen)
    buf = np.zeros(3 * 4 * N, np.int32)
    n = _load().or_schedule(N, _p(fr, C.c_uint8), int(bool(fast)), _p(buf, C.c_int), 4 * N)
    if n < 0:
        raise ValueError(f"or_schedule -> {n}")
    t = buf[: 3 * n].reshape(n, 3)
    return [(OP_NAMES[int(a)], int(b), int(c)) for a, b, c in t]


def _scales_arg(scales):
    if scales is None:
        return None, None
    sc = np.ascontiguousarray(scales, dtype=np.float32)
    return sc, _p(sc, C.c_float)


def scs_decode(llr: np.ndarray, N: int, K: int, frozen: np.ndarray, *, fast: bool, D: int, L: int, crc_len: int = 0,
               scales=None, systematic: bool = False):
    """One frame.  Returns (status, msg bits [K-crc], pm, codeword [N], stats dict).
    ``scales`` (n floats) multiplies every f output written at stage lambda;
    ``systematic`` reads the message off the codeword estimate."""
    llr = np.ascontiguousarray(llr, dtype=np.float32)
    fr = _u8(frozen)
    msg = np.zeros(K - crc_len, np.uint8)
    cw = np.zeros(N, np.uint8)
    pm = C.c_float(0.0)
    st = np.zeros(5, np.uint64)
    sc, scp = _scales_arg(scales)
    rc = _load().or_scs_decode_sx(_p(llr, C.c_float), N, K, _p(fr, C.c_uint8), int(bool(fast)), D, L, crc_len, scp,
                                  int(bool(systematic)), _p(msg, C.c_uint8), C.byref(pm), _p(cw, C.c_uint8),
                                  _p(st, C.c_uint64))
    if rc < 0:
        raise ValueError(f"or_scs_decode -> {rc}")
    stats = dict(iterations=int(st[0]), switches=int(st[1]), ops=int(st[2]), expansions=int(st[3]), max_visits=int(st[4]))
    return rc, msg, np.float32(pm.value), cw, stats


def scs_decode_trace(llr: np.ndarray, N: int, K: int, frozen: np.ndarray, *, fast: bool, D: int, L: int,
                     crc_len: int = 0, systematic: bool = False, max_pops: int = 4096):
    """scs_decode with a trace of every pop (test hook).  Returns (status, msg,
    pm, codeword, stats, trace) where trace is a list of (schedule position,
    pm, beta array [N]) per pop, the beta array being the popped path's right
    after its restore; a complete path has schedule position = the number of
    schedule operations."""
    llr = np.ascontiguousarray(llr, dtype=np.float32)
    fr = _u8(frozen)
    msg = np.zeros(K - crc_len, np.uint8)
    cw = np.zeros(N, np.uint8)
    pm = C.c_float(0.0)
    st = np.zeros(5, np.uint64)
    sched = np.zeros(max_pops, np.int32)
    pmt = np.zeros(max_pops, np.float32)
    beta = np.zeros((max_pops, N), np.uint8)
    nt = C.c_int(0)
    rc = _load().or_scs_decode_trace(_p(llr, C.c_float), N, K, _p(fr, C.c_uint8), int(bool(fast)), D, L, crc_len,
                                     int(bool(systematic)), max_pops, _p(sched, C.c_int), _p(pmt, C.c_float),
                                     _p(beta, C.c_uint8), C.byref(nt), _p(msg, C.c_uint8), C.byref(pm),
                                     _p(cw, C.c_uint8), _p(st, C.c_uint64))
    if rc < 0:
        raise ValueError(f"or_scs_decode_trace -> {rc}")
    stats = dict(iterations=int(st[0]), switches=int(st[1]), ops=int(st[2]), expansions=int(st[3]), max_visits=int(st[4]))
    trace = [(int(sched[k]), np.float32(pmt[k]), beta[k].copy()) for k in range(nt.value)]
    return rc, msg, np.float32(pm.value), cw, stats, trace


def scs_decode_batch(llr: np.ndarray, N: int, K: int, frozen: np.ndarray, *, fast: bool, D: int, L: int,
                     crc_len: int = 0, threads: int = 1, scales=None, systematic: bool = False):
    """B frames (rows of llr).  Returns (msg [B,K-crc] u8, pm [B] f32, status [B] i8, stats [B,4] u64).

    ``threads`` > 1 splits the frames into contiguous chunks decoded by host
    threads; each call into the C code decodes its chunk serially.
    """
    llr = np.ascontiguousarray(llr, dtype=np.float32).reshape(-1, N)
    B = llr.shape[0]
    fr = _u8(frozen)
    msg = np.zeros((B, K - crc_len), np.uint8)
    pm = np.zeros(B, np.float32)
    status = np.zeros(B, np.int8)
    stats = np.zeros((B, 4), np.uint64)
    lib = _load()
    sc, scp = _scales_arg(scales)

    def run(lo, hi):
        if hi <= lo:
            return 0
        return lib.or_scs_decode_batch_sx(_p(llr[lo:hi], C.c_float), hi - lo, N, K, _p(fr, C.c_uint8),
                                          int(bool(fast)), D, L, crc_len, scp, int(bool(systematic)),
                                          _p(msg[lo:hi], C.c_uint8), _p(pm[lo:hi], C.c_float),
                                          _p(status[lo:hi], C.c_int8), _p(stats[lo:hi], C.c_uint64))

    threads = max(1, min(int(threads), B))
    if threads == 1:
        rcs = [run(0, B)]
    else:
        bounds = np.linspace(0, B, threads + 1).astype(int)
        rcs = [0] * threads
        ths = [threading.Thread(target=lambda i=i: rcs.__setitem__(i, run(bounds[i], bounds[i + 1]))) for i in range(threads)]
        for th in ths:
            th.start()
        for th in ths:
            th.join()
    if any(r < 0 for r in rcs):
        raise ValueError(f"or_scs_decode_batch -> {rcs}")
    return msg, pm, status, stats


def scs_decode_exact(llr: np.ndarray, N: int, K: int, frozen: np.ndarray, *, D: int, L: int,
                     precision: str = "f64"):
    """Exact-f bit-level SCS without CRC, in double (``f64``) or float
    (``f32``).  Returns (status, codeword, pm)."""
    fr = _u8(frozen)
    cw = np.zeros(N, np.uint8)
    if precision == "f64":
        llr = np.ascontiguousarray(llr, dtype=np.float64)
        pm = C.c_double(0.0)
        rc = _load().or_scs_decode_exact(_p(llr, C.c_double), N, K, _p(fr, C.c_uint8), D, L, _p(cw, C.c_uint8),
                                         C.byref(pm))
    elif precision == "f32":
        llr = np.ascontiguousarray(llr, dtype=np.float32)
        pm = C.c_float(0.0)
        rc = _load().or_scs_decode_exact_f32(_p(llr, C.c_float), N, K, _p(fr, C.c_uint8), D, L, _p(cw, C.c_uint8),
                                             C.byref(pm))
    else:
        raise ValueError("precision is 'f64' or 'f32'")
    if rc < 0:
        raise ValueError(f"or_scs_decode_exact -> {rc}")
    return rc, cw, (float(pm.value) if precision == "f64" else np.float32(pm.value))


def gsc_forward(llr: np.ndarray, u: np.ndarray, scale: np.ndarray) -> np.ndarray:
    """Genie-aided SC leaf LLRs (double) with per-stage f scales."""
    llr = np.ascontiguousarray(llr, dtype=np.float64)
    u = _u8(u)
    scale = np.ascontiguousarray(scale, dtype=np.float64)
    out = np.zeros(llr.size, np.float64)
    rc = _load().or_gsc_forward(_p(llr, C.c_double), _p(u, C.c_uint8), llr.size, _p(scale, C.c_double), _p(out, C.c_double))
    if rc:
        raise ValueError(f"or_gsc_forward -> {rc}")
    return out


def gsc_loss_grad(llr: np.ndarray, u: np.ndarray, frozen: np.ndarray, scale: np.ndarray):
    """Mean BCE over information leaves and its gradient w.r.t. the n scales (double)."""
    llr = np.ascontiguousarray(llr, dtype=np.float64)
    B, N = llr.shape
    u = _u8(u)
    fr = _u8(frozen)
    scale = np.ascontiguousarray(scale, dtype=np.float64)
    grad = np.zeros(scale.size, np.float64)
    loss = C.c_double(0.0)
    rc = _load().or_gsc_loss_grad(_p(llr, C.c_double), _p(u, C.c_uint8), B, N, _p(fr, C.c_uint8), _p(scale, C.c_double),
                                  C.byref(loss), _p(grad, C.c_double))
    if rc:
        raise ValueError(f"or_gsc_loss_grad -> {rc}")
    return float(loss.value), grad
