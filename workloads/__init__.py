"""Seeded synthetic inputs for polar-code decoding: message bits, channel
noise and the BPSK/AWGN channel, plus the per-frame draws of the mixed and
served workloads.

This module holds none of the decoding method's arithmetic (no encoding, no
CRC, no tree updates).  It is the only code that both the CPU oracle side and
the GPU side of a comparison use: each side encodes the messages with its own
encoder and feeds the result through ``bpsk_awgn_llr`` below with the same
noise, so the two sides see the same LLR bytes.

Randomness: numpy's counter-based Philox bit generator, one generator per
(seed, stream, chunk of ``CHUNK`` frames), so any frame can be regenerated on
its own (for sampled checks at full size) and chunks can be drawn by parallel
threads.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

CHUNK = 4096
STREAM_MSG, STREAM_NOISE, STREAM_MIX, STREAM_ARRIVAL = 1, 2, 3, 4


def _gen(seed: int, stream: int, chunk: int) -> np.random.Generator:
    key = (int(seed) << 64) | (int(stream) << 48) | int(chunk)
    return np.random.Generator(np.random.Philox(key=key))


def _threads() -> int:
    return max(1, min(16, os.cpu_count() or 1))


def _chunked(seed: int, stream: int, B: int, first: int, row: int, draw, dtype) -> np.ndarray:
    """Rows [first, first + B) of a chunked stream; ``draw(gen, nrows)`` makes a chunk."""
    out = np.empty((B, row), dtype)
    if B == 0:
        return out
    c0, c1 = first // CHUNK, (first + B - 1) // CHUNK

    def one(c):
        full = draw(_gen(seed, stream, c), CHUNK)
        lo = max(first, c * CHUNK)
        hi = min(first + B, (c + 1) * CHUNK)
        out[lo - first:hi - first] = full[lo - c * CHUNK:hi - c * CHUNK]

    chunks = list(range(c0, c1 + 1))
    if len(chunks) == 1:
        one(chunks[0])
    else:
        with ThreadPoolExecutor(_threads()) as ex:
            list(ex.map(one, chunks))
    return out


def message_bits(seed: int, B: int, kmsg: int, first: int = 0) -> np.ndarray:
    """Uniform message bits, uint8 [B, kmsg], frames first .. first+B-1."""
    return _chunked(seed, STREAM_MSG, B, first, kmsg,
                    lambda g, n: g.integers(0, 2, size=(n, kmsg), dtype=np.uint8), np.uint8)


def awgn_noise(seed: int, B: int, N: int, first: int = 0) -> np.ndarray:
    """Standard normal noise, float32 [B, N], frames first .. first+B-1."""
    return _chunked(seed, STREAM_NOISE, B, first, N,
                    lambda g, n: g.standard_normal((n, N), dtype=np.float32), np.float32)


def sigma_from_ebn0(ebn0_db: float, rate: float) -> float:
    """Noise standard deviation for BPSK at Eb/N0 (dB) and code rate K/N."""
    return math.sqrt(1.0 / (2.0 * rate * 10.0 ** (ebn0_db / 10.0)))


def channel_constants(sigma: float) -> tuple[np.float32, np.float32]:
    """(sigma, 2/sigma^2) rounded to float32, as used by ``bpsk_awgn_llr``."""
    return np.float32(sigma), np.float32(2.0 / (sigma * sigma))


def bpsk_awgn_llr(codeword: np.ndarray, noise: np.ndarray, sigma) -> np.ndarray:
    """LLR = (2/sigma^2) * ((1 - 2c) + sigma * z), every step in float32.

    ``sigma`` is a scalar or one value per frame.  The operation order is
    fixed (multiply, add, multiply, each rounded to float32) so that another
    implementation of the same three steps gives the same bytes.
    """
    cw = np.asarray(codeword)
    z = np.asarray(noise, dtype=np.float32)
    sig = np.asarray(sigma, dtype=np.float64)
    if sig.ndim == 0:
        s, k = channel_constants(float(sig))
    else:
        s = sig.astype(np.float32)[:, None]
        k = (2.0 / (sig * sig)).astype(np.float32)[:, None]
    x = np.where(cw.astype(bool), np.float32(-1.0), np.float32(1.0)).astype(np.float32)
    y = np.add(x, np.multiply(s, z, dtype=np.float32), dtype=np.float32)
    return np.multiply(k, y, dtype=np.float32)


def integer_llr(codeword: np.ndarray, noise: np.ndarray, sigma: float, scale: float = 4.0) -> np.ndarray:
    """Integer-valued float32 LLRs round(scale * (2/sigma^2) * y): all sums of a
    few hundred of them are exact in float32, which makes the path-metric
    identities exact."""
    y = np.where(np.asarray(codeword).astype(bool), -1.0, 1.0) + sigma * np.asarray(noise, np.float64)
    return np.rint(scale * (2.0 / sigma ** 2) * y).astype(np.float32)


# ---- mixed-size workload (batching and serving configs) -------------------
MIX_N = (128, 256, 512, 1024, 2048)
MIX_RATES = ((1, 4), (1, 3), (1, 2), (2, 3), (3, 4))
MIX_D = (8, 16, 32, 64)


def mixed_frames(seed: int, B: int, ebn0_lo: float = 1.0, ebn0_hi: float = 4.0):
    """Per-frame draws for the mixed workload, in a seeded shuffled order.

    Returns a dict of arrays of length B: N, K (round(N * r)), D, ebn0_db.
    N, r and D are uniform over their sets, Eb/N0 uniform on [lo, hi]; the
    frame order is then shuffled with a Philox-seeded Fisher-Yates pass.
    """
    g = _gen(seed, STREAM_MIX, 0)
    ni = g.integers(0, len(MIX_N), size=B)
    ri = g.integers(0, len(MIX_RATES), size=B)
    di = g.integers(0, len(MIX_D), size=B)
    eb = g.uniform(ebn0_lo, ebn0_hi, size=B)
    Ns = np.asarray(MIX_N, np.int64)[ni]
    num = np.asarray([r[0] for r in MIX_RATES], np.int64)[ri]
    den = np.asarray([r[1] for r in MIX_RATES], np.int64)[ri]
    Ks = (Ns * num + den // 2) // den  # round half up of N * r
    Ds = np.asarray(MIX_D, np.int64)[di]
    perm = g.permutation(B)
    return dict(N=Ns[perm], K=Ks[perm], D=Ds[perm], ebn0_db=eb[perm])


def poisson_arrivals(seed: int, rate_hz: float, duration_s: float) -> np.ndarray:
    """Arrival times (s) of a Poisson process of the given rate over [0, duration)."""
    g = _gen(seed, STREAM_ARRIVAL, 0)
    n_guess = int(rate_hz * duration_s * 1.1 + 10 * math.sqrt(rate_hz * duration_s) + 16)
    t = np.cumsum(g.exponential(1.0 / rate_hz, size=n_guess))
    while t[-1] < duration_s:
        more = np.cumsum(g.exponential(1.0 / rate_hz, size=n_guess)) + t[-1]
        t = np.concatenate([t, more])
    return t[t < duration_s]
