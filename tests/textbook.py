"""Independent textbook restatements used to pin the oracle.

Nothing here is imported by the oracle or the GPU library.  These are the
plain recursive definitions (Arikan's SC decoder, the Kronecker-power
generator matrix, polynomial long division for CRCs, brute-force maximum
likelihood), written without the schedule/stack machinery of the oracle so
that a mistake in one is not repeated in the other.
"""
from __future__ import annotations

import itertools

import numpy as np

F32 = np.float32


def generator_matrix(N: int) -> np.ndarray:
    """F^{(x)n} with F = [[1, 0], [1, 1]] (Sec. 2.1), as a 0/1 matrix."""
    F = np.array([[1, 0], [1, 1]], dtype=np.int64)
    G = np.array([[1]], dtype=np.int64)
    while G.shape[0] < N:
        G = np.kron(G, F)
    return G


def encode_matrix(u: np.ndarray) -> np.ndarray:
    u = np.asarray(u, dtype=np.int64)
    return (u @ generator_matrix(u.size)) % 2


def crc_longdiv(bits, crc_len: int, poly: int) -> int:
    """Remainder of m(x) x^c divided by g(x) = x^c + poly(x), over GF(2)."""
    m = 0
    for b in bits:
        m = (m << 1) | (int(b) & 1)
    m <<= crc_len
    g = (1 << crc_len) | poly
    for sh in range(m.bit_length() - 1, crc_len - 1, -1):
        if (m >> sh) & 1:
            m ^= g << (sh - crc_len)
    return m


def f_minsum(a, b):
    a = np.asarray(a, F32)
    b = np.asarray(b, F32)
    m = np.minimum(np.abs(a), np.abs(b))
    return np.where(np.signbit(a) ^ np.signbit(b), -m, m).astype(F32)


def sc_decode(llr: np.ndarray, frozen: np.ndarray, scales=None):
    """Arikan's recursive SC decoder with min-sum f, float32 throughout.

    Returns (u_hat, codeword, pm) where pm accumulates |alpha| at every leaf
    whose decision differs from the hard decision of its LLR (Eq. PMupd).
    ``scales[lambda]`` (optional) multiplies the f output of a child at stage
    lambda.
    """
    pm = [F32(0.0)]

    def rec(alpha, fr):
        n = alpha.size
        if n == 1:
            a = alpha[0]
            h = 1 if a < 0 else 0
            u = 0 if fr[0] else h
            if u != h:
                pm[0] = F32(pm[0] + np.abs(a))
            return np.array([u], np.uint8), np.array([u], np.uint8)
        h = n // 2
        a, b = alpha[:h], alpha[h:]
        fv = f_minsum(a, b)
        if scales is not None:
            fv = (F32(scales[int(np.log2(h))]) * fv).astype(F32)
        ul, xl = rec(fv, fr[:h])
        right = np.where(xl.astype(bool), (b - a).astype(F32), (b + a).astype(F32)).astype(F32)
        ur, xr = rec(right, fr[h:])
        return np.concatenate([ul, ur]), np.concatenate([xl ^ xr, xr])

    u, x = rec(np.asarray(llr, F32), np.asarray(frozen).astype(bool))
    return u, x, pm[0]


def genie_leaf_llrs(llr: np.ndarray, u: np.ndarray, scale=None) -> np.ndarray:
    """Leaf LLRs of SC when every decision is the transmitted bit (float64).

    ``scale[lambda]`` multiplies the f output written at stage lambda.
    """
    n = int(np.log2(llr.size))
    scale = np.ones(n) if scale is None else np.asarray(scale, np.float64)
    out = np.zeros(llr.size)

    def rec(alpha, uu, s):
        m = alpha.size
        if m == 1:
            out[s] = alpha[0]
            return np.array([uu[0]], np.int64)
        h = m // 2
        lam = int(np.log2(h))
        a, b = alpha[:h], alpha[h:]
        fab = np.where((a < 0) ^ (b < 0), -1.0, 1.0) * np.minimum(np.abs(a), np.abs(b))
        xl = rec(scale[lam] * fab, uu[:h], s)
        xr = rec(np.where(xl.astype(bool), b - a, b + a), uu[h:], s + h)
        return np.concatenate([xl ^ xr, xr])

    rec(np.asarray(llr, np.float64), np.asarray(u, np.int64), 0)
    return out


def all_codewords(N: int, frozen: np.ndarray) -> np.ndarray:
    info = np.nonzero(np.asarray(frozen) == 0)[0]
    G = generator_matrix(N)
    words = []
    for bits in itertools.product((0, 1), repeat=info.size):
        u = np.zeros(N, np.int64)
        u[info] = bits
        words.append((u @ G) % 2)
    return np.array(words, np.uint8)


def minsum_ml_metric(llr: np.ndarray, frozen: np.ndarray) -> float:
    """min over codewords of sum_{i: x_i != HD(L_i)} |L_i| (float64)."""
    cws = all_codewords(llr.size, frozen)
    h = (np.asarray(llr) < 0).astype(np.uint8)
    return float(np.min(((cws != h) * np.abs(np.asarray(llr, np.float64))).sum(axis=1)))


def exact_ml_metric(llr: np.ndarray, frozen: np.ndarray) -> float:
    """min over codewords of sum_i ln(1 + exp(-(1 - 2x_i) L_i))  (negative log-likelihood)."""
    cws = all_codewords(llr.size, frozen).astype(np.float64)
    z = -(1.0 - 2.0 * cws) * np.asarray(llr, np.float64)[None, :]
    return float(np.min(np.logaddexp(0.0, z).sum(axis=1)))


def discrepancy(llr: np.ndarray, codeword: np.ndarray) -> float:
    h = (np.asarray(llr) < 0).astype(np.uint8)
    return float(((np.asarray(codeword) != h) * np.abs(np.asarray(llr, np.float64))).sum())
