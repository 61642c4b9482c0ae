"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names the passage it checks.  None of them re-types the oracle's
formulas: the references are the paper's worked example (Figs. encoder,
fsscsch, fsscsbmem), textbook definitions written independently in
``textbook.py`` (Kronecker-power generator, recursive SC, CRC long division,
brute-force ML), closed-form identities and invariants.
"""
import math

import numpy as np
import pytest

import textbook as tb
import workloads as W
from conftest import read_golden


def _frames(oracle, N, K, crc, B, ebn0, seed, integer=False):
    fr = oracle.construct(N, K, 0.0)
    msg = W.message_bits(seed, B, K - crc)
    cw = oracle.encode_batch(msg, N, K, fr, crc)
    sig = W.sigma_from_ebn0(ebn0, K / N)
    z = W.awgn_noise(seed, B, N)
    llr = W.integer_llr(cw, z, sig) if integer else W.bpsk_awgn_llr(cw, z, sig)
    return fr, msg, cw, llr


# ---------------------------------------------------------------- construction
def test_construct_matches_fig_encoder(oracle_lib):
    """Fig. encoder: PC(8,4) has information set {3,5,6,7}."""
    info = [int(v) for v in read_golden("pc8_4_encoder.txt")[0][1:]]
    fr = oracle_lib.construct(8, 4, 0.0)
    assert sorted(np.nonzero(fr == 0)[0].tolist()) == info


@pytest.mark.parametrize("N", [4, 16, 64, 256, 1024])
@pytest.mark.parametrize("snr", [-2.0, 0.0, 3.0])
def test_construct_against_z_domain(oracle_lib, N, snr):
    """Bhattacharyya recursion evaluated directly in the z domain (plain floats)
    must select the same K most reliable positions, up to near-ties."""
    for K in (1, N // 4, N // 2, 3 * N // 4, N):
        fr = oracle_lib.construct(N, K, snr)
        assert int(fr.sum()) == N - K
        z = [math.exp(-(K / N) * 10 ** (snr / 10))]
        while len(z) < N:
            z = [v for p in z for v in (2 * p - p * p, p * p)]
        z = np.array(z)
        info = np.nonzero(fr == 0)[0]
        frozen = np.nonzero(fr == 1)[0]
        if info.size and frozen.size:
            # every information position at least as reliable as every frozen one
            assert z[info].max() <= z[frozen].min() * (1 + 1e-9) + 1e-300


@pytest.mark.parametrize("N,K", [(16, 8), (64, 20), (256, 128), (1024, 512)])
def test_construct_partial_order(oracle_lib, N, K):
    """Invariant: if i is an information index, so is every j whose binary
    expansion contains i's (a g-step never makes a channel worse than an f-step)."""
    fr = oracle_lib.construct(N, K, 0.0)
    info = set(np.nonzero(fr == 0)[0].tolist())
    for i in info:
        for j in range(N):
            if (j & i) == i:
                assert j in info, (i, j)


# ------------------------------------------------------------------ encoding
def test_encoder_matches_fig_encoder_wiring(oracle_lib):
    """Fig. encoder: stage s XORs index i+2^(s-1) into i, in the drawn pairs."""
    rows = [r for r in read_golden("pc8_4_encoder.txt") if r[0] == "stage"]
    rng = np.random.default_rng(7)
    for _ in range(64):
        u = rng.integers(0, 2, 8).astype(np.uint8)
        x = u.copy()
        for stage in (1, 2, 3):
            for _, st, recv, src in [r for r in rows if int(r[1]) == stage]:
                x[int(recv)] ^= x[int(src)]
        assert np.array_equal(oracle_lib.encode(u), x)


@pytest.mark.parametrize("N", [2, 8, 32, 256])
def test_encoder_is_kronecker_power(oracle_lib, N):
    """c = u F^{(x)n} (Sec. 2.1) against the Kronecker-product matrix; F^{(x)n}
    squared is the identity over GF(2)."""
    rng = np.random.default_rng(N)
    for _ in range(16):
        u = rng.integers(0, 2, N).astype(np.uint8)
        c = oracle_lib.encode(u)
        assert np.array_equal(c, tb.encode_matrix(u))
        assert np.array_equal(oracle_lib.encode(c), u)


def test_beta_memory_layout_fig_fsscsbmem(oracle_lib):
    """Fig. fsscsbmem: node (2,0) in slots 0-3, node (2,1) in slots 4-7, then the
    in-place beta operation leaves node (3,0) = [beta(2,0) xor beta(2,1), beta(2,1)],
    which is the codeword."""
    rows = read_golden("pc8_4_beta_memory.txt")
    assert [r[0] for r in rows] == ["after_REP", "after_SPC", "after_beta"]
    fr = oracle_lib.construct(8, 4, 0.0)
    rng = np.random.default_rng(3)
    for _ in range(16):
        msg = rng.integers(0, 2, 4).astype(np.uint8)
        cw = oracle_lib.encode_msg(msg, 8, 4, fr)
        u = np.zeros(8, np.uint8)
        u[fr == 0] = msg
        b20, b21 = tb.encode_matrix(u[0:4]), tb.encode_matrix(u[4:8])
        assert np.array_equal(cw, np.concatenate([b20 ^ b21, b21]))
        llr = np.where(cw == 1, -8.0, 8.0).astype(np.float32)
        st, m, pm, xhat, _ = oracle_lib.scs_decode(llr, 8, 4, fr, fast=True, D=4, L=4)
        assert st == 0 and pm == 0.0 and np.array_equal(xhat, cw) and np.array_equal(m, msg)


def test_beta_memory_slots_fig_fsscsbmem(oracle_lib):
    """Fig. fsscsbmem, slot by slot: the golden file names, for each step of the
    PC(8,4) schedule, the node whose estimate the in-place beta array holds and
    its slots.  The oracle's beta array of the path popped right after that
    step must hold exactly the node's partial-sum estimate there (the
    Kronecker-power encoding of the node's leaves, Sec. 2.2.1), and, after the
    REP node, the SPC slots must still be untouched (zero)."""
    rows = read_golden("pc8_4_beta_memory.txt")
    sched = [(op, int(l), int(p)) for op, l, p in read_golden("pc8_4_fssc_schedule.txt")]
    after = {"after_REP": sched.index(("REP", 2, 0)) + 1, "after_SPC": sched.index(("SPC", 2, 1)) + 1,
             "after_beta": len(sched)}
    fr = oracle_lib.construct(8, 4, 0.0)
    rng = np.random.default_rng(4)
    for _ in range(24):
        msg = rng.integers(0, 2, 4).astype(np.uint8)
        cw = oracle_lib.encode_msg(msg, 8, 4, fr)
        u = np.zeros(8, np.uint8)
        u[fr == 0] = msg
        llr = np.where(cw == 1, -8.0, 8.0).astype(np.float32)
        st, m, pm, xhat, stats, trace = oracle_lib.scs_decode_trace(llr, 8, 4, fr, fast=True, D=1, L=4)
        assert st == 0 and np.array_equal(m, msg)
        popped = {t: beta for t, _, beta in trace}
        for step, lam, phi, first, last in rows:
            lam, phi, first, last = int(lam), int(phi), int(first), int(last)
            Lam = 1 << lam
            assert (first, last) == (phi * Lam, (phi + 1) * Lam - 1)  # the slots of node (lambda, phi)
            beta = popped[after[step]]
            assert np.array_equal(beta[first:last + 1], tb.encode_matrix(u[first:last + 1])), (step, msg)
            if step == "after_REP":
                assert not np.any(beta[last + 1:])
        assert np.array_equal(popped[after["after_beta"]], cw)


def _hand_cases():
    cases, cur = [], None
    for row in read_golden("op_counts_hand.txt"):
        key, vals = row[0], row[1:]
        if key == "case":
            cur = dict(name=vals[0], steps=[])
            cases.append(cur)
        elif key == "step":
            cur["steps"].append(int(vals[0]))
        elif key in ("code", "frozen", "stack", "total", "codeword"):
            cur[key] = [int(v) for v in vals]
        elif key == "llr":
            cur[key] = np.array([float(v) for v in vals], np.float32)
    return cases


@pytest.mark.parametrize("case", _hand_cases(), ids=lambda c: c["name"])
def test_operation_counts_derived_by_hand(oracle_lib, case):
    """The operation counters (the numerator of the roofline fraction) against
    counts worked out by hand from the counting convention for the worked
    example of Fig. fsscsch and two small bit-level codes, with and without a
    path switch (one of them with an alpha recompute below the root)."""
    N, K, fast = case["code"]
    D, L = case["stack"]
    ops, pops, switches, exps, pm_want = case["total"]
    assert sum(case["steps"]) == ops  # the file's own arithmetic
    fr = np.array(case["frozen"], np.uint8)
    st, m, pm, xhat, stats = oracle_lib.scs_decode(case["llr"], N, K, fr, fast=bool(fast), D=D, L=L)
    assert st == 0
    assert (stats["ops"], stats["iterations"], stats["switches"], stats["expansions"]) == (ops, pops, switches, exps)
    assert float(pm) == float(pm_want)
    assert np.array_equal(xhat, np.array(case["codeword"], np.uint8))
    assert tb.discrepancy(case["llr"], xhat) == float(pm)  # and the metric is the codeword's discrepancy


def test_crc_failure_returns_first_complete_path(oracle_lib):
    """Sec. 2.2.5 with reading R12: after L complete paths have failed the CRC,
    the decoder returns the FIRST complete path popped (status CRC_FAIL), not
    the last or the best one.  Frames are chosen where two different complete
    paths were popped and both fail the CRC (checked by long division)."""
    N, K, crc, D, L = 64, 32, 8, 32, 2
    fr, msg, cw, llr = _frames(oracle_lib, N, K, crc, 400, 0.0, seed=51)
    nops = len(oracle_lib.schedule(N, fr, True))
    checked = 0
    for b in range(llr.shape[0]):
        st, m, pm, xhat, stats, trace = oracle_lib.scs_decode_trace(llr[b], N, K, fr, fast=True, D=D, L=L,
                                                                    crc_len=crc)
        done = [(p, beta) for t, p, beta in trace if t == nops]
        if st != 1 or len(done) != L or np.array_equal(done[0][1], done[1][1]):
            continue
        for p, beta in done:  # both complete paths fail the CRC
            u = tb.encode_matrix(beta)[fr == 0]
            want = tb.crc_longdiv(u[:K - crc], crc, 0x07)
            got = int("".join(str(int(v)) for v in u[K - crc:]), 2)
            assert got != want
        assert np.array_equal(xhat, done[0][1]) and pm == done[0][0]
        assert not np.array_equal(xhat, done[1][1])
        checked += 1
    assert checked >= 5


# ----------------------------------------------------------------------- CRC
def test_crc_catalogue_check_values(oracle_lib):
    bits = np.unpackbits(np.frombuffer(b"123456789", np.uint8))
    for width, poly, check in read_golden("crc_check_values.txt"):
        assert oracle_lib.crc(bits, int(width)) == int(check, 16)
        assert tb.crc_longdiv(bits, int(width), int(poly, 16)) == int(check, 16)


@pytest.mark.parametrize("width,poly", [(8, 0x07), (16, 0x1021), (24, 0xB2B117)])
def test_crc_is_polynomial_remainder(oracle_lib, width, poly):
    rng = np.random.default_rng(width)
    for n in (1, 7, 33, 496, 1000):
        m = rng.integers(0, 2, n).astype(np.uint8)
        r = oracle_lib.crc(m, width)
        assert r == tb.crc_longdiv(m, width, poly)
        tail = np.array([(r >> (width - 1 - j)) & 1 for j in range(width)], np.uint8)
        assert oracle_lib.crc(np.concatenate([m, tail]), width) == 0  # zero syndrome


# ------------------------------------------------------------------ schedule
def test_schedule_matches_fig_fsscsch(oracle_lib):
    want = [(op, int(l), int(p)) for op, l, p in read_golden("pc8_4_fssc_schedule.txt")]
    fr = oracle_lib.construct(8, 4, 0.0)
    assert oracle_lib.schedule(8, fr, True) == want


@pytest.mark.parametrize("N", [8, 64])
def test_bit_level_schedule_is_sc_order(oracle_lib, N):
    """Fig. scdectree / Alg. reca, recb: the bit-level schedule reaches the leaves
    in index order, computes alpha of every node from its parent before use, and
    combines every odd node into its parent."""
    fr = oracle_lib.construct(N, N // 2, 0.0)
    ops = oracle_lib.schedule(N, fr, False)
    leaves = [p for op, l, p in ops if op.startswith("leaf")]
    assert leaves == list(range(N))
    assert all(l == 0 for op, l, p in ops if op.startswith("leaf"))
    assert sum(op == "alpha" for op, _, _ in ops) == 2 * (N - 1)
    assert sum(op == "beta" for op, _, _ in ops) == N - 1
    assert all(p % 2 == 1 for op, _, p in ops if op == "beta")
    kinds = {op: ("leaf0" if fr[p] else "leaf1") for op, l, p in ops if op.startswith("leaf")}
    for op, l, p in ops:
        if op.startswith("leaf"):
            assert op == ("leaf0" if fr[p] else "leaf1")
    assert kinds


def test_fast_node_classification(oracle_lib):
    """Sec. 2.2.2: R-0 all frozen, R-1 all information, REP only the last leaf
    information, SPC only the first leaf frozen (reading R6 precedence)."""
    cases = {
        (1, 1, 1, 1): "R0", (0, 0, 0, 0): "R1", (1, 1, 1, 0): "REP", (1, 0, 0, 0): "SPC",
        (1, 0): "REP", (0, 0): "R1", (1, 1): "R0",
    }
    for pat, want in cases.items():
        fr = np.array(pat, np.uint8)
        ops = oracle_lib.schedule(fr.size, fr, True)
        assert ops == [(want, int(np.log2(fr.size)), 0)]


# ----------------------------------------------------- decoding equivalences
@pytest.mark.parametrize("N,K", [(16, 8), (64, 32), (256, 128)])
def test_scs_depth1_is_sc(oracle_lib, N, K):
    """SCS with D = 1 extends only the best child at every information leaf:
    it is SC (Sec. 2.2.1); decisions and the float32 path metric agree bit for bit."""
    fr, msg, cw, llr = _frames(oracle_lib, N, K, 0, 200, 1.5, seed=11)
    for b in range(llr.shape[0]):
        u_sc, x_sc, pm_sc = tb.sc_decode(llr[b], fr)
        st, m, pm, xhat, _ = oracle_lib.scs_decode(llr[b], N, K, fr, fast=False, D=1, L=4)
        assert st == 0
        assert np.array_equal(xhat, x_sc)
        assert pm == pm_sc


@pytest.mark.parametrize("N,K", [(64, 32), (256, 128)])
def test_scaled_scs_depth1_is_scaled_sc(oracle_lib, N, K):
    """With per-stage scales on f, SCS(D = 1) is the scaled SC decoder, bit for
    bit; unit scales reproduce the unscaled decoder exactly."""
    fr, msg, cw, llr = _frames(oracle_lib, N, K, 0, 120, 1.5, seed=19)
    n = int(np.log2(N))
    scales = np.random.default_rng(N).uniform(0.5, 1.3, n).astype(np.float32)
    for b in range(llr.shape[0]):
        _, x_sc, pm_sc = tb.sc_decode(llr[b], fr, scales)
        st, m, pm, xhat, _ = oracle_lib.scs_decode(llr[b], N, K, fr, fast=False, D=1, L=4, scales=scales)
        assert np.array_equal(xhat, x_sc) and pm == pm_sc
        st1, m1, pm1, x1, _ = oracle_lib.scs_decode(llr[b], N, K, fr, fast=True, D=8, L=8, scales=np.ones(n))
        st0, m0, pm0, x0, _ = oracle_lib.scs_decode(llr[b], N, K, fr, fast=True, D=8, L=8)
        assert np.array_equal(x1, x0) and pm1 == pm0


@pytest.mark.parametrize("N,K,D", [(64, 32, 8), (256, 128, 16)])
def test_scs_visit_cap_one_is_sc(oracle_lib, N, K, D):
    """L = 1 deletes every older path at each branching: again SC."""
    fr, msg, cw, llr = _frames(oracle_lib, N, K, 0, 100, 1.0, seed=12)
    for b in range(llr.shape[0]):
        _, x_sc, pm_sc = tb.sc_decode(llr[b], fr)
        st, m, pm, xhat, _ = oracle_lib.scs_decode(llr[b], N, K, fr, fast=False, D=D, L=1)
        assert np.array_equal(xhat, x_sc) and pm == pm_sc


@pytest.mark.parametrize("N,K", [(32, 16), (128, 64)])
def test_sc_reduction_with_exact_ties(oracle_lib, N, K):
    """On integer LLRs, leaf LLRs of exactly +-0 give both children the same
    metric.  SC takes HD(0) = 0, the first candidate.  SCS(D = 1) reproduces it
    only if a full stack takes a candidate on a strictly smaller metric (Sec.
    2.2.5, replacement rule); SCS(L = 1) reproduces it only if equal metrics
    pop the newest path and the first candidate is the newest (reading R11)."""
    fr, msg, cw, llr = _frames(oracle_lib, N, K, 0, 300, 0.0, seed=15, integer=True)
    llr = np.rint(llr / 6.0).astype(np.float32)  # small integers: many exact zeros inside the tree
    ties = 0
    for b in range(llr.shape[0]):
        _, x_sc, pm_sc = tb.sc_decode(llr[b], fr)
        for D, L in ((1, 4), (4 * N, 1)):
            st, m, pm, xhat, _ = oracle_lib.scs_decode(llr[b], N, K, fr, fast=False, D=D, L=L)
            assert np.array_equal(xhat, x_sc) and pm == pm_sc, (b, D, L)
        ties += int(np.any(llr[b] == 0))
    assert ties > 50


@pytest.mark.parametrize("fast", [False, True])
def test_visit_cap_bounds_extensions(oracle_lib, fast):
    """Sec. 2.2.5: once L paths have been extended at a length, shorter-or-equal
    paths are removed, so no branching position is ever extended more than L
    times; at low SNR the cap is reached."""
    N, K = 256, 128
    fr, msg, cw, llr = _frames(oracle_lib, N, K, 0, 60, 0.0, seed=16, integer=True)
    reached = 0
    for L in (1, 2, 4):
        for b in range(llr.shape[0]):
            st, m, pm, xhat, stats = oracle_lib.scs_decode(llr[b], N, K, fr, fast=fast, D=64, L=L)
            assert stats["max_visits"] <= L
            reached += stats["max_visits"] == L
    assert reached > 60


@pytest.mark.parametrize("N,K", [(64, 32), (256, 128), (1024, 512)])
def test_fssc_depth1_matches_sc_decisions(oracle_lib, N, K):
    """Fast nodes (Sec. 2.2.2) reproduce SC decisions: R-0, R-1, REP exactly; SPC
    equals SC on the node (asserted empirically).  On integer LLRs the node-level
    path metric equals the leaf-level one (the sums are exact)."""
    fr, msg, cw, llr = _frames(oracle_lib, N, K, 0, 60, 2.0, seed=13)
    for b in range(llr.shape[0]):
        _, x_sc, pm_sc = tb.sc_decode(llr[b], fr)
        st, m, pm, xhat, _ = oracle_lib.scs_decode(llr[b], N, K, fr, fast=True, D=1, L=4)
        assert np.array_equal(xhat, x_sc)
    # integer LLRs have exact ties (zeros, equal magnitudes) where the node
    # decoders and SC may pick different equally good bits; where they agree,
    # the metrics must agree exactly
    fr, msg, cw, llr = _frames(oracle_lib, N, K, 0, 60, 2.0, seed=13, integer=True)
    agree = 0
    for b in range(llr.shape[0]):
        _, x_sc, pm_sc = tb.sc_decode(llr[b], fr)
        st, m, pm, xhat, _ = oracle_lib.scs_decode(llr[b], N, K, fr, fast=True, D=1, L=4)
        if np.array_equal(xhat, x_sc):
            agree += 1
            assert pm == pm_sc
    assert agree >= 0.9 * llr.shape[0]


@pytest.mark.parametrize("fast", [False, True])
@pytest.mark.parametrize("N,K,D,L,crc", [(64, 32, 8, 4, 0), (256, 128, 16, 4, 0), (512, 256, 32, 8, 8), (1024, 512, 32, 32, 16)])
def test_path_metric_identity(oracle_lib, fast, N, K, D, L, crc):
    """Min-sum path metric of any complete path = sum of |L_i| where the codeword
    disagrees with the channel hard decision (Eq. PMupd summed over the tree);
    exact on integer-valued LLRs."""
    fr, msg, cw, llr = _frames(oracle_lib, N, K, crc, 40, 1.5, seed=14, integer=True)
    for b in range(llr.shape[0]):
        st, m, pm, xhat, _ = oracle_lib.scs_decode(llr[b], N, K, fr, fast=fast, D=D, L=L, crc_len=crc)
        assert float(pm) == tb.discrepancy(llr[b], xhat)
        u = tb.encode_matrix(xhat)
        assert not np.any(u[fr == 1])  # a codeword of this code


@pytest.mark.parametrize("N,K", [(8, 4), (16, 8), (16, 5)])
def test_unbounded_minsum_search_is_ml(oracle_lib, N, K):
    """With D and L at least 2^K the best-first search returns a path of minimum
    discrepancy over all 2^K codewords (brute force), i.e. correlation ML."""
    fr = oracle_lib.construct(N, K, 0.0)
    rng = np.random.default_rng(N * 100 + K)
    big = 2 ** (K + 1)
    for _ in range(150):
        llr = rng.integers(-6, 7, N).astype(np.float32)
        st, m, pm, xhat, _ = oracle_lib.scs_decode(llr, N, K, fr, fast=False, D=big, L=big)
        assert st == 0 and float(pm) == tb.minsum_ml_metric(llr, fr)
        assert tb.discrepancy(llr, xhat) == float(pm)


def test_fast_nodes_full_expansion_is_ml(oracle_lib):
    """PC(8,4) splits into REP(4) and SPC(4): both candidate lists are complete
    (2 and 8 words), so the fast search with an unbounded stack is ML too; this
    pins the REP and SPC candidate sets and their path-metric deltas (Sec. 2.2.4)."""
    fr = oracle_lib.construct(8, 4, 0.0)
    rng = np.random.default_rng(5)
    for _ in range(300):
        llr = rng.integers(-9, 10, 8).astype(np.float32)
        st, m, pm, xhat, stats = oracle_lib.scs_decode(llr, 8, 4, fr, fast=True, D=64, L=64)
        assert float(pm) == tb.minsum_ml_metric(llr, fr)
    # R-0(2) R-1(2) SPC(4): R-1 of size 2 has all four patterns as candidates
    fr2 = np.array([1, 1, 0, 0, 1, 0, 0, 0], np.uint8)
    fr3 = np.array([1, 0, 0, 0, 0, 0, 0, 0], np.uint8)  # SPC(8): 8 of 64 candidates; not ML
    for _ in range(100):
        llr = rng.integers(-9, 10, 8).astype(np.float32)
        st, m, pm, xhat, _ = oracle_lib.scs_decode(llr, 8, 5, fr2, fast=True, D=64, L=64)
        assert float(pm) == tb.minsum_ml_metric(llr, fr2)
        st, m, pm, xhat, _ = oracle_lib.scs_decode(llr, 8, 7, fr3, fast=True, D=64, L=64)
        assert float(pm) == tb.minsum_ml_metric(llr, fr3)  # SPC ML is Wagner: one flip


def _node_candidate_minimum(llr, Lam, kind):
    """min over the node's candidate patterns c (left half, right half frozen)
    of the discrepancy of the codeword [c, 0].  The node LLRs are the min-sum
    f of the two halves; candidates follow Sec. 2.2.4 (Chase-II for R-1, the
    8 parity-consistent flips of the 4 least reliable positions for SPC)."""
    a = tb.f_minsum(llr[:Lam], llr[Lam:])
    h = (a < 0).astype(np.uint8)
    order = sorted(range(Lam), key=lambda i: (abs(float(a[i])), i))
    best = None
    if kind == "R1":
        m = order[:2]
        flips = [(), (m[0],), (m[1],), (m[0], m[1])]
    else:
        m = order[:4]
        q = int(h.sum() % 2)
        flips = [tuple(m[j] for j in range(4) if mask >> j & 1) for mask in range(16) if bin(mask).count("1") % 2 == q]
    for fl in flips:
        c = h.copy()
        for i in fl:
            c[i] ^= 1
        x = np.concatenate([c, np.zeros(Lam, np.uint8)])
        d = tb.discrepancy(llr, x)
        best = d if best is None else min(best, d)
    return best


@pytest.mark.parametrize("kind,Lam", [("R1", 4), ("R1", 8), ("SPC", 8), ("SPC", 16)])
def test_fast_node_candidate_sets(oracle_lib, kind, Lam):
    """A fast node followed by a Rate-0 half: with a stack that never drops a
    path, best-first search returns the minimum over exactly the node's candidate
    patterns (Sec. 2.2.4), so a wrong choice of the least reliable positions, a
    wrong parity rule or a wrong delta changes the result."""
    N = 2 * Lam
    fr = np.ones(N, np.uint8)
    fr[:Lam] = 0
    if kind == "SPC":
        fr[0] = 1
    K = int((fr == 0).sum())
    assert oracle_lib.schedule(N, fr, True)[1][0] == kind
    rng = np.random.default_rng(Lam + len(kind))
    for _ in range(300):
        llr = rng.integers(-9, 10, N).astype(np.float32)
        st, m, pm, xhat, _ = oracle_lib.scs_decode(llr, N, K, fr, fast=True, D=64, L=64)
        assert float(pm) == _node_candidate_minimum(llr, Lam, kind)


@pytest.mark.parametrize("N,K", [(8, 4), (16, 6)])
def test_exact_f_search_is_likelihood_ml(oracle_lib, N, K):
    """Exact box-plus f and the exact leaf metric ln(1+exp(-(1-2u)alpha)): the final
    metric is the negative log-likelihood of the codeword, and the unbounded
    search returns its minimum over all codewords (brute force), to 1e-9."""
    fr = oracle_lib.construct(N, K, 0.0)
    rng = np.random.default_rng(N + K)
    big = 2 ** (K + 2)
    for _ in range(100):
        llr = rng.normal(1.0, 1.5, N)
        st, cw, pm = oracle_lib.scs_decode_exact(llr, N, K, fr, D=big, L=big)
        assert st == 0
        ml = tb.exact_ml_metric(llr, fr)
        assert abs(pm - ml) <= 1e-9 * max(1.0, ml)
        z = -(1.0 - 2.0 * cw.astype(np.float64)) * llr
        assert abs(np.logaddexp(0.0, z).sum() - pm) <= 1e-9 * max(1.0, pm)


# ------------------------------------------------------------- round trips
@pytest.mark.parametrize("fast", [False, True])
@pytest.mark.parametrize("N,K,D,L,crc", [(256, 128, 16, 4, 0), (1024, 512, 32, 32, 16), (128, 43, 8, 8, 8),
                                         (2048, 1536, 64, 64, 8), (4, 2, 1, 1, 0)])
def test_noiseless_round_trip(oracle_lib, fast, N, K, D, L, crc):
    """Large-magnitude LLRs with the transmitted signs: every decoder returns the
    message with path metric 0 and status OK."""
    fr = oracle_lib.construct(N, K, 0.0)
    msg = W.message_bits(21, 8, K - crc)
    cw = oracle_lib.encode_batch(msg, N, K, fr, crc)
    llr = W.bpsk_awgn_llr(cw, np.zeros(cw.shape, np.float32), 0.5)
    m, pm, st, stats = oracle_lib.scs_decode_batch(llr, N, K, fr, fast=fast, D=D, L=L, crc_len=crc)
    assert np.array_equal(m, msg) and np.all(pm == 0) and np.all(st == 0)
    assert np.all(stats[:, 1] == 0)  # no path switch


# -------------------------------------------------------------- stack rules
@pytest.mark.parametrize("N,K,D,L,crc", [(256, 128, 16, 4, 8), (1024, 512, 32, 32, 16), (512, 171, 8, 8, 8)])
def test_crc_status_and_bounds(oracle_lib, N, K, D, L, crc):
    """Sec. 2.2.5: status OK implies the returned message passes the CRC; after L
    failures the first complete path is returned (status CRC_FAIL); the number of
    pops is bounded by L per branching node plus the completion pops."""
    fr, msg, cw, llr = _frames(oracle_lib, N, K, crc, 60, 0.5, seed=31)
    nbranch = sum(op in ("leaf1", "REP", "R1", "SPC") for op, _, _ in oracle_lib.schedule(N, fr, True))
    m, pm, st, stats = oracle_lib.scs_decode_batch(llr, N, K, fr, fast=True, D=D, L=L, crc_len=crc)
    assert set(np.unique(st).tolist()) <= {0, 1}
    assert np.any(st == 1)  # at 0.5 dB some frames must fail
    for b in range(m.shape[0]):
        r = oracle_lib.crc(m[b], crc)
        tail_ok = None
        st1, m1, pm1, xhat, _ = oracle_lib.scs_decode(llr[b], N, K, fr, fast=True, D=D, L=L, crc_len=crc)
        u = tb.encode_matrix(xhat)[fr == 0].astype(np.uint8)
        tail = u[K - crc:]
        tail_ok = all(int(tail[j]) == ((r >> (crc - 1 - j)) & 1) for j in range(crc))
        assert tail_ok == (st[b] == 0)
        assert stats[b, 0] <= L * nbranch + 9 * L + 2
    # deterministic: a second run gives the same bytes
    m2, pm2, st2, _ = oracle_lib.scs_decode_batch(llr, N, K, fr, fast=True, D=D, L=L, crc_len=crc, threads=3)
    assert np.array_equal(m, m2) and np.array_equal(pm.view(np.uint32), pm2.view(np.uint32)) and np.array_equal(st, st2)


def test_small_stack_never_beats_large_stack_metric(oracle_lib):
    """A larger stack explores a superset of the paths of a smaller one when no
    path is ever dropped: with D = L*N the returned metric is never worse than
    the D = 1 (SC) metric on integer LLRs."""
    N, K = 128, 64
    fr, msg, cw, llr = _frames(oracle_lib, N, K, 0, 80, 1.0, seed=41, integer=True)
    for b in range(llr.shape[0]):
        _, _, pm1, _, _ = oracle_lib.scs_decode(llr[b], N, K, fr, fast=False, D=1, L=4)
        _, _, pmb, _, _ = oracle_lib.scs_decode(llr[b], N, K, fr, fast=False, D=4 * N, L=4)
        assert pmb <= pm1


# ------------------------------------------------------ genie-aided SC (S2)
def test_gsc_forward_matches_textbook_genie_sc(oracle_lib):
    N = 16
    rng = np.random.default_rng(1)
    for _ in range(20):
        llr = rng.normal(0, 3, N)
        u = rng.integers(0, 2, N).astype(np.uint8)
        scale = rng.uniform(0.5, 1.5, 4)
        assert np.allclose(oracle_lib.gsc_forward(llr, u, scale), tb.genie_leaf_llrs(llr, u, scale), rtol=1e-13, atol=1e-13)


def test_gsc_gradient_matches_finite_differences(oracle_lib):
    """Reverse-mode gradient of the mean BCE w.r.t. the per-stage f scales against
    central finite differences in double precision (N = 16, K = 8)."""
    N, K, B = 16, 8, 32
    fr = oracle_lib.construct(N, K, 0.0)
    rng = np.random.default_rng(2)
    u = np.zeros((B, N), np.uint8)
    u[:, fr == 0] = rng.integers(0, 2, (B, K))
    cw = np.array([oracle_lib.encode(r) for r in u])
    llr = (2.0 / 0.8) * ((1.0 - 2.0 * cw) + 0.9 * rng.normal(size=(B, N)))
    scale = rng.uniform(0.6, 1.2, 4)
    loss, grad = oracle_lib.gsc_loss_grad(llr, u, fr, scale)
    h = 1e-6
    for lam in range(4):
        sp, sm = scale.copy(), scale.copy()
        sp[lam] += h
        sm[lam] -= h
        fd = (oracle_lib.gsc_loss_grad(llr, u, fr, sp)[0] - oracle_lib.gsc_loss_grad(llr, u, fr, sm)[0]) / (2 * h)
        assert abs(fd - grad[lam]) <= 1e-6 * max(1.0, abs(fd)), (lam, fd, grad[lam])
    # closed form at the leaves: loss = mean softplus(-(1-2u) L_leaf)
    leaves = np.array([tb.genie_leaf_llrs(llr[b], u[b], scale) for b in range(B)])
    ref = np.logaddexp(0.0, -(1.0 - 2.0 * u[:, fr == 0]) * leaves[:, fr == 0]).mean()
    assert abs(ref - loss) <= 1e-12
