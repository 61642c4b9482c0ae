"""Exact-f stack decoding: the box-plus f of Eq. llrcalc (before its min-sum
approximation) and the exact leaf metric ln(1 + exp(-(1 - 2u) alpha)).

CPU part: the oracle's float instantiation against closed forms, against
maximum likelihood over all codewords of tiny codes, and against its double
instantiation.  GPU part: the library's exact-f decoder against the float
oracle (same decisions, path metrics within 1e-5 relative)."""
import numpy as np
import pytest

import textbook as tb
import workloads as W


def _llr(N, K, fr, B, ebn0, seed, oracle_lib):
    msg = W.message_bits(seed, B, K)
    cw = oracle_lib.encode_batch(msg, N, K, fr, 0)
    return W.bpsk_awgn_llr(cw, W.awgn_noise(seed, B, N), W.sigma_from_ebn0(ebn0, K / N))


def test_exact_two_leaf_closed_form(oracle_lib):
    """N = 2, both leaves information, unbounded stack: the decoder returns the
    better of the four (u0, u1) words; its metric is the closed form
    softplus(-(1-2u0) boxplus(l0, l1)) + softplus(-(1-2u1) (l1 + (1-2u0) l0)),
    boxplus(a, b) = 2 atanh(tanh(a/2) tanh(b/2))."""
    rng = np.random.default_rng(5)
    fr = np.zeros(2, np.uint8)
    for _ in range(40):
        l = rng.uniform(-6, 6, 2)
        best = None
        for u0 in (0, 1):
            for u1 in (0, 1):
                bp = 2 * np.arctanh(np.tanh(l[0] / 2) * np.tanh(l[1] / 2))
                m = np.logaddexp(0, -(1 - 2 * u0) * bp) + np.logaddexp(0, -(1 - 2 * u1) * (l[1] + (1 - 2 * u0) * l[0]))
                best = m if best is None else min(best, m)
        for prec, tol in (("f64", 1e-12), ("f32", 1e-5)):
            st, cw, pm = oracle_lib.scs_decode_exact(l, 2, 2, fr, D=8, L=8, precision=prec)
            assert st == 0 and abs(float(pm) - best) <= tol * max(1.0, best)


@pytest.mark.parametrize("N,K", [(8, 4), (16, 8), (16, 11)])
def test_exact_f32_search_is_ml(oracle_lib, N, K):
    """Unbounded stack and visit cap: the float search returns the likelihood
    ML codeword (brute force) with its metric to float accuracy."""
    fr = oracle_lib.construct(N, K, 0.0)
    llr = _llr(N, K, fr, 30, 1.0, 40 + N + K, oracle_lib)
    big = 1 << (K + 1)
    cws = tb.all_codewords(N, fr).astype(np.float64)
    for b in range(30):
        st, cw, pm = oracle_lib.scs_decode_exact(llr[b], N, K, fr, D=big, L=big, precision="f32")
        z = -(1.0 - 2.0 * cws) * llr[b].astype(np.float64)[None, :]
        metrics = np.logaddexp(0.0, z).sum(axis=1)
        ml = float(metrics.min())
        assert st == 0
        assert abs(float(pm) - ml) <= 1e-5 * max(1.0, ml)
        # the returned word is optimal to float accuracy (a near-tie may pick another optimum)
        mine = float(np.logaddexp(0.0, -(1.0 - 2.0 * cw) * llr[b].astype(np.float64)).sum())
        assert mine - ml <= 1e-5 * max(1.0, ml)


@pytest.mark.parametrize("N,K,D,L", [(16, 8, 4, 2), (64, 32, 8, 4), (256, 128, 16, 4)])
def test_exact_f32_agrees_with_f64(oracle_lib, N, K, D, L):
    """The float and double instantiations make the same decisions on random
    frames and their metrics agree to 1e-5 relative."""
    fr = oracle_lib.construct(N, K, 0.0)
    B = 60 if N < 256 else 20
    llr = _llr(N, K, fr, B, 1.5, 7 * N + D, oracle_lib)
    for b in range(B):
        s64, c64, p64 = oracle_lib.scs_decode_exact(llr[b].astype(np.float64), N, K, fr, D=D, L=L)
        s32, c32, p32 = oracle_lib.scs_decode_exact(llr[b], N, K, fr, D=D, L=L, precision="f32")
        assert s64 == s32 == 0
        assert np.array_equal(c64, c32)
        assert abs(float(p32) - p64) <= 1e-5 * max(1.0, abs(p64))


def test_exact_noiseless_round_trip(oracle_lib):
    N, K = 128, 64
    fr = oracle_lib.construct(N, K, 0.0)
    msg = W.message_bits(3, 5, K)
    cw = oracle_lib.encode_batch(msg, N, K, fr, 0)
    llr = W.bpsk_awgn_llr(cw, np.zeros(cw.shape, np.float32), 0.6)
    for b in range(5):
        st, out, pm = oracle_lib.scs_decode_exact(llr[b], N, K, fr, D=4, L=2, precision="f32")
        assert st == 0 and np.array_equal(out, cw[b])


# ----------------------------------------------------------------- GPU part
@pytest.mark.gpu
@pytest.mark.parametrize("N,K,D,L,B", [(64, 32, 8, 4, 400), (256, 128, 16, 4, 200), (512, 256, 32, 8, 60),
                                       (1024, 512, 32, 32, 40), (256, 128, 48, 8, 100)])
def test_gpu_exact_f_parity(oracle_lib, N, K, D, L, B):
    """polar_plan_set_exact: same decisions as the float oracle (decoded
    message, status) and path metrics within 1e-5 relative (the two sides'
    log1p/exp differ in the last bits)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1809_03606_gb300 as ps

    ps.load(build_if_missing=True)
    fr = oracle_lib.construct(N, K, 0.0)
    A = np.nonzero(fr == 0)[0]
    plan = ps.Plan(N, K, fr, fast_nodes=False, exact=True)
    for ebn0 in (1.0, 2.5):
        llr = _llr(N, K, fr, B, ebn0, 11 * N + D, oracle_lib)
        info, pm, st = ps.decode(plan, torch.from_numpy(llr).cuda(), D, L)
        torch.cuda.synchronize()
        got = ps.unpack_bits(info.cpu().numpy(), K)
        pm = pm.cpu().numpy()
        st = st.cpu().numpy()
        for b in range(B):
            rs, cw, rpm = oracle_lib.scs_decode_exact(llr[b], N, K, fr, D=D, L=L, precision="f32")
            assert rs == 0 and st[b] == 0
            assert np.array_equal(got[b], oracle_lib.encode(cw)[A]), b
            assert abs(float(pm[b]) - float(rpm)) <= 1e-5 * max(1.0, abs(float(rpm))), (b, pm[b], rpm)
