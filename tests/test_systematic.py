"""Systematic encoding (Sec. 2.2.2, Sec. 4): the codeword carries the
information bits on the information set and the decoder reads the message
straight from its final beta array.

CPU part: the oracle's systematic encoder against brute force over all
codewords of tiny codes and against the textbook generator matrix, and its
decoder against the non-systematic search (identical without a CRC) and the
noiseless round trip.  GPU part: the library's systematic encoder and decoder
against the oracle, bit for bit."""
import itertools

import numpy as np
import pytest

import textbook as tb
import workloads as W


def _frozen_sets(N):
    import oracle

    sets = [oracle.construct(N, K, snr) for K in (1, N // 4, N // 2, 3 * N // 4, N - 1) for snr in (0.0, 3.0)]
    for info in ([1, 3, 7], [1, 7], [2, 4, 6, 7], [0, 5]):  # sets not closed under the bit-subset order
        fr = np.ones(N, np.uint8)
        fr[info] = 0
        sets.append(fr)
    return sets


@pytest.mark.parametrize("N", [8, 16])
def test_systematic_encoder_brute_force(oracle_lib, N):
    """The oracle's codeword is the one codeword whose bits on A are the info bits."""
    for fr in _frozen_sets(N):
        A = np.nonzero(fr == 0)[0]
        cws = tb.all_codewords(N, fr)
        for info in itertools.islice(itertools.product((0, 1), repeat=A.size), 64):
            info = np.array(info, np.uint8)
            x = oracle_lib.encode_sys(info, N, fr)
            match = np.nonzero((cws[:, A] == info).all(axis=1))[0]
            assert match.size == 1
            assert np.array_equal(x, cws[match[0]])


def test_systematic_encoder_generator_matrix(oracle_lib):
    """PC(1024,512): u = x G (G an involution) is zero on the frozen set and x_A = info."""
    N, K = 1024, 512
    fr = oracle_lib.construct(N, K, 0.0)
    G = tb.generator_matrix(N)
    info = W.message_bits(31, 3, K)
    for b in range(3):
        x = oracle_lib.encode_sys(info[b], N, fr)
        u = (x.astype(np.int64) @ G) % 2
        assert not u[fr == 1].any()
        assert np.array_equal(x[fr == 0], info[b])


@pytest.mark.parametrize("crc", [0, 8, 16])
def test_systematic_message_with_crc(oracle_lib, crc):
    """Message + CRC (long division) sit on the information set, in order."""
    N, K = 256, 128
    fr = oracle_lib.construct(N, K, 0.0)
    poly = {8: 0x07, 16: 0x1021}.get(crc)
    msg = W.message_bits(7, 4, K - crc)
    for b in range(4):
        x = oracle_lib.encode_msg(msg[b], N, K, fr, crc, systematic=True)
        info = x[fr == 0]
        assert np.array_equal(info[: K - crc], msg[b])
        if crc:
            reg = tb.crc_longdiv(msg[b], crc, poly)
            assert [int(v) for v in info[K - crc:]] == [(reg >> (crc - 1 - j)) & 1 for j in range(crc)]


@pytest.mark.parametrize("fast", [False, True])
@pytest.mark.parametrize("crc", [0, 16])
def test_systematic_noiseless_round_trip(oracle_lib, fast, crc):
    N, K = 256, 128
    fr = oracle_lib.construct(N, K, 0.0)
    msg = W.message_bits(9, 6, K - crc)
    cw = oracle_lib.encode_batch(msg, N, K, fr, crc, systematic=True)
    llr = W.bpsk_awgn_llr(cw, np.zeros(cw.shape, np.float32), 0.7)
    out, pm, st, _ = oracle_lib.scs_decode_batch(llr, N, K, fr, fast=fast, D=8, L=4, crc_len=crc, systematic=True)
    assert np.array_equal(out, msg)
    assert not st.any() and not pm.any()


@pytest.mark.parametrize("fast", [False, True])
def test_systematic_search_equals_nonsystematic(oracle_lib, fast):
    """Without a CRC the search does not depend on the encoding: same pm,
    status and codeword estimate; the message is that estimate on A, and the
    counted work differs only by the output re-encode (n N/32)."""
    N, K, D, L = 256, 128, 16, 4
    fr = oracle_lib.construct(N, K, 0.0)
    A = np.nonzero(fr == 0)[0]
    msg = W.message_bits(13, 24, K)
    cw = oracle_lib.encode_batch(msg, N, K, fr, 0, systematic=True)
    llr = W.bpsk_awgn_llr(cw, W.awgn_noise(13, 24, N), W.sigma_from_ebn0(1.5, K / N))
    for b in range(24):
        r0, m0, p0, c0, s0 = oracle_lib.scs_decode(llr[b], N, K, fr, fast=fast, D=D, L=L)
        r1, m1, p1, c1, s1 = oracle_lib.scs_decode(llr[b], N, K, fr, fast=fast, D=D, L=L, systematic=True)
        assert r0 == r1 and p0.view(np.uint32) == p1.view(np.uint32)
        assert np.array_equal(c0, c1)
        assert np.array_equal(m1, c1[A])
        assert np.array_equal(m0, oracle_lib.encode(c0)[A])
        assert s0["ops"] - s1["ops"] == 8 * (N // 32)
        assert s0["iterations"] == s1["iterations"] and s0["switches"] == s1["switches"]


# ----------------------------------------------------------------- GPU part
def _gpu_ready():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1809_03606_gb300 as ps

    ps.load(build_if_missing=True)
    return torch, ps


@pytest.mark.gpu
@pytest.mark.parametrize("N,K,crc", [(256, 128, 0), (1024, 512, 16), (512, 340, 8)])
def test_gpu_systematic_encoder(oracle_lib, N, K, crc):
    torch, ps = _gpu_ready()
    fr = oracle_lib.construct(N, K, 0.0)
    plan = ps.Plan(N, K, fr, fast_nodes=True, crc=crc, systematic=True)
    B = 300
    msg = W.message_bits(N + crc, B, K - crc)
    d_cw = torch.empty((B, plan.words), dtype=torch.int32, device="cuda")
    ps.polar_encode_batch(plan, torch.from_numpy(ps.pack_bits(msg)).cuda(), d_cw)
    torch.cuda.synchronize()
    got = ps.unpack_bits(d_cw.cpu().numpy(), N)
    ref = oracle_lib.encode_batch(msg, N, K, fr, crc, systematic=True)
    assert np.array_equal(got, ref)


@pytest.mark.gpu
@pytest.mark.parametrize("N,K,crc,D,L,fast", [(256, 128, 0, 16, 4, False), (1024, 512, 16, 32, 32, True),
                                              (512, 340, 8, 64, 64, True)])
def test_gpu_systematic_decoder_parity(oracle_lib, N, K, crc, D, L, fast):
    torch, ps = _gpu_ready()
    fr = oracle_lib.construct(N, K, 0.0)
    plan = ps.Plan(N, K, fr, fast_nodes=fast, crc=crc, systematic=True)
    B = 1500
    msg = W.message_bits(3 * N + D, B, K - crc)
    cw = oracle_lib.encode_batch(msg, N, K, fr, crc, systematic=True)
    z = W.awgn_noise(3 * N + D, B, N)
    for ebn0 in (1.0, 2.5):
        llr = W.bpsk_awgn_llr(cw, z, W.sigma_from_ebn0(ebn0, K / N))
        m_ref, pm_ref, st_ref, stats_ref = oracle_lib.scs_decode_batch(llr, N, K, fr, fast=fast, D=D, L=L,
                                                                       crc_len=crc, threads=8, systematic=True)
        info, pm, st, stats = ps.decode(plan, torch.from_numpy(llr).cuda(), D, L, with_stats=True)
        torch.cuda.synchronize()
        assert np.array_equal(ps.unpack_bits(info.cpu().numpy(), K - crc), m_ref)
        assert np.array_equal(pm.cpu().numpy().view(np.uint32), pm_ref.view(np.uint32))
        assert np.array_equal(st.cpu().numpy(), st_ref)
        s = stats.cpu().numpy().astype(np.int64) & 0xFFFFFFFF
        assert np.array_equal(s[:, 2], stats_ref[:, 2].astype(np.int64))
