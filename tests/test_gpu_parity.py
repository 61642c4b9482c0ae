"""GPU parity: the CUDA decoder and encoder against the CPU oracle, through the
C ABI, on identical seeded inputs.

The bar is bit-exact: decoded message bits, float32 path metric bits, frame
status and the per-frame counters (pops, path switches, counted operations,
expansions) must all equal the oracle's, because both sides apply the same
float32 operations in the same order (halving-order sums, no FMA)."""
import numpy as np
import pytest

import paper_1809_03606_gb300 as ps
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    ps.load(build_if_missing=True)


def make_frames(oracle, N, K, crc, B, ebn0, seed, integer=False, frozen=None):
    fr = oracle.construct(N, K, 0.0) if frozen is None else frozen
    msg = W.message_bits(seed, B, K - crc)
    cw = oracle.encode_batch(msg, N, K, fr, crc)
    sig = W.sigma_from_ebn0(ebn0, K / N)
    z = W.awgn_noise(seed, B, N)
    llr = W.integer_llr(cw, z, sig) if integer else W.bpsk_awgn_llr(cw, z, sig)
    return fr, msg, cw, llr


def gpu_decode(N, K, fr, llr, fast, D, L, crc):
    plan = ps.Plan(N, K, fr, fast_nodes=fast, crc=crc)
    x = torch.from_numpy(np.ascontiguousarray(llr, np.float32)).cuda()
    info, pm, st, stats = ps.decode(plan, x, D, L, with_stats=True)
    torch.cuda.synchronize()
    msg = ps.unpack_bits(info.cpu().numpy(), K - crc)
    return msg, pm.cpu().numpy(), st.cpu().numpy(), stats.cpu().numpy().view(np.uint32)


def assert_parity(oracle, N, K, fr, llr, fast, D, L, crc, threads=8):
    m_o, pm_o, st_o, stats_o = oracle.scs_decode_batch(llr, N, K, fr, fast=fast, D=D, L=L, crc_len=crc, threads=threads)
    m_g, pm_g, st_g, stats_g = gpu_decode(N, K, fr, llr, fast, D, L, crc)
    bad = np.nonzero(np.any(m_o != m_g, axis=1) | (pm_o.view(np.uint32) != pm_g.view(np.uint32)) | (st_o != st_g))[0]
    assert bad.size == 0, f"{bad.size} frames differ, first {bad[:5]}: pm {pm_o[bad[:3]]} vs {pm_g[bad[:3]]}, st {st_o[bad[:3]]} vs {st_g[bad[:3]]}"
    assert np.array_equal(stats_o.astype(np.uint32), stats_g), "per-frame counters differ"
    return m_g, pm_g, st_g, stats_g


# config 1 of the workload: plain SCS, N=256, K=128, D=16, L=4, no CRC, 2.5 dB
def test_plain_scs_256(oracle_lib):
    fr, msg, cw, llr = make_frames(oracle_lib, 256, 128, 0, 2000, 2.5, seed=1)
    m, pm, st, stats = assert_parity(oracle_lib, 256, 128, fr, llr, False, 16, 4, 0)
    assert np.all(st == 0)
    assert np.mean(np.any(m != msg, axis=1)) < 0.2


@pytest.mark.parametrize("ebn0", [1.5, 2.0, 2.5, 3.0])
def test_crc_scs_1024(oracle_lib, ebn0):
    """config 2 shape (N=1024, K=512, CRC-16, D=L=32, fast nodes) at 2048 frames."""
    fr, msg, cw, llr = make_frames(oracle_lib, 1024, 512, 16, 2048, ebn0, seed=2 + int(ebn0 * 10))
    m, pm, st, stats = assert_parity(oracle_lib, 1024, 512, fr, llr, True, 32, 32, 16)
    assert stats[:, 1].sum() > 0  # path switches happened


CASES = [
    # N, K, crc, fast, D, L, ebn0
    (2, 1, 0, True, 1, 1, 1.0), (2, 2, 0, True, 4, 2, 1.0), (4, 2, 0, False, 2, 2, 0.0), (8, 4, 0, True, 8, 8, 0.0),
    (16, 8, 0, True, 64, 64, 0.0), (32, 16, 8, True, 33, 5, 1.0), (64, 48, 8, False, 7, 3, 2.0),
    (128, 43, 8, True, 8, 8, 1.0), (256, 171, 16, True, 64, 64, 1.0), (512, 256, 24, True, 64, 255, 1.5),
    (512, 384, 8, False, 3, 1, 3.0), (2048, 1024, 16, True, 64, 64, 2.0), (2048, 512, 8, True, 16, 16, 1.0),
    (4096, 2048, 16, True, 32, 32, 2.0), (8192, 4096, 24, True, 16, 8, 2.5), (1024, 1024, 0, True, 32, 32, 5.0),
    (1024, 1, 0, True, 32, 32, -2.0), (64, 63, 16, True, 64, 64, 3.0),
]


@pytest.mark.parametrize("N,K,crc,fast,D,L,ebn0", CASES)
def test_parity_shapes(oracle_lib, N, K, crc, fast, D, L, ebn0):
    B = max(40, min(600, 200000 // N))
    fr, msg, cw, llr = make_frames(oracle_lib, N, K, crc, B, ebn0, seed=N + K + D)
    assert_parity(oracle_lib, N, K, fr, llr, fast, D, L, crc)


@pytest.mark.parametrize("fast", [False, True])
def test_parity_exact_ties(oracle_lib, fast):
    """Small integer LLRs: many exact zeros and equal magnitudes exercise every
    tie rule (HD(-0), argmin to the lower index, newest-first pops, strict
    replacement)."""
    N, K = 128, 64
    fr, msg, cw, llr = make_frames(oracle_lib, N, K, 8, 1500, 0.0, seed=9, integer=True)
    llr = np.rint(llr / 5.0).astype(np.float32)
    llr[:, ::7] = -0.0
    assert_parity(oracle_lib, N, K, fr, llr, fast, 16, 4, 8)


def test_parity_random_frozen_sets(oracle_lib):
    rng = np.random.default_rng(3)
    for i in range(12):
        N = int(2 ** rng.integers(3, 10))
        K = int(rng.integers(2, N))
        fr = np.ones(N, np.uint8)
        fr[rng.choice(N, K, replace=False)] = 0
        crc = int(rng.choice([0, 8])) if K > 8 else 0
        fr2, msg, cw, llr = make_frames(oracle_lib, N, K, crc, 150, 1.0, seed=100 + i, frozen=fr)
        assert_parity(oracle_lib, N, K, fr, llr, bool(i % 2), int(rng.integers(1, 65)), int(rng.integers(1, 40)), crc)


def test_noiseless_and_large_magnitudes(oracle_lib):
    N, K, crc = 1024, 512, 16
    fr = oracle_lib.construct(N, K, 0.0)
    msg = W.message_bits(4, 64, K - crc)
    cw = oracle_lib.encode_batch(msg, N, K, fr, crc)
    for scale in (1.0, 1e30):
        llr = (np.where(cw == 1, -1.0, 1.0) * scale).astype(np.float32)
        m, pm, st, stats = assert_parity(oracle_lib, N, K, fr, llr, True, 32, 32, crc)
        assert np.array_equal(m, msg) and np.all(pm == 0) and np.all(st == 0)


def test_batch_sizes_and_empty(oracle_lib):
    N, K = 256, 128
    fr, msg, cw, llr = make_frames(oracle_lib, N, K, 0, 1000, 1.5, seed=5)
    for B in (1, 2, 3, 31, 33, 1000):
        assert_parity(oracle_lib, N, K, fr, llr[:B], True, 16, 8, 0)
    plan = ps.Plan(N, K, fr)
    empty = torch.empty((0, N), dtype=torch.float32, device="cuda")
    info, pm, st = ps.decode(plan, empty, 16, 8)
    torch.cuda.synchronize()
    assert info.shape[0] == 0


def test_encoder_parity(oracle_lib):
    for N, K, crc in [(8, 4, 0), (256, 128, 0), (1024, 512, 16), (2048, 1365, 24), (128, 96, 8), (32, 1, 0)]:
        fr = oracle_lib.construct(N, K, 0.0)
        msg = W.message_bits(N + crc, 300, K - crc)
        want = oracle_lib.encode_batch(msg, N, K, fr, crc)
        plan = ps.Plan(N, K, fr, crc=crc)
        d_msg = torch.from_numpy(ps.pack_bits(msg)).cuda()
        d_cw = torch.empty((300, plan.words), dtype=torch.int32, device="cuda")
        ps.polar_encode_batch(plan, d_msg, d_cw)
        torch.cuda.synchronize()
        got = ps.unpack_bits(d_cw.cpu().numpy(), N)
        assert np.array_equal(got, want)
        assert np.array_equal(ps.polar_encode(msg[0], N, K, fr, crc), want[0])


def test_single_frame_host_call(oracle_lib):
    N, K, crc = 512, 256, 16
    fr, msg, cw, llr = make_frames(oracle_lib, N, K, crc, 8, 1.5, seed=6)
    for b in range(8):
        st, m, pm = ps.scs_decode(llr[b], N, K, fr, 16, 16, crc)
        st_o, m_o, pm_o, _, _ = oracle_lib.scs_decode(llr[b], N, K, fr, fast=True, D=16, L=16, crc_len=crc)
        assert st == st_o and np.array_equal(m, m_o) and pm.view(np.uint32) == pm_o.view(np.uint32)


def test_streams_and_repeatability(oracle_lib):
    """Two streams decoding different halves concurrently give the same bytes
    as one launch; a repeated launch is bit-identical."""
    N, K, crc = 1024, 512, 16
    fr, msg, cw, llr = make_frames(oracle_lib, N, K, crc, 4096, 2.0, seed=7)
    plan = ps.Plan(N, K, fr, crc=crc)
    x = torch.from_numpy(llr).cuda()
    ref = ps.decode(plan, x, 32, 32)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(s1):
        a = ps.decode(plan, x[:2048], 32, 32)
    with torch.cuda.stream(s2):
        b = ps.decode(plan, x[2048:], 32, 32)
    torch.cuda.synchronize()
    for r, p, q in zip(ref, a, b):
        assert torch.equal(r, torch.cat([p, q]))
    again = ps.decode(plan, x, 32, 32)
    torch.cuda.synchronize()
    for r, g in zip(ref, again):
        assert torch.equal(r, g)


@pytest.mark.parametrize("N,K,crc,fast,D,L", [(256, 128, 0, False, 16, 4), (1024, 512, 16, True, 32, 32)])
def test_scaled_min_sum_parity(oracle_lib, N, K, crc, fast, D, L):
    """Per-stage f scales (plan option) against the oracle's scaled decoder; a
    plan whose scales are reset decodes exactly like the unscaled one."""
    fr, msg, cw, llr = make_frames(oracle_lib, N, K, crc, 600, 2.0, seed=31)
    n = int(np.log2(N))
    scales = np.random.default_rng(n).uniform(0.55, 1.25, n).astype(np.float32)
    plan = ps.Plan(N, K, fr, fast_nodes=fast, crc=crc)
    plan.set_scales(scales)
    x = torch.from_numpy(llr).cuda()
    info, pm, st, stats = ps.decode(plan, x, D, L, with_stats=True)
    torch.cuda.synchronize()
    m_o, pm_o, st_o, stats_o = oracle_lib.scs_decode_batch(llr, N, K, fr, fast=fast, D=D, L=L, crc_len=crc,
                                                           threads=8, scales=scales)
    assert np.array_equal(ps.unpack_bits(info.cpu().numpy(), K - crc), m_o)
    assert np.array_equal(pm.cpu().numpy().view(np.uint32), pm_o.view(np.uint32))
    assert np.array_equal(st.cpu().numpy(), st_o)
    plan.set_scales(None)
    info2, pm2, st2 = ps.decode(plan, x, D, L)
    torch.cuda.synchronize()
    m_u, pm_u, st_u, _ = oracle_lib.scs_decode_batch(llr, N, K, fr, fast=fast, D=D, L=L, crc_len=crc, threads=8)
    assert np.array_equal(ps.unpack_bits(info2.cpu().numpy(), K - crc), m_u)
    assert np.array_equal(pm2.cpu().numpy().view(np.uint32), pm_u.view(np.uint32))


def test_full_size_launch(oracle_lib):
    """The bench's launch: 1,048,576 frames of PC(1024,512) CRC-16, D = L = 32,
    at 1.5 dB (the hardest point) in one scs_decode_batch call.  The batch
    tiles 4,096 host-made frames 256 times, so every one of the 2^20 outputs
    has an oracle value (that of its row modulo 4,096)."""
    N, K, crc, D, L = 1024, 512, 16, 32, 32
    base = 4096
    fr, msg, cw, llr = make_frames(oracle_lib, N, K, crc, base, 1.5, seed=77)
    m_o, pm_o, st_o, _ = oracle_lib.scs_decode_batch(llr, N, K, fr, fast=True, D=D, L=L, crc_len=crc, threads=8)
    plan = ps.Plan(N, K, fr, fast_nodes=True, crc=crc)
    x = torch.from_numpy(llr).cuda().repeat(256, 1)
    info, pm, st = ps.decode(plan, x, D, L)
    torch.cuda.synchronize()
    del x
    words_o = torch.from_numpy(ps.pack_bits(m_o)).cuda().repeat(256, 1)
    assert torch.equal(info, words_o)
    assert torch.equal(pm.view(torch.int32), torch.from_numpy(pm_o.view(np.int32)).cuda().repeat(256))
    assert torch.equal(st, torch.from_numpy(st_o).cuda().repeat(256))
