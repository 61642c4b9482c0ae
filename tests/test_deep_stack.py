"""Deep stacks (D > 64): the memory-stack decoder against the oracle.

The paper's own setting (Sec. 5) is PC(1024,512) with CRC-24C, L = 8 and
D = 8192, far beyond the register stack's 64 entries.  scs_decode_batch then
keeps the stack in per-warp scratch memory with the same search order:
smallest path metric first (ties newest), strict replacement of the worst
entry (largest metric, ties oldest) when the stack is full, and the L-prune.

CPU part: invariants of the oracle at large D (no dependence on D once the
stack can never fill; the bound on live entries the kernel's scratch is sized
by).  GPU part: bit-exact parity (message bits, metric bits, status,
counters) on cases that reach every branch: a full stack with replacements,
prunes, many blocks of 32 entries, tie-heavy integer LLRs."""
import numpy as np
import pytest

import paper_1809_03606_gb300 as ps
import workloads as W


def _frames(oracle, N, K, crc, B, ebn0, seed, integer=False):
    fr = oracle.construct(N, K, 0.0)
    msg = W.message_bits(seed, B, K - crc)
    cw = oracle.encode_batch(msg, N, K, fr, crc)
    sig = W.sigma_from_ebn0(ebn0, K / N)
    z = W.awgn_noise(seed, B, N)
    llr = W.integer_llr(cw, z, sig) if integer else W.bpsk_awgn_llr(cw, z, sig)
    return fr, llr


def _nbranch(N, K, fr, fast):
    """Branching nodes of the schedule: information leaves, R-1, REP, SPC."""
    ops = ps.polar_plan_schedule(ps.Plan(N, K, fr, fast_nodes=fast))
    return sum(1 for op, _, _ in ops if op in ("leaf1", "R1", "REP", "SPC"))


@pytest.mark.parametrize("N,K,crc,fast,L", [(256, 128, 8, True, 4), (128, 64, 0, False, 2)])
def test_deep_results_do_not_depend_on_d_once_it_cannot_fill(oracle_lib, N, K, crc, fast, L):
    """Each iteration pops one path and pushes at most 8, so a stack of
    1 + 7 * (iterations) entries never fills and never evicts: every larger D
    gives the same decisions, metrics and counters (except the stack-cost
    term of the operation count, which depends on ceil(log2 D))."""
    fr, llr = _frames(oracle_lib, N, K, crc, 40, 0.5, seed=N + L)
    nb = _nbranch(N, K, fr, fast)
    max_iter = L * (nb + 9) + 2
    d0 = 1 + 7 * max_iter
    ref = oracle_lib.scs_decode_batch(llr, N, K, fr, fast=fast, D=d0, L=L, crc_len=crc)
    for D in (d0 + 1, 4 * d0, 1 << 16):
        got = oracle_lib.scs_decode_batch(llr, N, K, fr, fast=fast, D=D, L=L, crc_len=crc)
        assert np.array_equal(ref[0], got[0])
        assert np.array_equal(ref[1].view(np.uint32), got[1].view(np.uint32))
        assert np.array_equal(ref[2], got[2])
        assert np.array_equal(ref[3][:, [0, 1, 3]], got[3][:, [0, 1, 3]])


def test_deep_pops_respect_the_iteration_bound(oracle_lib):
    """The scratch of the memory stack holds one snapshot per iteration: the
    oracle's pop count stays within L * (branching nodes + 9) + 2 even on
    frames that end by the CRC-failure limit."""
    N, K, crc, L = 256, 128, 16, 3
    fr, llr = _frames(oracle_lib, N, K, crc, 60, -1.0, seed=5)
    nb = _nbranch(N, K, fr, True)
    _, _, st, stats = oracle_lib.scs_decode_batch(llr, N, K, fr, fast=True, D=4096, L=L, crc_len=crc)
    assert (st != 2).all()  # no frame ran out of iterations
    assert int(stats[:, 0].max()) <= L * (nb + 9) + 2


def test_paper_setting_noiseless_round_trip(oracle_lib):
    """The paper's decoder setting in the oracle (systematic PC(1024,512),
    CRC-24C, D = 8192, L = 8): noiseless frames come back as their messages
    with status 0 and path metric 0, the search never leaving the correct path:
    the first pop, one pop per branching node, then the complete path."""
    N, K, crc = 1024, 512, 24
    fr = oracle_lib.construct(N, K, 0.0)
    msg = W.message_bits(8, 6, K - crc)
    cw = oracle_lib.encode_batch(msg, N, K, fr, crc, systematic=True)
    llr = W.bpsk_awgn_llr(cw, np.zeros(cw.shape, np.float32), 0.6)
    m, pm, st, stats = oracle_lib.scs_decode_batch(llr, N, K, fr, fast=True, D=8192, L=8, crc_len=crc,
                                                   systematic=True)
    assert (st == 0).all() and (pm == 0).all() and np.array_equal(m, msg)
    assert (stats[:, 0] == _nbranch(N, K, fr, True) + 2).all()
    assert (stats[:, 1] == 0).all()  # no path switch


# ----------------------------------------------------------------- GPU part
def _gpu(N, K, fr, llr, fast, D, L, crc):
    torch = pytest.importorskip("torch")
    plan = ps.Plan(N, K, fr, fast_nodes=fast, crc=crc)
    x = torch.from_numpy(np.ascontiguousarray(llr, np.float32)).cuda()
    info, pm, st, stats = ps.decode(plan, x, D, L, with_stats=True)
    torch.cuda.synchronize()
    return (ps.unpack_bits(info.cpu().numpy(), K - crc), pm.cpu().numpy(), st.cpu().numpy(),
            stats.cpu().numpy().view(np.uint32))


DEEP_CASES = [
    # N, K, crc, fast, D, L, Eb/N0, frames, integer LLRs
    (1024, 512, 24, True, 8192, 8, 1.0, 1000, False),  # the decoder setting of Sec. 5
    (1024, 512, 24, True, 8192, 8, 2.0, 1000, False),
    (128, 64, 8, True, 65, 16, 0.5, 2000, False),      # one entry above the register stack, full stacks
    (256, 128, 0, False, 100, 4, 1.0, 1500, False),    # bit-level, replacements of the worst entry
    (512, 256, 16, True, 300, 32, 0.0, 400, False),    # many blocks of 32 entries
    (64, 32, 8, True, 90, 255, -1.0, 1500, False),     # long searches, up to 255 CRC failures
    (128, 64, 8, True, 80, 6, 0.0, 3000, True),        # ties everywhere
    (2048, 1024, 16, True, 1000, 4, 1.5, 200, False),
]


@pytest.mark.gpu
@pytest.mark.parametrize("N,K,crc,fast,D,L,ebn0,B,integer", DEEP_CASES)
def test_gpu_deep_stack_parity(oracle_lib, N, K, crc, fast, D, L, ebn0, B, integer):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    ps.load(build_if_missing=True)
    fr, llr = _frames(oracle_lib, N, K, crc, B, ebn0, seed=N + D + L, integer=integer)
    if integer:
        llr = np.rint(llr / 5.0).astype(np.float32)
        llr[:, ::7] = -0.0
    m_o, pm_o, st_o, stats_o = oracle_lib.scs_decode_batch(llr, N, K, fr, fast=fast, D=D, L=L, crc_len=crc, threads=8)
    m_g, pm_g, st_g, stats_g = _gpu(N, K, fr, llr, fast, D, L, crc)
    bad = np.nonzero(np.any(m_o != m_g, axis=1) | (pm_o.view(np.uint32) != pm_g.view(np.uint32)) | (st_o != st_g))[0]
    assert bad.size == 0, f"{bad.size} frames differ, first {bad[:5]}"
    assert np.array_equal(stats_o.astype(np.uint32), stats_g), "per-frame counters differ"
    assert stats_g[:, 0].max() > 8  # the search went deep


@pytest.mark.gpu
def test_gpu_deep_stack_fills_and_prunes(oracle_lib):
    """A case whose stacks provably fill (pushes beyond D) and prune (L
    reached), checked through the oracle's counters, then parity."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    ps.load(build_if_missing=True)
    N, K, crc, D, L = 256, 128, 8, 70, 8
    fr, llr = _frames(oracle_lib, N, K, crc, 300, 0.0, seed=77)
    m_o, pm_o, st_o, stats_o = oracle_lib.scs_decode_batch(llr, N, K, fr, fast=True, D=D, L=L, crc_len=crc)
    # pushes: at least 2 per expansion; pops: one per iteration; a frame with
    # more than D + pops pushes must have evicted or dropped candidates
    assert (2 * stats_o[:, 3] > D + stats_o[:, 0]).any()
    m_g, pm_g, st_g, stats_g = _gpu(N, K, fr, llr, True, D, L, crc)
    assert np.array_equal(m_o, m_g)
    assert np.array_equal(pm_o.view(np.uint32), pm_g.view(np.uint32))
    assert np.array_equal(st_o, st_g)
    assert np.array_equal(stats_o.astype(np.uint32), stats_g)


@pytest.mark.gpu
def test_gpu_deep_stack_empty_and_single_frames(oracle_lib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    ps.load(build_if_missing=True)
    N, K, crc = 1024, 512, 24
    fr, llr = _frames(oracle_lib, N, K, crc, 3, 1.5, seed=3)
    plan = ps.Plan(N, K, fr, fast_nodes=True, crc=crc)
    x = torch.from_numpy(llr).cuda()
    info, pm, st = ps.decode(plan, x[:0], 8192, 8)
    assert info.shape[0] == 0
    for b in range(3):
        m_g, pm_g, st_g, _ = _gpu(N, K, fr, llr[b:b + 1], True, 8192, 8, crc)
        m_o, pm_o, st_o, _ = oracle_lib.scs_decode_batch(llr[b:b + 1], N, K, fr, fast=True, D=8192, L=8, crc_len=crc)
        assert np.array_equal(m_o, m_g) and pm_o.view(np.uint32)[0] == pm_g.view(np.uint32)[0] and st_o[0] == st_g[0]


@pytest.mark.gpu
@pytest.mark.parametrize("N,K,crc,D,L,ebn0,B", [
    (1024, 512, 24, 65536, 8, 1.0, 32),      # the largest depth
    (8192, 4096, 16, 65536, 255, 3.0, 8),    # the longest code, largest depth and cap: 90 MB of scratch per
                                             # warp, so the 8 GiB budget leaves fewer than 100 resident warps
])
def test_gpu_deep_stack_limits(oracle_lib, N, K, crc, D, L, ebn0, B):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    ps.load(build_if_missing=True)
    fr, llr = _frames(oracle_lib, N, K, crc, B, ebn0, seed=N + D + L)
    m_o, pm_o, st_o, stats_o = oracle_lib.scs_decode_batch(llr, N, K, fr, fast=True, D=D, L=L, crc_len=crc, threads=2)
    m_g, pm_g, st_g, stats_g = _gpu(N, K, fr, llr, True, D, L, crc)
    assert np.array_equal(m_o, m_g)
    assert np.array_equal(pm_o.view(np.uint32), pm_g.view(np.uint32))
    assert np.array_equal(st_o, st_g)
    assert np.array_equal(stats_o.astype(np.uint32), stats_g)


@pytest.mark.gpu
def test_gpu_paper_setting_full_size_launch(oracle_lib):
    """The paper-setting bench's launch: 524,288 frames of systematic
    PC(1024,512) CRC-24C, D = 8192, L = 8, at 0 dB (its hardest point), in one
    scs_decode_batch call.  The batch tiles 2,048 host-made frames 256 times,
    so every output has an oracle value (that of its row modulo 2,048)."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    ps.load(build_if_missing=True)
    N, K, crc, D, L, base = 1024, 512, 24, 8192, 8, 2048
    fr = oracle_lib.construct(N, K, 0.0)
    msg = W.message_bits(606, base, K - crc)
    cw = oracle_lib.encode_batch(msg, N, K, fr, crc, systematic=True)
    llr = W.bpsk_awgn_llr(cw, W.awgn_noise(606, base, N), W.sigma_from_ebn0(0.0, K / N))
    m_o, pm_o, st_o, _ = oracle_lib.scs_decode_batch(llr, N, K, fr, fast=True, D=D, L=L, crc_len=crc, threads=8,
                                                      systematic=True)
    plan = ps.Plan(N, K, fr, fast_nodes=True, crc=crc, systematic=True)
    x = torch.from_numpy(llr).cuda().repeat(256, 1)
    info, pm, st = ps.decode(plan, x, D, L)
    torch.cuda.synchronize()
    del x
    assert torch.equal(info, torch.from_numpy(ps.pack_bits(m_o)).cuda().repeat(256, 1))
    assert torch.equal(pm.view(torch.int32), torch.from_numpy(pm_o.view(np.int32)).cuda().repeat(256))
    assert torch.equal(st, torch.from_numpy(st_o).cuda().repeat(256))


@pytest.mark.gpu
def test_gpu_deep_stack_scaled_and_host_call(oracle_lib):
    """The memory stack with per-stage f scales (against the oracle's scaled
    decoder), and the host single-frame call at the paper's depth."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    ps.load(build_if_missing=True)
    N, K, crc, D, L = 512, 256, 16, 500, 6
    fr, llr = _frames(oracle_lib, N, K, crc, 400, 1.0, seed=91)
    scales = np.random.default_rng(9).uniform(0.55, 1.25, 9).astype(np.float32)
    plan = ps.Plan(N, K, fr, fast_nodes=True, crc=crc)
    plan.set_scales(scales)
    info, pm, st, stats = ps.decode(plan, torch.from_numpy(llr).cuda(), D, L, with_stats=True)
    torch.cuda.synchronize()
    m_o, pm_o, st_o, stats_o = oracle_lib.scs_decode_batch(llr, N, K, fr, fast=True, D=D, L=L, crc_len=crc, threads=8,
                                                           scales=scales)
    assert np.array_equal(ps.unpack_bits(info.cpu().numpy(), K - crc), m_o)
    assert np.array_equal(pm.cpu().numpy().view(np.uint32), pm_o.view(np.uint32))
    assert np.array_equal(st.cpu().numpy(), st_o)
    assert np.array_equal(stats.cpu().numpy().view(np.uint32), stats_o.astype(np.uint32))
    N, K, crc = 1024, 512, 24
    fr, llr = _frames(oracle_lib, N, K, crc, 6, 1.0, seed=92)
    for b in range(6):
        st1, m1, pm1 = ps.scs_decode(llr[b], N, K, fr, 8192, 8, crc)
        st_o1, m_o1, pm_o1, _, _ = oracle_lib.scs_decode(llr[b], N, K, fr, fast=True, D=8192, L=8, crc_len=crc)
        assert st1 == st_o1 and np.array_equal(m1, m_o1) and pm1.view(np.uint32) == pm_o1.view(np.uint32)
