"""Mixed batches: frames of different codes, stack depths and visit caps in
one persistent launch (scs_decode_mixed), or in two launches split by stack
rows (scs_decode_mixed_split).  Each frame must come out exactly as if it
had been decoded alone with its own plan, D and L."""
import ctypes as C

import numpy as np
import pytest

import paper_1809_03606_gb300 as ps
import workloads as W


@pytest.fixture(scope="module")
def lib():
    ps.load(build_if_missing=True)
    return ps.load()


# ------------------------------------------------------------ host-side checks
def test_plan_set_validation(lib):
    p = ps.Plan(64, 32, ps.polar_construct(64, 32, 0.0))
    with pytest.raises(ps.PolarError):
        ps.PlanSet([])
    with pytest.raises(ps.PolarError):
        ps.PlanSet([p] * 65)
    big = ps.Plan(16384, 8192, ps.polar_construct(16384, 8192, 0.0))
    with pytest.raises(ps.PolarError) as e:
        ps.PlanSet([p, big])
    assert e.value.rc == ps.POLAR_ELIMIT
    s = ps.PlanSet([p, p])
    d = C.c_void_p(256)
    args = lambda B, Dmax, fr: (s.handle, fr, None, B, Dmax, d, d, d, d, d, d, None, None)
    assert lib.scs_decode_mixed(*args(4, 65, d)) == ps.POLAR_ELIMIT
    assert lib.scs_decode_mixed(*args(4, 0, d)) == ps.POLAR_EINVAL
    assert lib.scs_decode_mixed(*args(4, 8, C.c_void_p(260))) == ps.POLAR_EINVAL  # frames not 16-byte aligned
    assert lib.scs_decode_mixed(*args(0, 8, d)) == 0


def test_split_order_and_validation(lib):
    """polar_mixed_split_order: frames with 32 < D <= 64 first (longest first
    within each part), invalid descriptors with the one-row part; the split
    decode rejects a missing order, n_two outside [0, B] and a Dmax that
    cannot hold the two-row part."""
    p1 = ps.Plan(64, 32, ps.polar_construct(64, 32, 0.0))
    p2 = ps.Plan(256, 128, ps.polar_construct(256, 128, 0.0))
    s = ps.PlanSet([p1, p2])
    fr = np.array([[0, 8, 8, 0], [1, 40, 40, 0], [0, 64, 64, 0], [1, 32, 32, 0], [5, 64, 64, 0], [1, 33, 1, 0]],
                  np.int32)
    order, n_two = ps.polar_mixed_split_order(s, fr)
    assert n_two == 3
    assert sorted(order[:3].tolist()) == [1, 2, 5] and sorted(order[3:].tolist()) == [0, 3, 4]
    assert order[:3].tolist() == [1, 5, 2]  # 256*(8+40) > 256*(8+33) > 64*(8+64)
    assert order[3:].tolist() == [3, 0, 4]  # the invalid descriptor (plan 5) weighs 0: last
    d = C.c_void_p(256)
    args = lambda order, n, Dmax: (s.handle, d, order, 6, n, Dmax, d, d, d, d, d, d, None, None)
    assert lib.scs_decode_mixed_split(*args(None, 3, 64)) == ps.POLAR_EINVAL
    assert lib.scs_decode_mixed_split(*args(d, 7, 64)) == ps.POLAR_EINVAL
    assert lib.scs_decode_mixed_split(*args(d, -1, 64)) == ps.POLAR_EINVAL
    assert lib.scs_decode_mixed_split(*args(d, 3, 32)) == ps.POLAR_EINVAL
    assert lib.scs_decode_mixed_split(*args(d, 3, 65)) == ps.POLAR_ELIMIT


# ----------------------------------------------------------------- GPU tests
def _mixed_problem(oracle, codes, B, seed, ebn0_lo=1.0, ebn0_hi=4.0):
    """codes: list of (N, K, crc).  Returns plans, per-frame arrays and LLR rows."""
    rng = np.random.default_rng(seed)
    plans, frozens = [], []
    for N, K, crc in codes:
        fr = oracle.construct(N, K, 0.0)
        frozens.append(fr)
        plans.append(ps.Plan(N, K, fr, fast_nodes=True, crc=crc))
    idx = rng.integers(0, len(codes), B).astype(np.int32)
    D = rng.integers(1, 65, B).astype(np.int32)
    L = rng.integers(1, 65, B).astype(np.int32)
    eb = rng.uniform(ebn0_lo, ebn0_hi, B)
    rows = [None] * B
    msgs = [None] * B
    for ci, (N, K, crc) in enumerate(codes):
        sel = np.nonzero(idx == ci)[0]
        if sel.size == 0:
            continue
        msg = W.message_bits(seed + 17 * ci, sel.size, K - crc)
        cw = oracle.encode_batch(msg, N, K, frozens[ci], crc)
        z = W.awgn_noise(seed + 17 * ci, sel.size, N)
        sig = np.array([W.sigma_from_ebn0(e, K / N) for e in eb[sel]])
        llr = W.bpsk_awgn_llr(cw, z, sig)
        for j, b in enumerate(sel):
            rows[b] = llr[j]
            msgs[b] = msg[j]
    return plans, frozens, idx, D, L, rows, msgs


CODES = [(64, 32, 8), (128, 43, 8), (256, 171, 8), (512, 256, 8), (1024, 683, 8), (2048, 1024, 8), (256, 64, 8),
         (128, 96, 0)]


def _solo(torch, plan, rows, D, L):
    x = torch.from_numpy(np.stack(rows).astype(np.float32)).cuda()
    info, pm, st, stats = ps.decode(plan, x, int(D), int(L), with_stats=True)
    return info.cpu().numpy(), pm.cpu().numpy(), st.cpu().numpy(), stats.cpu().numpy()


@pytest.mark.gpu
def test_mixed_equals_solo_and_oracle(lib, oracle_lib):
    torch = pytest.importorskip("torch")
    plans, frozens, idx, D, L, rows, msgs = _mixed_problem(oracle_lib, CODES, 3000, seed=5)
    pset = ps.PlanSet(plans)
    mb = ps.MixedBatch(pset, idx, D, L, rows)
    stats = torch.empty((mb.B, 4), dtype=torch.int32, device="cuda")
    mb.decode(pset, stats)
    torch.cuda.synchronize()
    pm = mb.pm.cpu().numpy()
    st = mb.status.cpu().numpy()
    stn = stats.cpu().numpy()
    # every frame equals its solo decode (grouped by code, D and L)
    groups = {}
    for b in range(mb.B):
        groups.setdefault((int(idx[b]), int(D[b]), int(L[b])), []).append(b)
    for (ci, d, l), bs in groups.items():
        info_s, pm_s, st_s, stats_s = _solo(torch, plans[ci], [rows[b] for b in bs], d, l)
        for j, b in enumerate(bs):
            assert np.array_equal(mb.message_words(b), info_s[j]), b
            assert pm[b].view(np.uint32) == pm_s[j].view(np.uint32) and st[b] == st_s[j]
            assert np.array_equal(stn[b], stats_s[j])
    # and a sample against the oracle
    for b in range(0, mb.B, 10):
        N, K, crc = CODES[idx[b]]
        st_o, m_o, pm_o, _, _ = oracle_lib.scs_decode(rows[b], N, K, frozens[idx[b]], fast=True, D=int(D[b]),
                                                      L=int(L[b]), crc_len=crc)
        got = ps.unpack_bits(mb.message_words(b)[None, :], K - crc)[0]
        assert np.array_equal(got, m_o) and pm[b].view(np.uint32) == pm_o.view(np.uint32) and st[b] == st_o


@pytest.mark.gpu
def test_mixed_invalid_descriptors_are_isolated(lib, oracle_lib):
    torch = pytest.importorskip("torch")
    plans, frozens, idx, D, L, rows, msgs = _mixed_problem(oracle_lib, CODES[:4], 400, seed=6)
    pset = ps.PlanSet(plans)
    good = ps.MixedBatch(pset, idx, D, L, rows)
    good.decode(pset)
    mb = ps.MixedBatch(pset, idx, D, L, rows)
    bad = [3, 50, 51, 200, 201]
    mb.frames[3, 0] = 99  # plan index out of range
    mb.frames[50, 1] = 0  # D < 1
    mb.frames[51, 2] = 0  # L < 1
    mb.frames[200, 0] = -1
    mb.frames[201, 1] = mb.Dmax + 1  # D beyond the scratch sizing
    mb.decode(pset)
    torch.cuda.synchronize()
    st = mb.status.cpu().numpy()
    assert all(st[b] == 3 for b in bad)
    keep = np.setdiff1d(np.arange(mb.B), bad)
    assert np.array_equal(st[keep], good.status.cpu().numpy()[keep])
    assert np.array_equal(mb.pm.cpu().numpy()[keep].view(np.uint32), good.pm.cpu().numpy()[keep].view(np.uint32))


@pytest.mark.gpu
def test_mixed_graph_replay_and_tuner(lib, oracle_lib):
    torch = pytest.importorskip("torch")
    plans, frozens, idx, D, L, rows, msgs = _mixed_problem(oracle_lib, CODES, 2000, seed=7)
    pset = ps.PlanSet(plans)
    mb = ps.MixedBatch(pset, idx, D, L, rows)
    mb.decode(pset)  # first call on the device builds the set's tables
    torch.cuda.synchronize()
    ref = (mb.info.clone(), mb.pm.clone(), mb.status.clone())
    wpb, chunk = mb.tune(pset)
    assert wpb in (1, 2, 4) and chunk in (1, 4, 16)
    torch.cuda.synchronize()
    for r, g in zip(ref, (mb.info, mb.pm, mb.status)):
        assert torch.equal(r, g)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        mb.decode(pset, stream=s)
    torch.cuda.current_stream().wait_stream(s)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        mb.decode(pset)
    for _ in range(2):
        mb.info.zero_()
        mb.pm.zero_()
        g.replay()
        torch.cuda.synchronize()
        for r, x in zip(ref, (mb.info, mb.pm, mb.status)):
            assert torch.equal(r, x)


@pytest.mark.gpu
def test_mixed_with_systematic_plans(lib, oracle_lib):
    """Systematic and non-systematic plans in one launch: every frame equals
    the oracle's decode with its own encoding, D and L."""
    torch = pytest.importorskip("torch")
    codes = [(256, 128, 8, True), (512, 256, 8, False), (1024, 512, 16, True), (128, 64, 0, True)]
    rng = np.random.default_rng(12)
    B = 800
    plans, frozens = [], []
    for N, K, crc, sysf in codes:
        fr = oracle_lib.construct(N, K, 0.0)
        frozens.append(fr)
        plans.append(ps.Plan(N, K, fr, fast_nodes=True, crc=crc, systematic=sysf))
    idx = rng.integers(0, len(codes), B).astype(np.int32)
    D = rng.integers(1, 65, B).astype(np.int32)
    L = rng.integers(1, 65, B).astype(np.int32)
    rows, msgs = [None] * B, [None] * B
    for ci, (N, K, crc, sysf) in enumerate(codes):
        sel = np.nonzero(idx == ci)[0]
        msg = W.message_bits(90 + ci, sel.size, K - crc)
        cw = oracle_lib.encode_batch(msg, N, K, frozens[ci], crc, systematic=sysf)
        llr = W.bpsk_awgn_llr(cw, W.awgn_noise(90 + ci, sel.size, N), W.sigma_from_ebn0(2.0, K / N))
        for j, b in enumerate(sel):
            rows[b], msgs[b] = llr[j], msg[j]
    pset = ps.PlanSet(plans)
    mb = ps.MixedBatch(pset, idx, D, L, rows)
    mb.decode(pset)
    torch.cuda.synchronize()
    pm, st = mb.pm.cpu().numpy(), mb.status.cpu().numpy()
    for b in range(B):
        N, K, crc, sysf = codes[idx[b]]
        st_o, m_o, pm_o, _, _ = oracle_lib.scs_decode(rows[b], N, K, frozens[idx[b]], fast=True, D=int(D[b]),
                                                      L=int(L[b]), crc_len=crc, systematic=sysf)
        got = ps.unpack_bits(mb.message_words(b)[None, :], K - crc)[0]
        assert np.array_equal(got, m_o), b
        assert pm[b].view(np.uint32) == pm_o.view(np.uint32) and st[b] == st_o, b


@pytest.mark.gpu
def test_split_launches_equal_one_launch_and_oracle(lib, oracle_lib):
    """The batch split by stack rows into two launches on two streams gives
    every frame exactly the one-launch result (message words, metric bits,
    status, counters), which is also the oracle's on a sample; the split is
    captured in a CUDA graph and replayed; batches with only one kind of
    frame take a single launch."""
    torch = pytest.importorskip("torch")
    plans, frozens, idx, D, L, rows, msgs = _mixed_problem(oracle_lib, CODES, 3000, seed=25)
    pset = ps.PlanSet(plans)
    mb = ps.MixedBatch(pset, idx, D, L, rows)
    assert 0 < mb.n_two < mb.B
    stats1 = torch.empty((mb.B, 4), dtype=torch.int32, device="cuda")
    mb.decode(pset, stats1)
    torch.cuda.synchronize()
    ref = (mb.info.clone(), mb.pm.clone(), mb.status.clone(), stats1.clone())
    mb.info.zero_()
    mb.pm.zero_()
    stats2 = torch.zeros_like(stats1)
    mb.decode_split(pset, stats2)
    torch.cuda.synchronize()
    for r, g in zip(ref, (mb.info, mb.pm, mb.status, stats2)):
        assert torch.equal(r, g)
    pm, st = mb.pm.cpu().numpy(), mb.status.cpu().numpy()
    for b in range(0, mb.B, 15):
        N, K, crc = CODES[idx[b]]
        st_o, m_o, pm_o, _, _ = oracle_lib.scs_decode(rows[b], N, K, frozens[idx[b]], fast=True, D=int(D[b]),
                                                      L=int(L[b]), crc_len=crc)
        got = ps.unpack_bits(mb.message_words(b)[None, :], K - crc)[0]
        assert np.array_equal(got, m_o) and pm[b].view(np.uint32) == pm_o.view(np.uint32) and st[b] == st_o
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        mb.decode_split(pset)
    for _ in range(2):
        mb.info.zero_()
        mb.pm.zero_()
        g.replay()
        torch.cuda.synchronize()
        for r, x in zip(ref[:3], (mb.info, mb.pm, mb.status)):
            assert torch.equal(r, x)
    for keep in (D <= 32, D > 32):  # one kind of frame only
        sel = np.nonzero(keep)[0][:500]
        one = ps.MixedBatch(pset, idx[sel], D[sel], L[sel], [rows[b] for b in sel])
        assert one.n_two in (0, one.B)
        one.decode(pset)
        torch.cuda.synchronize()
        r1 = (one.info.clone(), one.pm.clone(), one.status.clone())
        one.decode_split(pset)
        torch.cuda.synchronize()
        for r, x in zip(r1, (one.info, one.pm, one.status)):
            assert torch.equal(r, x)


@pytest.mark.gpu
def test_full_code_table_and_largest_code(lib, oracle_lib):
    """A set of 64 codes, the most a set holds, one of them N = 8192: the code
    table and the largest warp areas share the block's shared memory.  Every
    frame equals its solo decode, in one launch and split by stack rows; a
    sample also equals the oracle."""
    torch = pytest.importorskip("torch")
    codes = []
    for N in (16, 32, 64, 128, 256, 512, 1024):
        for r in (1 / 8, 1 / 4, 1 / 3, 3 / 8, 1 / 2, 5 / 8, 2 / 3, 3 / 4, 7 / 8):
            K = max(1, round(N * r))
            codes.append((N, K, 8 if K > 16 else 0))
    codes.append((8192, 4096, 16))
    assert len(codes) == 64
    plans, frozens, idx, D, L, rows, msgs = _mixed_problem(oracle_lib, codes, 640, seed=41, ebn0_lo=2.5)
    pset = ps.PlanSet(plans)
    mb = ps.MixedBatch(pset, idx, D, L, rows)
    mb.decode(pset)
    torch.cuda.synchronize()
    ref = (mb.info.clone(), mb.pm.clone(), mb.status.clone())
    pm, st = mb.pm.cpu().numpy(), mb.status.cpu().numpy()
    assert (idx == 63).sum() > 0
    groups = {}
    for b in range(mb.B):
        groups.setdefault((int(idx[b]), int(D[b]), int(L[b])), []).append(b)
    for (ci, d, l), bs in groups.items():
        info_s, pm_s, st_s, _ = _solo(torch, plans[ci], [rows[b] for b in bs], d, l)
        for j, b in enumerate(bs):
            assert np.array_equal(mb.message_words(b), info_s[j]), b
            assert pm[b].view(np.uint32) == pm_s[j].view(np.uint32) and st[b] == st_s[j], b
    mb.info.zero_()
    mb.pm.zero_()
    mb.decode_split(pset)
    torch.cuda.synchronize()
    for r, g in zip(ref, (mb.info, mb.pm, mb.status)):
        assert torch.equal(r, g)
    for b in list(range(0, mb.B, 20)) + [int(np.nonzero(idx == 63)[0][0])]:
        N, K, crc = codes[idx[b]]
        st_o, m_o, pm_o, _, _ = oracle_lib.scs_decode(rows[b], N, K, frozens[idx[b]], fast=True, D=int(D[b]),
                                                      L=int(L[b]), crc_len=crc)
        got = ps.unpack_bits(mb.message_words(b)[None, :], K - crc)[0]
        assert np.array_equal(got, m_o) and pm[b].view(np.uint32) == pm_o.view(np.uint32) and st[b] == st_o, b
