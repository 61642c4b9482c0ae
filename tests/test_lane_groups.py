"""The decoder on lane groups: a warp decodes 32 / G frames at once, each on
G = 8, 16 or 32 lanes with its stack spread over them.  The mapping must not
change any result: message bits, path-metric bits, status and every counter
equal the CPU oracle's for each G, across code shapes, tie-heavy integer
LLRs, random frozen sets, stack depths up to 64, batch sizes that leave
groups of a warp idle, and plans with stage scales or systematic encoding."""
import numpy as np
import pytest

import paper_1809_03606_gb300 as ps
import workloads as W
from test_gpu_parity import make_frames

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
LANES = [8, 16, 32]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    ps.load(build_if_missing=True)


def _decode(plan, llr, D, L, lanes):
    plan.set_lanes(lanes)
    x = torch.from_numpy(np.ascontiguousarray(llr, np.float32)).cuda()
    info, pm, st, stats = ps.decode(plan, x, D, L, with_stats=True)
    torch.cuda.synchronize()
    return (ps.unpack_bits(info.cpu().numpy(), plan.kmsg), pm.cpu().numpy(), st.cpu().numpy(),
            stats.cpu().numpy().view(np.uint32))


def _check(oracle, plan, llr, D, L, scales=None, systematic=False):
    m_o, pm_o, st_o, stats_o = oracle.scs_decode_batch(llr, plan.N, plan.K, plan.frozen, fast=plan.fast, D=D, L=L,
                                                       crc_len=plan.crc, threads=8, scales=scales,
                                                       systematic=systematic)
    for lanes in LANES:
        m, pm, st, stats = _decode(plan, llr, D, L, lanes)
        bad = np.nonzero(np.any(m_o != m, axis=1) | (pm_o.view(np.uint32) != pm.view(np.uint32)) | (st_o != st))[0]
        assert bad.size == 0, f"G={lanes}: {bad.size} frames differ, first {bad[:5]}"
        assert np.array_equal(stats_o.astype(np.uint32), stats), f"G={lanes}: counters differ"
    return st_o


SHAPES = [
    # N, K, crc, fast, D, L, ebn0
    (1024, 512, 16, True, 32, 32, 1.5), (1024, 512, 16, True, 32, 32, 3.0), (256, 128, 0, False, 16, 4, 2.5),
    (2, 1, 0, True, 1, 1, 1.0), (8, 4, 0, True, 8, 8, 0.0), (16, 8, 0, True, 64, 64, 0.0),
    (32, 16, 8, True, 33, 5, 1.0), (64, 48, 8, False, 7, 3, 2.0), (128, 43, 8, True, 8, 8, 1.0),
    (256, 171, 16, True, 64, 64, 1.0), (512, 256, 24, True, 64, 255, 1.5), (512, 384, 8, False, 3, 1, 3.0),
    (2048, 1024, 16, True, 64, 64, 2.0), (4096, 2048, 16, True, 32, 32, 2.0), (8192, 4096, 24, True, 16, 8, 2.5),
    (1024, 1024, 0, True, 32, 32, 5.0), (1024, 1, 0, True, 32, 32, -2.0), (64, 63, 16, True, 64, 64, 3.0),
]


@pytest.mark.parametrize("N,K,crc,fast,D,L,ebn0", SHAPES)
def test_lane_groups_shapes(oracle_lib, N, K, crc, fast, D, L, ebn0):
    B = max(40, min(1000, 300000 // N))
    fr, msg, cw, llr = make_frames(oracle_lib, N, K, crc, B, ebn0, seed=3 * N + K + D)
    _check(oracle_lib, ps.Plan(N, K, fr, fast_nodes=fast, crc=crc), llr, D, L)


@pytest.mark.parametrize("fast", [False, True])
def test_lane_groups_exact_ties(oracle_lib, fast):
    N, K = 128, 64
    fr, msg, cw, llr = make_frames(oracle_lib, N, K, 8, 1500, 0.0, seed=19, integer=True)
    llr = np.rint(llr / 5.0).astype(np.float32)
    llr[:, ::7] = -0.0
    _check(oracle_lib, ps.Plan(N, K, fr, fast_nodes=fast, crc=8), llr, 16, 4)


def test_lane_groups_random_frozen_sets(oracle_lib):
    rng = np.random.default_rng(23)
    for i in range(16):
        N = int(2 ** rng.integers(3, 11))
        K = int(rng.integers(2, N))
        fr = np.ones(N, np.uint8)
        fr[rng.choice(N, K, replace=False)] = 0
        crc = int(rng.choice([0, 8])) if K > 8 else 0
        _, msg, cw, llr = make_frames(oracle_lib, N, K, crc, 200, 1.0, seed=300 + i, frozen=fr)
        _check(oracle_lib, ps.Plan(N, K, fr, fast_nodes=bool(i % 2), crc=crc), llr, int(rng.integers(1, 65)),
               int(rng.integers(1, 40)))


def test_lane_groups_batch_sizes(oracle_lib):
    """Batches of 1 .. 9 frames leave groups of the last warps without a frame."""
    N, K, crc = 512, 256, 8
    fr, msg, cw, llr = make_frames(oracle_lib, N, K, crc, 64, 1.5, seed=29)
    plan = ps.Plan(N, K, fr, fast_nodes=True, crc=crc)
    for B in (1, 2, 3, 5, 9, 64):
        _check(oracle_lib, plan, llr[:B], 32, 32)


def test_lane_groups_scaled_and_systematic(oracle_lib):
    N, K, crc, D, L = 1024, 512, 16, 32, 32
    fr, msg, cw, llr = make_frames(oracle_lib, N, K, crc, 600, 2.0, seed=37)
    plan = ps.Plan(N, K, fr, fast_nodes=True, crc=crc)
    scales = np.random.default_rng(4).uniform(0.55, 1.25, 10).astype(np.float32)
    plan.set_scales(scales)
    _check(oracle_lib, plan, llr, D, L, scales=scales)
    sys_plan = ps.Plan(N, K, fr, fast_nodes=True, crc=crc, systematic=True)
    cw_s = oracle_lib.encode_batch(msg, N, K, fr, crc, systematic=True)
    llr_s = W.bpsk_awgn_llr(cw_s, W.awgn_noise(37, 600, N), W.sigma_from_ebn0(2.0, K / N))
    st = _check(oracle_lib, sys_plan, llr_s, D, L, systematic=True)
    assert np.any(st == 0)

