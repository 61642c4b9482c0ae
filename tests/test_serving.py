"""Serving with continuous batching (polar_serve) and its one-size-per-launch
baseline: every served request's result equals the CPU oracle's decode of
its frame (message bits, path-metric bits, status) and the same frame
decoded alone on the GPU, under arena pressure (admission stalls) and
interleaving; a device wait that runs out ends the engine cleanly with
POLAR_ETIMEOUT."""
import numpy as np
import pytest

import paper_1809_03606_gb300 as ps
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CODES = [(128, 64, 8), (256, 171, 8), (512, 128, 8), (1024, 683, 8), (2048, 1024, 8)]


@pytest.fixture(scope="module")
def pool(oracle_lib):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    ps.load(build_if_missing=True)
    rng = np.random.default_rng(8)
    plans = [ps.Plan(N, K, oracle_lib.construct(N, K, 0.0), fast_nodes=True, crc=crc) for N, K, crc in CODES]
    P = 1200
    idx = rng.integers(0, len(CODES), P).astype(np.int32)
    D = rng.choice([8, 16, 32, 64], P).astype(np.int32)
    eb = rng.uniform(1.0, 4.0, P)
    rows = []
    for p in range(P):
        N, K, crc = CODES[idx[p]]
        msg = W.message_bits(1000 + p, 1, K - crc)
        cw = oracle_lib.encode_msg(msg[0], N, K, plans[idx[p]].frozen, crc)
        rows.append(W.bpsk_awgn_llr(cw[None, :], W.awgn_noise(1000 + p, 1, N), W.sigma_from_ebn0(eb[p], K / N))[0])
    off = np.concatenate([[0], np.cumsum([r.size for r in rows])[:-1]]).astype(np.int64)
    flat = np.concatenate(rows).astype(np.float32)
    return dict(plans=plans, pset=ps.PlanSet(plans), idx=idx, D=D, rows=rows, off=off, flat=flat, P=P)


def _oracle(pool, oracle_lib):
    """The CPU oracle's (message bits, pm, status) of every pool frame, decoded
    with its own code, D and L = D (fast nodes, CRC-8)."""
    out = {}
    for p in range(pool["P"]):
        N, K, crc = CODES[pool["idx"][p]]
        d = int(pool["D"][p])
        st, m, pm, _, _ = oracle_lib.scs_decode(pool["rows"][p], N, K, pool["plans"][pool["idx"][p]].frozen,
                                                fast=True, D=d, L=d, crc_len=crc)
        out[p] = (m, np.float32(pm), int(st))
    return out


def _solo(pool):
    """pm, status and message words of every pool frame decoded alone."""
    out = {}
    for key in sorted(set(zip(pool["idx"].tolist(), pool["D"].tolist()))):
        ci, d = key
        sel = [p for p in range(pool["P"]) if pool["idx"][p] == ci and pool["D"][p] == d]
        x = torch.from_numpy(np.stack([pool["rows"][p] for p in sel])).cuda()
        info, pm, st = ps.decode(pool["plans"][ci], x, d, d)
        torch.cuda.synchronize()
        for j, p in enumerate(sel):
            out[p] = (pm[j].item(), int(st[j].item()), info[j].cpu().numpy().view(np.uint32))
    return out


def _requests(pool, R, rate, seed):
    arr = W.poisson_arrivals(seed, rate, R / rate * 1.5)[:R]
    p = np.arange(R) % pool["P"]
    req = np.stack([pool["idx"][p], pool["D"][p], pool["D"][p], p], axis=1).astype(np.int32)
    return req, arr, p


def test_served_results_equal_oracle_and_solo_under_arena_pressure(pool, oracle_lib):
    solo = _solo(pool)
    ref = _oracle(pool, oracle_lib)
    # the GPU's solo decode is itself bit-exact against the oracle on the pool
    for p in range(pool["P"]):
        m_o, pm_o, st_o = ref[p]
        pm_s, st_s, info_s = solo[p]
        kmsg = m_o.size
        assert np.array_equal(ps.unpack_bits(info_s[None, :], kmsg)[0], m_o), p
        assert np.float32(pm_s).view(np.uint32) == pm_o.view(np.uint32) and st_s == st_o, p
    R = 3000
    req, arr, p = _requests(pool, R, 3e5, seed=21)
    words = np.array([pool["plans"][i].msg_words for i in req[:, 0]], np.int64)
    ioff = np.concatenate([[0], np.cumsum(words)[:-1]])
    out = ps.polar_serve(pool["pset"], req, arr, pool["flat"], pool["off"], arena_floats=20000, wait_s=20.0,
                         info_off=ioff)
    assert out["rc"] == 0 and out["report"]["completed"] == R
    assert out["report"]["arena_full_stalls"] > 0  # admission by memory really happened
    assert np.all(out["latency"] >= 0)
    # service time (a warp's start to completion, device clock) within latency
    assert np.all(out["service"] > 0) and np.all(out["service"] <= out["latency"] + 1e-4)
    for r in range(R):
        pm_s, st_s, info_s = solo[int(p[r])]
        m_o, pm_o, st_o = ref[int(p[r])]
        served = out["info"][ioff[r]:ioff[r] + words[r]]
        # against the oracle: message bits, path-metric bits, status
        assert np.array_equal(ps.unpack_bits(np.asarray(served)[None, :], m_o.size)[0], m_o), r
        assert np.float32(out["pm"][r]).view(np.uint32) == pm_o.view(np.uint32), r
        assert int(out["status"][r]) == st_o, r
        # and against the same frame decoded alone
        assert np.float32(out["pm"][r]) == np.float32(pm_s) and out["status"][r] == st_s
        assert np.array_equal(served, info_s)
    base = ps.polar_serve_baseline(pool["pset"], req, arr, pool["flat"], pool["off"], arena_floats=200000,
                                   interval_s=2e-3, wait_s=20.0)
    assert base["rc"] == 0 and base["report"]["completed"] == R
    assert np.array_equal(base["pm"].view(np.uint32), out["pm"].view(np.uint32))
    assert np.array_equal(base["status"], out["status"])


def test_served_wait_runs_out_cleanly(pool):
    """The last request arrives long after the device-side wait limit: the
    waiting warps give up, the engine returns POLAR_ETIMEOUT, every earlier
    request is complete and the GPU is usable afterwards."""
    R = 400
    req, arr, p = _requests(pool, R, 1e5, seed=22)
    arr = arr.copy()
    arr[-1] = arr[-2] + 0.6
    out = ps.polar_serve(pool["pset"], req, arr, pool["flat"], pool["off"], arena_floats=1 << 20, wait_s=0.1)
    assert out["rc"] == ps.POLAR_ETIMEOUT and out["report"]["error"] == 1.0
    assert out["report"]["completed"] >= R - 1 - 256  # requests published before the warps gave up
    assert np.all(out["latency"][: R - 300] >= 0)
    x = torch.ones(4, device="cuda")
    assert float(x.sum().item()) == 4.0  # the context is alive
    again = ps.polar_serve(pool["pset"], req[:100], arr[:100], pool["flat"], pool["off"], arena_floats=1 << 20,
                           wait_s=10.0)
    assert again["rc"] == 0 and again["report"]["completed"] == 100
