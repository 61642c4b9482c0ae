"""The bounds-checked debug build (POLAR_DEBUG): it compiles for sm_103a, and
on the GPU it decodes exactly like the regular library (bit-exact against
the oracle) with no index check failing (no POLAR_DEBUG_FAIL status), over
the register stack, the memory stack, systematic and mixed batches."""
import os
import subprocess
import sys

import pytest

from paper_1809_03606_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHECK = r'''
import sys
import numpy as np
import torch
sys.path.insert(0, sys.argv[1])
sys.path.insert(0, sys.argv[1] + "/tests")
import oracle
import paper_1809_03606_gb300 as ps
import workloads as W
from test_gpu_parity import make_frames
assert ps.lib_path().endswith("libpolarscs_debug.so")
ps.load()
cases = [(1024, 512, 16, True, 32, 32, 1.5, False), (256, 128, 0, False, 16, 4, 2.5, False),
         (512, 256, 8, True, 64, 64, 1.0, False), (1024, 512, 24, True, 8192, 8, 1.0, True),
         (2048, 1024, 8, True, 100, 16, 1.5, False), (8, 4, 0, True, 8, 8, 0.0, False)]
for N, K, crc, fast, D, L, e, sysf in cases:
    fr = oracle.construct(N, K, 0.0)
    msg = W.message_bits(N + D, 300, K - crc)
    cw = oracle.encode_batch(msg, N, K, fr, crc, systematic=sysf)
    llr = W.bpsk_awgn_llr(cw, W.awgn_noise(N + D, 300, N), W.sigma_from_ebn0(e, K / N))
    plan = ps.Plan(N, K, fr, fast_nodes=fast, crc=crc, systematic=sysf)
    info, pm, st, stats = ps.decode(plan, torch.from_numpy(llr).cuda(), D, L, with_stats=True)
    torch.cuda.synchronize()
    st = st.cpu().numpy()
    assert not np.any(st == ps.POLAR_DEBUG_FAIL), (N, D)
    m_o, pm_o, st_o, stats_o = oracle.scs_decode_batch(llr, N, K, fr, fast=fast, D=D, L=L, crc_len=crc,
                                                       threads=8, systematic=sysf)
    assert np.array_equal(ps.unpack_bits(info.cpu().numpy(), K - crc), m_o), (N, D)
    assert np.array_equal(pm.cpu().numpy().view(np.uint32), pm_o.view(np.uint32)) and np.array_equal(st, st_o)
    assert np.array_equal(stats.cpu().numpy().view(np.uint32), stats_o.astype(np.uint32)), (N, D)
# a mixed batch
codes = [(128, 64, 8), (512, 256, 8), (1024, 683, 8)]
plans = [ps.Plan(N, K, oracle.construct(N, K, 0.0), fast_nodes=True, crc=c) for N, K, c in codes]
rng = np.random.default_rng(3)
idx = rng.integers(0, 3, 600).astype(np.int32)
D = rng.integers(1, 65, 600).astype(np.int32)
rows = []
for b in range(600):
    N, K, c = codes[idx[b]]
    msg = W.message_bits(500 + b, 1, K - c)
    cw = oracle.encode_msg(msg[0], N, K, plans[idx[b]].frozen, c)
    rows.append(W.bpsk_awgn_llr(cw[None, :], W.awgn_noise(500 + b, 1, N), W.sigma_from_ebn0(2.0, K / N))[0])
pset = ps.PlanSet(plans)
mb = ps.MixedBatch(pset, idx, D, D, rows)
mb.decode_split(pset)
torch.cuda.synchronize()
st = mb.status.cpu().numpy()
assert not np.any(st == ps.POLAR_DEBUG_FAIL)
for b in range(0, 600, 7):
    N, K, c = codes[idx[b]]
    st_o, m_o, pm_o, _, _ = oracle.scs_decode(rows[b], N, K, plans[idx[b]].frozen, fast=True, D=int(D[b]), L=int(D[b]),
                                               crc_len=c)
    assert np.array_equal(ps.unpack_bits(mb.message_words(b)[None, :], K - c)[0], m_o) and st[b] == st_o
print("debug build ok")
'''


def test_debug_build_compiles():
    lib = _build.build(variant="debug")
    assert os.path.exists(lib) and lib.endswith("libpolarscs_debug.so")


@pytest.mark.gpu
def test_debug_build_decodes_like_the_library(oracle_lib):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    lib = _build.build(variant="debug")
    env = dict(os.environ, POLARSCS_LIB=lib)
    r = subprocess.run([sys.executable, "-c", CHECK, ROOT], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    assert "debug build ok" in r.stdout
