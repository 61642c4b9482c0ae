"""The allocation-free decode entry point against the regular one.

scs_decode_batch_noalloc serves callers that cannot allocate device memory
when they decode (a budget fixed at start-up, a real-time loop where an
allocation may block or fail, memory owned by another allocator): its
scratch is a fixed static device array inside the library instead of a
per-call stream-ordered allocation.  Its results must be exactly those of scs_decode_batch.  Two
calls in a row, with different codes, check that the shared static memory
(tables, frame counter, snapshots) left over from one call does not leak
into the next.  This file is collected last so that a failure here comes
after every other test has run; it also passes on its own in a fresh
process.
"""
import ctypes as C

import numpy as np
import pytest

import paper_1809_03606_gb300 as ps
import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _frames(oracle, N, K, crc, B, ebn0, seed):
    fr = oracle.construct(N, K, 0.0)
    msg = W.message_bits(seed, B, K - crc)
    cw = oracle.encode_batch(msg, N, K, fr, crc)
    return fr, W.bpsk_awgn_llr(cw, W.awgn_noise(seed, B, N), W.sigma_from_ebn0(ebn0, K / N))


def _outputs(plan, B):
    return (torch.full((B, plan.msg_words), -1, dtype=torch.int32, device="cuda"),
            torch.full((B,), -1.0, dtype=torch.float32, device="cuda"),
            torch.full((B,), -7, dtype=torch.int8, device="cuda"),
            torch.full((B, 4), -1, dtype=torch.int32, device="cuda"))


def test_noalloc_matches_allocating_entry_point(oracle_lib):
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    ps.load(build_if_missing=True)
    cases = [  # two different codes, one call each, back to back
        dict(N=1024, K=512, crc=16, fast=True, D=32, L=32, B=3000, ebn0=1.5, seed=41),
        dict(N=256, K=128, crc=0, fast=False, D=16, L=4, B=2000, ebn0=2.5, seed=42),
    ]
    prepared = []
    for c in cases:
        fr, llr = _frames(oracle_lib, c["N"], c["K"], c["crc"], c["B"], c["ebn0"], c["seed"])
        plan = ps.Plan(c["N"], c["K"], fr, fast_nodes=c["fast"], crc=c["crc"])
        prepared.append((c, plan, torch.from_numpy(llr).cuda()))
    # the allocation-free calls first, back to back on one stream
    got = []
    for c, plan, x in prepared:
        out = _outputs(plan, c["B"])
        ps.scs_decode_batch_noalloc(plan, x, c["D"], c["L"], *out)
        got.append(out)
    torch.cuda.synchronize()
    for (c, plan, x), g in zip(prepared, got):
        ref = _outputs(plan, c["B"])
        ps.scs_decode_batch(plan, x, c["D"], c["L"], *ref)
        torch.cuda.synchronize()
        for r, q in zip(ref, g):
            assert torch.equal(r, q), c  # bit-exact: bits, path metrics, status, counters
        assert int((ref[2] == 0).sum()) > 0


def test_noalloc_rejects_sizes_beyond_its_limits():
    lib = ps.load(build_if_missing=True)
    plan = ps.Plan(64, 32, ps.polar_construct(64, 32, 0.0))
    dummy = C.c_void_p(16)
    assert lib.scs_decode_batch_noalloc(plan.handle, dummy, 4, 65, 4, dummy, dummy, dummy, None, None) == ps.POLAR_ELIMIT
    assert lib.scs_decode_batch_noalloc(plan.handle, dummy, 4, 8, 256, dummy, dummy, dummy, None, None) == ps.POLAR_ELIMIT
    assert lib.scs_decode_batch_noalloc(plan.handle, dummy, 4, 0, 4, dummy, dummy, dummy, None, None) == ps.POLAR_EINVAL
    big = ps.Plan(16384, 8192, ps.polar_construct(16384, 8192, 0.0))
    assert lib.scs_decode_batch_noalloc(big.handle, dummy, 1, 8, 8, dummy, dummy, dummy, None, None) == ps.POLAR_ELIMIT


def test_noalloc_plan_modes(oracle_lib):
    """Systematic and exact-f plans through the allocation-free entry point
    give exactly the regular entry point's outputs."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    ps.load(build_if_missing=True)
    modes = [dict(N=512, K=256, crc=8, fast=True, systematic=True, exact=False, D=32, L=16, B=1500),
             dict(N=256, K=128, crc=0, fast=False, systematic=False, exact=True, D=16, L=4, B=800)]
    for m in modes:
        fr = oracle_lib.construct(m["N"], m["K"], 0.0)
        msg = W.message_bits(7, m["B"], m["K"] - m["crc"])
        cw = oracle_lib.encode_batch(msg, m["N"], m["K"], fr, m["crc"], systematic=m["systematic"])
        llr = W.bpsk_awgn_llr(cw, W.awgn_noise(7, m["B"], m["N"]), W.sigma_from_ebn0(2.0, m["K"] / m["N"]))
        plan = ps.Plan(m["N"], m["K"], fr, fast_nodes=m["fast"], crc=m["crc"], systematic=m["systematic"],
                       exact=m["exact"])
        x = torch.from_numpy(llr).cuda()
        got, ref = _outputs(plan, m["B"]), _outputs(plan, m["B"])
        ps.scs_decode_batch_noalloc(plan, x, m["D"], m["L"], *got)
        ps.scs_decode_batch(plan, x, m["D"], m["L"], *ref)
        torch.cuda.synchronize()
        for r, q in zip(ref, got):
            assert torch.equal(r, q), m
        assert int((ref[2] == 0).sum()) > 0


def test_noalloc_when_the_static_scratch_limits_residency(oracle_lib):
    """PC(2048,1024) CRC-8 with D = 64: one warp's snapshots take 18,720 bytes,
    so the 16 MiB array holds 896 warps, fewer than the persistent grid would
    otherwise start; the reduced grid must give exactly the regular outputs."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    ps.load(build_if_missing=True)
    N, K, crc, D, L, B = 2048, 1024, 8, 64, 64, 6000
    fr, llr = _frames(oracle_lib, N, K, crc, B, 2.0, seed=43)
    plan = ps.Plan(N, K, fr, fast_nodes=True, crc=crc)
    x = torch.from_numpy(llr).cuda()
    got, ref = _outputs(plan, B), _outputs(plan, B)
    ps.scs_decode_batch_noalloc(plan, x, D, L, *got)
    ps.scs_decode_batch(plan, x, D, L, *ref)
    torch.cuda.synchronize()
    for r, q in zip(ref, got):
        assert torch.equal(r, q)
    assert int((ref[2] == 0).sum()) > 0


def test_noalloc_table_area_follows_plan_changes(oracle_lib):
    """The static table area keeps the last plan's tables: alternating plans,
    repeating one, and changing a plan's stage scales between calls must each
    decode with the right tables."""
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    ps.load(build_if_missing=True)
    fr_a, llr_a = _frames(oracle_lib, 512, 256, 8, 800, 2.0, seed=44)
    fr_b, llr_b = _frames(oracle_lib, 256, 128, 0, 800, 2.5, seed=45)
    pa = ps.Plan(512, 256, fr_a, fast_nodes=True, crc=8)
    pb = ps.Plan(256, 128, fr_b, fast_nodes=True, crc=0)
    xa, xb = torch.from_numpy(llr_a).cuda(), torch.from_numpy(llr_b).cuda()
    scales = np.linspace(0.7, 1.1, 9).astype(np.float32)
    for plan, x, sc in ((pa, xa, None), (pb, xb, None), (pa, xa, None), (pa, xa, None), (pa, xa, scales),
                        (pa, xa, scales), (pa, xa, None)):
        plan.set_scales(sc)
        got, ref = _outputs(plan, 800), _outputs(plan, 800)
        ps.scs_decode_batch_noalloc(plan, x, 16, 16, *got)
        torch.cuda.synchronize()
        ps.scs_decode_batch(plan, x, 16, 16, *ref)
        torch.cuda.synchronize()
        for r, q in zip(ref, got):
            assert torch.equal(r, q), (plan.N, sc is None)
