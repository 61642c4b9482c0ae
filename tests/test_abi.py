"""Host-side checks of the C ABI (no GPU): the library loads, exports every
function that include/polarscs.h declares, builds the same schedule and code
as the oracle from the same definitions, and rejects invalid arguments before
any device work."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import paper_1809_03606_gb300 as ps

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1809_03606_gb300 import _build

    _build.build()
    return ps.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "polarscs.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void)\s+\**\s*(\w+)\s*\(", text, flags=re.M)))


def test_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert len(names) >= 9
    for name in names:
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), C._CFuncPtr)
    assert set(names) == set(ps.EXPORTED)


@pytest.mark.parametrize("N", [2, 8, 64, 256, 1024, 2048])
@pytest.mark.parametrize("snr", [0.0, 2.0])
def test_construct_agrees_with_oracle(lib, oracle_lib, N, snr):
    for K in sorted({1, max(1, N // 4), N // 2, (3 * N) // 4, N}):
        assert np.array_equal(ps.polar_construct(N, K, snr), oracle_lib.construct(N, K, snr))


def test_construct_rejects_bad_sizes(lib):
    with pytest.raises(ps.PolarError):
        ps.polar_construct(12, 4, 0.0)
    with pytest.raises(ps.PolarError):
        ps.polar_construct(16, 0, 0.0)
    with pytest.raises(ps.PolarError):
        ps.polar_construct(16, 17, 0.0)


@pytest.mark.parametrize("fast", [False, True])
@pytest.mark.parametrize("N,K", [(8, 4), (16, 5), (64, 32), (256, 128), (1024, 512), (2048, 1365), (128, 32)])
def test_plan_schedule_agrees_with_oracle(lib, oracle_lib, fast, N, K):
    """The plan builder and the oracle both follow Sec. 3.1 / Fig. fsscsch."""
    fr = oracle_lib.construct(N, K, 0.0)
    plan = ps.Plan(N, K, fr, fast_nodes=fast)
    assert plan.schedule() == oracle_lib.schedule(N, fr, fast)


def test_plan_schedule_fig_fsscsch(lib):
    from conftest import read_golden

    want = [(op, int(l), int(p)) for op, l, p in read_golden("pc8_4_fssc_schedule.txt")]
    plan = ps.Plan(8, 4, ps.polar_construct(8, 4, 0.0), fast_nodes=True)
    assert plan.schedule() == want


def test_plan_random_frozen_sets(lib, oracle_lib):
    rng = np.random.default_rng(0)
    for _ in range(200):
        N = int(2 ** rng.integers(1, 9))
        K = int(rng.integers(1, N + 1))
        fr = np.ones(N, np.uint8)
        fr[rng.choice(N, K, replace=False)] = 0
        for fast in (False, True):
            assert ps.Plan(N, K, fr, fast_nodes=fast).schedule() == oracle_lib.schedule(N, fr, fast)


def test_plan_rejects_invalid(lib):
    fr = ps.polar_construct(16, 8, 0.0)
    for args in [(16, 9, fr, True, 0), (16, 8, fr, True, 12), (16, 8, fr, True, 8), (12, 8, np.zeros(12, np.uint8), True, 0)]:
        with pytest.raises(ps.PolarError) as e:
            ps.Plan(*args)
        assert e.value.rc == ps.POLAR_EINVAL


def test_decode_batch_validates_before_device_work(lib):
    """Argument and size checks return before any CUDA call, so they run here."""
    fr = ps.polar_construct(64, 32, 0.0)
    plan = ps.Plan(64, 32, fr)
    h = plan.handle
    dummy = C.c_void_p(16)
    assert lib.scs_decode_batch(h, dummy, 4, 0, 4, dummy, dummy, dummy, None, None) == ps.POLAR_EINVAL
    assert lib.scs_decode_batch(h, dummy, 4, 4, 0, dummy, dummy, dummy, None, None) == ps.POLAR_EINVAL
    assert lib.scs_decode_batch(h, None, 4, 4, 4, dummy, dummy, dummy, None, None) == ps.POLAR_EINVAL
    assert lib.scs_decode_batch(h, dummy, 4, ps.MAX_D_GPU_DEEP + 1, 4, dummy, dummy, dummy, None, None) == ps.POLAR_ELIMIT
    # D > 64 needs the memory stack: the uniform decoder of a min-sum plan only
    assert lib.scs_decode_batch_noalloc(h, dummy, 4, 65, 4, dummy, dummy, dummy, None, None) == ps.POLAR_ELIMIT
    ex = ps.Plan(64, 32, fr, fast_nodes=False, exact=True)
    assert lib.scs_decode_batch(ex.handle, dummy, 4, 65, 4, dummy, dummy, dummy, None, None) == ps.POLAR_ELIMIT
    assert lib.scs_decode_batch(h, dummy, 4, 8, 256, dummy, dummy, dummy, None, None) == ps.POLAR_ELIMIT
    assert lib.scs_decode_batch(h, dummy, 0, 8, 8, None, None, None, None, None) == 0  # empty batch: no-op
    big = ps.Plan(16384, 8192, ps.polar_construct(16384, 8192, 0.0))
    assert lib.scs_decode_batch(big.handle, dummy, 1, 8, 8, dummy, dummy, dummy, None, None) == ps.POLAR_ELIMIT
    assert lib.polar_encode_batch(None, dummy, 1, dummy, None) == ps.POLAR_EINVAL
    assert lib.polar_encode_batch(h, dummy, 0, None, None) == 0


def test_bit_packing_round_trip():
    rng = np.random.default_rng(1)
    for k in (1, 31, 32, 33, 496, 1024):
        bits = rng.integers(0, 2, (5, k)).astype(np.uint8)
        w = ps.pack_bits(bits)
        assert w.shape == (5, (k + 31) // 32)
        assert np.array_equal(ps.unpack_bits(w, k), bits)
    w = ps.pack_bits(np.array([[1, 0, 1] + [0] * 29 + [1]], np.uint8))
    assert w.view(np.uint32)[0, 0] == 0b101 and w.view(np.uint32)[0, 1] == 1


def test_set_systematic_host_checks(lib):
    """polar_plan_set_systematic: the two-pass encoder check and argument checks
    (host logic only; nothing touches a device)."""
    N, K = 1024, 512
    fr = ps.polar_construct(N, K, 0.0)
    plan = ps.Plan(N, K, fr, fast_nodes=True, crc=16, systematic=True)
    assert plan.systematic
    ps.polar_plan_set_systematic(plan, False)
    assert not plan.systematic
    assert lib.polar_plan_set_systematic(None, 1) == ps.POLAR_EINVAL
    # information set {1, 3, 7} of N = 8: three members lie between 1 and 7
    # in the bit-subset order, so two passes of the XOR tree are not systematic
    fr8 = np.ones(8, np.uint8)
    fr8[[1, 3, 7]] = 0
    p8 = ps.Plan(8, 3, fr8, fast_nodes=False)
    assert lib.polar_plan_set_systematic(p8.handle, 1) == ps.POLAR_EINVAL
    assert lib.polar_plan_set_systematic(p8.handle, 0) == 0
    # {1, 7}: two members between 1 and 7 (an even number), so two passes
    # are systematic although 3 and 5 are frozen
    fr8 = np.ones(8, np.uint8)
    fr8[[1, 7]] = 0
    p8b = ps.Plan(8, 2, fr8, fast_nodes=False)
    assert lib.polar_plan_set_systematic(p8b.handle, 1) == 0


def test_set_exact_host_checks(lib):
    """polar_plan_set_exact takes bit-level plans without scales only, and
    plan sets refuse exact plans (host logic only)."""
    fr = ps.polar_construct(256, 128, 0.0)
    fast = ps.Plan(256, 128, fr, fast_nodes=True)
    assert lib.polar_plan_set_exact(fast.handle, 1) == ps.POLAR_EINVAL
    assert lib.polar_plan_set_exact(None, 1) == ps.POLAR_EINVAL
    scaled = ps.Plan(256, 128, fr, fast_nodes=False)
    scaled.set_scales(np.ones(8, np.float32))
    assert lib.polar_plan_set_exact(scaled.handle, 1) == ps.POLAR_EINVAL
    ex = ps.Plan(256, 128, fr, fast_nodes=False, exact=True)
    assert ex.exact
    with pytest.raises(ps.PolarError):
        ex.set_scales(np.ones(8, np.float32))
    with pytest.raises(ps.PolarError) as e:
        ps.PlanSet([ex])
    assert e.value.rc == ps.POLAR_EINVAL
