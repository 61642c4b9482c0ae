"""Persisted state: the mixed-batch autotuner's results kept in a JSON file
(polar_plan_set_tuning / polar_plan_set_get_tuning, TuningCache,
tune_mixed_cached) and learned stage scales written to and read from a file.
The decoder itself is stateless across frames; these are the two results a
later run restores instead of recomputing."""
import json

import numpy as np
import pytest

import paper_1809_03606_gb300 as ps


@pytest.fixture(scope="module")
def lib():
    ps.load(build_if_missing=True)
    return ps.load()


def _set(Ns=((64, 32, 8), (128, 64, 8))):
    plans = [ps.Plan(N, K, ps.polar_construct(N, K, 0.0), fast_nodes=True, crc=crc) for N, K, crc in Ns]
    return ps.PlanSet(plans)


def test_set_tuning_round_trip_and_limits(lib):
    pset = _set()
    assert ps.polar_plan_set_get_tuning(pset) == (0, 0)
    for w, c in ((1, 1), (2, 16), (4, 1024)):
        ps.polar_plan_set_tuning(pset, w, c)
        assert ps.polar_plan_set_get_tuning(pset) == (w, c)
    ps.polar_plan_set_tuning(pset, 0, 0)  # back to the defaults
    assert ps.polar_plan_set_get_tuning(pset) == (0, 0)
    for w, c in ((3, 1), (8, 1), (4, 0), (4, 1025), (0, 4), (-1, 1)):
        assert lib.polar_plan_set_tuning(pset.handle, w, c) == ps.POLAR_EINVAL
    assert ps.polar_plan_set_get_tuning(pset) == (0, 0)  # a refused call changes nothing
    assert lib.polar_plan_set_tuning(None, 4, 1) == ps.POLAR_EINVAL
    assert lib.polar_plan_set_get_tuning(pset.handle, None, None) == ps.POLAR_EINVAL


def test_tuning_key_names_gpu_d_and_every_code(lib):
    a, b = _set(), _set(((64, 32, 8), (128, 64, 0)))
    keys = {ps.tuning_key(a, 32, "GPU A"), ps.tuning_key(a, 64, "GPU A"), ps.tuning_key(a, 32, "GPU B"),
            ps.tuning_key(b, 32, "GPU A")}
    assert len(keys) == 4
    assert ps.tuning_key(a, 32, "GPU A") == ps.tuning_key(_set(), 32, "GPU A")  # same codes, same key
    fr = ps.polar_construct(128, 64, 0.0).copy()
    i0, i1 = np.nonzero(fr == 1)[0][0], np.nonzero(fr == 0)[0][0]
    fr[i0], fr[i1] = 0, 1  # another frozen set of the same size
    c = ps.PlanSet([a.plans[0], ps.Plan(128, 64, fr, fast_nodes=True, crc=8)])
    assert ps.tuning_key(c, 32, "GPU A") != ps.tuning_key(a, 32, "GPU A")


def test_cache_runs_the_tuner_once_per_key(lib, tmp_path):
    path = str(tmp_path / "tuning.json")
    cache = ps.TuningCache(path)
    calls = []

    def tuner(pset, *args, **kw):
        calls.append(1)
        return 2, 4

    args = (None, 32) + (None,) * 6  # D = 32; the stub tuner needs no batch
    pset = _set()
    assert ps.tune_mixed_cached(cache, pset, *args, device="GPU A", tuner=tuner) == (2, 4, False)
    assert ps.polar_plan_set_get_tuning(pset) == (2, 4)
    fresh = _set()  # a later run: same codes, a new set without tuning
    assert ps.tune_mixed_cached(ps.TuningCache(path), fresh, *args, device="GPU A", tuner=tuner) == (2, 4, True)
    assert ps.polar_plan_set_get_tuning(fresh) == (2, 4)
    assert len(calls) == 1
    ps.tune_mixed_cached(cache, _set(), None, 64, *args[2:], device="GPU A", tuner=tuner)  # another D
    assert len(calls) == 2
    data = json.load(open(path))
    assert sorted(data.values()) == [[2, 4], [2, 4]]
    with open(path, "w") as f:
        f.write("[1, 2]")
    with pytest.raises(ValueError):
        cache.lookup("x")


def test_scales_round_trip_exactly(tmp_path):
    rng = np.random.default_rng(7)
    sc = (rng.random(10) * 1.5 + 0.25).astype(np.float32)
    sc[3] = np.float32(1.0) - np.float32(2.0 ** -24)  # values that need every mantissa bit
    sc[7] = np.nextafter(np.float32(0.8), np.float32(1.0))
    path = str(tmp_path / "scales.json")
    ps.save_scales(path, sc)
    back = ps.load_scales(path)
    assert back.dtype == np.float32 and np.array_equal(back.view(np.uint32), sc.view(np.uint32))
    data = json.load(open(path))
    data["stages"] = 9
    json.dump(data, open(path, "w"))
    with pytest.raises(ValueError):
        ps.load_scales(path)


@pytest.mark.gpu
def test_cached_tuning_on_gpu(lib, tmp_path):
    """The native autotuner through the cache: the first call times the shapes
    and stores the winner, a new set with the same codes takes it from the
    file, and decoding with the restored shape gives the same outputs as with
    the defaults."""
    torch = pytest.importorskip("torch")
    codes = [(128, 64, 8), (256, 128, 8), (512, 256, 8)]
    plans = [ps.Plan(N, K, ps.polar_construct(N, K, 0.0), fast_nodes=True, crc=crc) for N, K, crc in codes]
    rng = np.random.default_rng(11)
    B = 4000
    idx = rng.integers(0, len(codes), B).astype(np.int32)
    D = rng.choice([8, 16, 32], B).astype(np.int32)
    # LLRs of the all-zero codeword with Gaussian noise: any codeword decodes the same way
    llr = (rng.standard_normal((B, 512)) * 1.5 + 2.0).astype(np.float32)
    rows = [llr[b, :codes[idx[b]][0]] for b in range(B)]
    path = str(tmp_path / "tuning.json")
    pset = ps.PlanSet(plans)
    mb = ps.MixedBatch(pset, idx, D, D, rows)
    mb.decode(pset)
    torch.cuda.synchronize()
    ref = (mb.info.clone(), mb.pm.clone(), mb.status.clone())
    args = (mb.frames, mb.Dmax, mb.llr, mb.llr_off, mb.info, mb.info_off, mb.pm, mb.status)
    w, c, hit = ps.tune_mixed_cached(ps.TuningCache(path), pset, *args)
    assert not hit and w in (1, 2, 4) and c in (1, 4, 16)
    fresh = ps.PlanSet(plans)
    mb2 = ps.MixedBatch(fresh, idx, D, D, rows)
    args2 = (mb2.frames, mb2.Dmax, mb2.llr, mb2.llr_off, mb2.info, mb2.info_off, mb2.pm, mb2.status)
    assert ps.tune_mixed_cached(ps.TuningCache(path), fresh, *args2) == (w, c, True)
    mb2.decode(fresh)
    torch.cuda.synchronize()
    for r, g in zip(ref, (mb2.info, mb2.pm, mb2.status)):
        assert torch.equal(r, g)
