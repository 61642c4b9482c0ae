"""Genie-aided SC with per-stage min-sum scales: forward and hand-written
reverse kernels against the double-precision oracle, autograd gradcheck of
the CUDA kernels in float64, determinism, and a short training run."""
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


def _problem(oracle, N, K, B, ebn0, seed):
    fr = oracle.construct(N, K, 0.0)
    msg = W.message_bits(seed, B, K)
    cw = oracle.encode_batch(msg, N, K, fr, 0)
    llr = W.bpsk_awgn_llr(cw, W.awgn_noise(seed, B, N), W.sigma_from_ebn0(ebn0, K / N))
    u = np.zeros((B, N), np.uint8)
    u[:, fr == 0] = msg
    plan = ps.Plan(N, K, fr, fast_nodes=False)
    return fr, plan, llr, u, torch.from_numpy(ps.pack_bits(u)).cuda()


@pytest.mark.parametrize("N,K", [(16, 8), (256, 128), (1024, 512)])
def test_forward_and_gradient_match_fp64_oracle(oracle_lib, N, K):
    B = 192
    fr, plan, llr, u, uw = _problem(oracle_lib, N, K, B, 2.0, seed=N)
    n = int(np.log2(N))
    scales = np.random.default_rng(N).uniform(0.6, 1.2, n)
    ref_loss, ref_grad = oracle_lib.gsc_loss_grad(llr.astype(np.float64), u, fr, scales)
    ref_leaf = np.array([oracle_lib.gsc_forward(llr[b].astype(np.float64), u[b], scales) for b in range(8)])
    for dt, tol in ((torch.float32, 1e-4), (torch.float64, 1e-10)):
        x = torch.from_numpy(llr).to(dt).cuda()
        s = torch.from_numpy(scales).to(dt).cuda()
        leaf = torch.empty_like(x)
        loss0 = ps.gsc_loss(plan, x, uw, s, leaf=leaf)
        loss, g, gl = ps.gsc_loss_grad(plan, x, uw, s, want_llr_grad=True)
        torch.cuda.synchronize()
        lf = leaf[:8].double().cpu().numpy()
        assert np.max(np.abs(lf - ref_leaf)) <= tol * 10 * max(1.0, np.max(np.abs(ref_leaf)))
        assert abs(loss0.item() - ref_loss) <= tol * abs(ref_loss) and loss.item() == loss0.item()
        gg = g.double().cpu().numpy()
        assert np.max(np.abs(gg - ref_grad)) <= tol * max(1e-3, np.max(np.abs(ref_grad))), (dt, gg, ref_grad)
        assert gl is not None and gl.shape == x.shape


def test_gradcheck_cuda_fp64():
    """torch.autograd.gradcheck of the CUDA forward and reverse kernels in float64 (N = 16, K = 8)."""
    import oracle

    fr, plan, llr, u, uw = _problem(oracle, 16, 8, 6, 1.0, seed=3)
    x = torch.from_numpy(llr.astype(np.float64)).cuda().requires_grad_(True)
    s = torch.tensor(np.random.default_rng(4).uniform(0.7, 1.1, 4), dtype=torch.float64, device="cuda",
                     requires_grad=True)
    assert torch.autograd.gradcheck(lambda a, b: ps.genie_sc_loss(a, b, uw, plan), (x, s), eps=1e-6, atol=1e-7,
                                    rtol=1e-5)


def test_deterministic_and_training_reduces_loss(oracle_lib):
    fr, plan, llr, u, uw = _problem(oracle_lib, 1024, 512, 4096, 2.0, seed=11)
    x = torch.from_numpy(llr).cuda()
    s = torch.ones(10, dtype=torch.float32, device="cuda", requires_grad=True)
    l1, g1, _ = ps.gsc_loss_grad(plan, x, uw, s.detach())
    l2, g2, _ = ps.gsc_loss_grad(plan, x, uw, s.detach())
    torch.cuda.synchronize()
    assert torch.equal(l1, l2) and torch.equal(g1, g2)
    opt = torch.optim.Adam([s], lr=0.02)
    first = None
    for _ in range(30):
        opt.zero_grad()
        loss = ps.genie_sc_loss(x, s, uw, plan)
        loss.backward()
        opt.step()
        first = loss.item() if first is None else first
    final = ps.genie_sc_loss(x, s, uw, plan).item()
    assert final < first


def test_llr_gradient_at_n1024(oracle_lib):
    """d loss / d llr at N = 1024, where the float kernel takes its vector
    paths: central differences of the double-precision loss at a few entries
    pin the double gradient, and the float gradient agrees with it."""
    B, N, K = 64, 1024, 512
    fr, plan, llr, u, uw = _problem(oracle_lib, N, K, B, 2.0, seed=17)
    scales = np.random.default_rng(17).uniform(0.6, 1.2, 10)
    x64 = torch.from_numpy(llr.astype(np.float64)).cuda()
    s64 = torch.from_numpy(scales).cuda()
    _, _, gl64 = ps.gsc_loss_grad(plan, x64, uw, s64, want_llr_grad=True)
    torch.cuda.synchronize()
    rng = np.random.default_rng(18)
    h = 1e-7  # the loss is piecewise smooth: a small step rarely crosses a min-sum kink
    for b, i in zip(rng.integers(0, B, 8), rng.integers(0, N, 8)):
        xp, xm = x64.clone(), x64.clone()
        xp[b, i] += h
        xm[b, i] -= h
        fd = (ps.gsc_loss(plan, xp, uw, s64).item() - ps.gsc_loss(plan, xm, uw, s64).item()) / (2 * h)
        got = gl64[b, i].item()
        assert abs(fd - got) <= 1e-5 * max(abs(fd), 1.0 / (B * K)), (b, i, fd, got)
    _, _, gl32 = ps.gsc_loss_grad(plan, x64.float(), uw, s64.float(), want_llr_grad=True)
    torch.cuda.synchronize()
    ref = gl64.cpu().numpy()
    assert np.max(np.abs(gl32.double().cpu().numpy() - ref)) <= 1e-4 * np.max(np.abs(ref))
