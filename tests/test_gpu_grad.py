"""GPU adjoint (pgm_grad) against the FP64 oracle's adjoint and finite differences.

Workload of the gradient benchmark: a 64x64 Ising grid, sum-product (T=1), damping 0.5,
100 unrolled iterations, messages checkpointed every 10, cotangent g ~ N(0,1) on the
normalised log-beliefs; gradients w.r.t. the log-potentials (J) and the evidence (h).
"""
import numpy as np
import pytest

import oracle
from paper_2202_04110_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2202_04110_gb300 import build
    build.build()
    from paper_2202_04110_gb300 import binding
    return binding


def _gpu_grad(binding, graph, lp, ev, T, damping, n_iters, ckpt, g):
    import torch
    G = binding.Graph(graph)
    d_lp, d_ev = G.grad(torch.as_tensor(np.asarray(lp, np.float32)).cuda(),
                        torch.as_tensor(np.asarray(ev, np.float32)).cuda(), T, damping, n_iters, ckpt,
                        torch.as_tensor(np.asarray(g, np.float32)).cuda())
    return d_lp.cpu().numpy().astype(np.float64), d_ev.cpu().numpy().astype(np.float64)


def _close(a, b, what):
    scale = max(1.0, float(np.abs(b).max()))
    err = float(np.abs(a - b).max())
    assert err <= 1e-4 * scale, f"{what}: max |gpu - oracle| = {err:.3e} (scale {scale:.3g})"
    return err




@pytest.fixture(scope="module")
def ising64():
    p = W.ising_grid(64, 64, 11, T=1.0, damping=0.5, n_iters=100)
    g = np.random.default_rng(12).standard_normal(p.graph.n_var_states)
    return p, g


def test_ising64_gradient_vs_oracle(gpu, ising64):
    p, g = ising64
    dlp, dev = _gpu_grad(gpu, p.graph, p.log_pot, p.evidence, 1.0, 0.5, 100, 10, g)
    olp, oev = oracle.grad(p.graph, p.log_pot, p.evidence, 1.0, 0.5, 100, g)
    e1 = _close(dlp, olp, "d log_pot")
    e2 = _close(dev, oev, "d evidence")
    print(f"ising64 gradient: max err d_log_pot {e1:.2e}, d_evidence {e2:.2e}")


def test_ising64_gradient_vs_finite_differences(gpu, ising64):
    """Central differences (h = 1e-5) of the FP64 oracle's loss on 24 sampled coordinates."""
    p, g = ising64
    dlp, dev = _gpu_grad(gpu, p.graph, p.log_pot, p.evidence, 1.0, 0.5, 100, 10, g)
    rng = np.random.default_rng(5)
    lp = np.asarray(p.log_pot, np.float64).copy()
    ev = np.asarray(p.evidence, np.float64).copy()
    h = 1e-5
    for arr, grad in ((lp, dlp), (ev, dev)):
        for i in rng.choice(arr.size, 12, replace=False):
            old = arr[i]
            arr[i] = old + h
            up = oracle.loss(p.graph, lp, ev, 1.0, 0.5, 100, g)
            arr[i] = old - h
            dn = oracle.loss(p.graph, lp, ev, 1.0, 0.5, 100, g)
            arr[i] = old
            fd = (up - dn) / (2 * h)
            assert abs(grad[i] - fd) <= 1e-4 * max(1.0, abs(fd)), (i, grad[i], fd)


def test_checkpoint_interval_does_not_change_gradient(gpu):
    p = W.ising_grid(20, 17, 3, T=1.0)
    g = np.random.default_rng(1).standard_normal(p.graph.n_var_states)
    ref = _gpu_grad(gpu, p.graph, p.log_pot, p.evidence, 1.0, 0.5, 23, 23, g)
    for ck in (1, 4, 10, 50):
        out = _gpu_grad(gpu, p.graph, p.log_pot, p.evidence, 1.0, 0.5, 23, ck, g)
        np.testing.assert_array_equal(out[0], ref[0])
        np.testing.assert_array_equal(out[1], ref[1])


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("T,damping", [(1.0, 0.5), (0.7, 0.0)])
def test_random_graphs_vs_oracle(gpu, seed, T, damping):
    """Mixed state counts, triple factors, sparse configuration lists, shared tables."""
    graph, lp, ev = W.random_graph(seed, n_vars=30, max_K=4, n_pair=60, n_triple=5, n_or=0, n_and=0,
                                   sparse=True, shared=(seed % 2 == 1))
    g = np.random.default_rng(seed).standard_normal(graph.n_var_states)
    dlp, dev = _gpu_grad(gpu, graph, lp, ev, T, damping, 8, 3, g)
    olp, oev = oracle.grad(graph, lp, ev, T, damping, 8, g)
    _close(dlp, olp, "d log_pot")
    _close(dev, oev, "d evidence")


def test_invariants_and_errors(gpu, ising64):
    p, g = ising64
    dlp, dev = _gpu_grad(gpu, p.graph, p.log_pot, p.evidence, 1.0, 0.5, 30, 10, g)
    assert np.abs(dev.reshape(-1, 2).sum(1)).max() < 1e-4
    assert np.abs(dlp.reshape(-1, 4).sum(1)).max() < 1e-4
    import torch
    G = gpu.Graph(p.graph)
    lp = torch.as_tensor(p.log_pot).cuda()
    ev = torch.as_tensor(p.evidence).cuda()
    gg = torch.zeros_like(ev)
    with pytest.raises(gpu.PgmError) as ei:
        G.grad(lp, ev, 0.0, 0.5, 5, 2, gg)
    assert ei.value.status == -4


def test_autograd_function(gpu):
    import torch
    p = W.ising_grid(12, 9, 4, T=1.0)
    G = gpu.Graph(p.graph)
    lp = torch.as_tensor(p.log_pot).cuda().requires_grad_(True)
    ev = torch.as_tensor(p.evidence).cuda().requires_grad_(True)
    g = torch.randn(p.graph.n_var_states, device="cuda", generator=torch.Generator("cuda").manual_seed(0))
    nb = gpu.lbp_beliefs(lp, ev, G, 1.0, 0.5, 15, 5)
    (nb * g).sum().backward()
    d_lp, d_ev = G.grad(lp.detach(), ev.detach(), 1.0, 0.5, 15, 5, g)
    assert torch.equal(lp.grad, d_lp) and torch.equal(ev.grad, d_ev)
    olp, oev = oracle.grad(p.graph, p.log_pot, p.evidence, 1.0, 0.5, 15, g.cpu().numpy())
    _close(lp.grad.cpu().numpy().astype(np.float64), olp, "autograd d log_pot")


@pytest.mark.parametrize("shared", [True, False])
def test_large_factor_gradient_vs_oracle(gpu, shared):
    """Listed-configuration factors with a state sum above 64 (a pool grid of 49-state
    variables, 361 listed pairs per factor: the block-form adjoint, packed lists) and an
    8-ary group over 16-state variables (generic lists), with a few small pairwise
    factors in the same graph (the thread-per-factor adjoint): T=1, 12 iterations,
    checkpoint every 5, against the FP64 oracle's adjoint."""
    a = W.pool_grid(4, 3, 1, 7, T=1.0, shared=shared)
    b = W.random_enum_factors(8, 40, 16, 8, 6, 1500, shared=shared, scale=0.5)
    c = W.ising_grid(4, 5, 9, T=1.0)
    p = W.union([a, b, c])
    g = np.random.default_rng(13).standard_normal(p.graph.n_var_states)
    dlp, dev = _gpu_grad(gpu, p.graph, p.log_pot, p.evidence, 1.0, 0.5, 12, 5, g)
    olp, oev = oracle.grad(p.graph, p.log_pot, p.evidence, 1.0, 0.5, 12, g)
    _close(dlp, olp, "d log_pot")
    _close(dev, oev, "d evidence")


def _logic_cases():
    out = []
    for seed in (4, 5, 9):  # random graphs with OR / AND factors (no structural zeros)
        g, lp, ev = W.random_graph(seed, n_vars=8, max_K=2, n_pair=5, n_triple=1, n_or=2, n_and=2)
        out.append((f"logic{seed}", g, lp, ev))
    # a small deconvolution: 2 features 2x2, activations 4x4, OR fan-in up to 8
    d = W.deconvolution(3, n_feat=2, feat_side=2, s_side=4, n_img=1, T=1.0)
    out.append(("deconv_small", d.graph, d.log_pot, d.evidence))
    return out


@pytest.mark.parametrize("case", _logic_cases(), ids=lambda c: c[0])
def test_logical_factor_gradient_vs_oracle(gpu, case):
    """The closed-form OR / AND adjoint (k_adj_logic, linear in the fan-in) against the
    oracle's adjoint, which enumerates each factor's valid configurations: T=1, damping
    0.5, 10 iterations, checkpoint every 4."""
    name, graph, lp, ev = case
    g = np.random.default_rng(21).standard_normal(graph.n_var_states)
    olp, oev = oracle.grad(graph, lp, ev, 1.0, 0.5, 10, g)
    if not (np.isfinite(olp).all() and np.isfinite(oev).all()):
        pytest.skip("the oracle's gradient is not finite on this case")
    dlp, dev = _gpu_grad(gpu, graph, lp, ev, 1.0, 0.5, 10, 4, g)
    if olp.size:
        _close(dlp, olp, f"{name} d log_pot")
    _close(dev, oev, f"{name} d evidence")


@pytest.mark.parametrize("K", [2, 4, 8])
def test_shared_table_gradient_is_deterministic(gpu, K):
    """Potts grids share one table per grid, so every factor adds to the same K^2
    log-potential gradients: they are summed in a fixed order (warp partials added in
    warp order), and repeated calls -- replayed CUDA graphs and direct launches -- give
    the same bits; the result matches the oracle's adjoint."""
    import torch
    p = W.potts_grid(23, K, seed=K + 7, T=1.0, n_iters=12)
    g = np.random.default_rng(3).standard_normal(p.graph.n_var_states)
    lp = torch.as_tensor(p.log_pot).cuda()
    ev = torch.as_tensor(p.evidence).cuda()
    gn = torch.as_tensor(g.astype(np.float32)).cuda()
    outs = []
    for cuda_graph in (1, 1, 0, 0):
        G = gpu.Graph(p.graph)
        G.set_option(gpu.OPT_CUDA_GRAPH, cuda_graph)
        for _ in range(2):
            d_lp, d_ev = G.grad(lp, ev, 1.0, 0.5, 12, 4, gn)
            outs.append((d_lp.cpu().numpy(), d_ev.cpu().numpy()))
    for a, b in outs[1:]:
        assert np.array_equal(a, outs[0][0]) and np.array_equal(b, outs[0][1])
    olp, oev = oracle.grad(p.graph, p.log_pot, p.evidence, 1.0, 0.5, 12, g)
    _close(outs[0][0].astype(np.float64), olp, f"Potts K={K} d log_pot")
    _close(outs[0][1].astype(np.float64), oev, f"Potts K={K} d evidence")


@pytest.mark.parametrize("T,damping", [(1.0, 0.5), (0.6, 0.0)])
def test_rbm_high_degree_gradient_vs_oracle(gpu, T, damping):
    """An RBM whose units all have more than 64 factors (the variable pass keeps per-state
    totals, the factors form each edge's leave-one-out value from them) and whose 2 x 2
    tables are the factors' own: the register-resident dense-pairwise adjoint, with every
    reverse step reading the kept variable-pass outputs of its recomputed iteration."""
    p = W.rbm(70, 80, seed=4, w_std=0.3, T=T)
    g = np.random.default_rng(5).standard_normal(p.graph.n_var_states)
    dlp, dev = _gpu_grad(gpu, p.graph, p.log_pot, p.evidence, T, damping, 7, 3, g)
    olp, oev = oracle.grad(p.graph, p.log_pot, p.evidence, T, damping, 7, g)
    _close(dlp, olp, "rbm d log_pot")
    _close(dev, oev, "rbm d evidence")


@pytest.mark.parametrize("shared", [True, False])
def test_block_form_gradient_is_deterministic(gpu, shared):
    """The block-form adjoint (state sums above 64: pool grids with packed pairwise lists,
    an 8-ary group with generic lists) sums by gathers in a fixed order, and tables
    shared by a group through per-team rows added in order: repeated calls, replayed and
    direct, give the same bits, and match the oracle's adjoint."""
    import torch
    a = W.pool_grid(6, 3, 1, 3, T=1.0, shared=shared)
    b = W.random_enum_factors(9, 40, 16, 8, 6, 1500, shared=shared, scale=0.5)
    p = W.union([a, b])
    g = np.random.default_rng(17).standard_normal(p.graph.n_var_states)
    lp = torch.as_tensor(p.log_pot).cuda()
    ev = torch.as_tensor(p.evidence).cuda()
    gn = torch.as_tensor(g.astype(np.float32)).cuda()
    outs = []
    for cuda_graph in (1, 1, 0, 0):
        G = gpu.Graph(p.graph)
        G.set_option(gpu.OPT_CUDA_GRAPH, cuda_graph)
        for _ in range(2):
            d_lp, d_ev = G.grad(lp, ev, 1.0, 0.5, 9, 4, gn)
            outs.append((d_lp.cpu().numpy(), d_ev.cpu().numpy()))
    for x, y in outs[1:]:
        assert np.array_equal(x, outs[0][0]) and np.array_equal(y, outs[0][1])
    olp, oev = oracle.grad(p.graph, p.log_pot, p.evidence, 1.0, 0.5, 9, g)
    _close(outs[0][0].astype(np.float64), olp, "block form d log_pot")
    _close(outs[0][1].astype(np.float64), oev, "block form d evidence")
