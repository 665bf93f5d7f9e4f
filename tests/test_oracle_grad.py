"""Pins for the oracle's adjoint (gradient of normalised log-beliefs; Sec. 5.3 on using LBP inside differentiable programs):
central finite differences of the oracle's own pinned forward pass, in FP64, on every
coordinate of small graphs (including logical OR / AND factors), plus the shift invariances the gradient must satisfy
(normalised beliefs do not change when a constant is added to one variable's evidence or
to one factor's log-potentials, so those gradients sum to zero)."""
import numpy as np
import pytest

import oracle
from paper_2202_04110_gb300 import workloads as W


def _fd(graph, lp, ev, T, damping, n_iters, g, h=1e-6):
    lp = np.asarray(lp, np.float64)
    ev = np.asarray(ev, np.float64)
    dlp = np.zeros_like(lp)
    dev = np.zeros_like(ev)
    for arr, out in ((lp, dlp), (ev, dev)):
        for i in range(arr.size):
            old = arr[i]
            arr[i] = old + h
            up = oracle.loss(graph, lp, ev, T, damping, n_iters, g)
            arr[i] = old - h
            dn = oracle.loss(graph, lp, ev, T, damping, n_iters, g)
            arr[i] = old
            out[i] = (up - dn) / (2 * h)
    return dlp, dev


def _cases():
    out = []
    p = W.ising_grid(4, 5, 3, T=1.0)
    out.append(("ising4x5", p.graph, p.log_pot, p.evidence))
    for seed in (1, 2):
        g, lp, ev = W.random_graph(seed, n_vars=7, max_K=3, n_pair=6, n_triple=2, n_or=0, n_and=0,
                                   sparse=False, shared=(seed == 2))
        out.append((f"random{seed}", g, lp, ev))
    p = W.potts_grid(3, 3, 4, T=1.0)
    out.append(("potts3x3K3", p.graph, p.log_pot, p.evidence))
    # logical OR / AND factors (fan-in 1..4) among pairwise and triple factors (seeds
    # whose runs have no structural zero: a -inf belief makes the loss undefined)
    for seed in (4, 5, 9):
        g, lp, ev = W.random_graph(seed, n_vars=8, max_K=2, n_pair=5, n_triple=1, n_or=2, n_and=2)
        out.append((f"logic{seed}", g, lp, ev))
    # XOR (parity) factors with OR / AND
    for seed in (4, 5):
        g, lp, ev = W.random_graph(seed, n_vars=8, max_K=2, n_pair=5, n_triple=1, n_or=1, n_and=1, n_xor=2)
        out.append((f"xor{seed}", g, lp, ev))
    return out


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
@pytest.mark.parametrize("T,damping,n_iters", [(1.0, 0.5, 12), (0.7, 0.0, 6), (1.0, 0.3, 20)])
def test_grad_matches_finite_differences(case, T, damping, n_iters):
    name, graph, lp, ev = case
    rng = np.random.default_rng(7)
    g = rng.standard_normal(graph.n_var_states)
    dlp, dev = oracle.grad(graph, lp, ev, T, damping, n_iters, g)
    flp, fev = _fd(graph, lp, ev, T, damping, n_iters, g)
    np.testing.assert_allclose(dlp, flp, atol=2e-7, rtol=1e-5)
    np.testing.assert_allclose(dev, fev, atol=2e-7, rtol=1e-5)


@pytest.mark.parametrize("case", _cases(), ids=lambda c: c[0])
def test_grad_shift_invariances(case):
    name, graph, lp, ev = case
    rng = np.random.default_rng(3)
    g = rng.standard_normal(graph.n_var_states)
    dlp, dev = oracle.grad(graph, lp, ev, 1.0, 0.5, 15, g)
    vs = np.concatenate([[0], np.cumsum(graph.num_states)])
    for v in range(graph.n_vars):
        assert abs(dev[vs[v]:vs[v + 1]].sum()) < 1e-10
    off = 0
    for grp in graph.enum_groups:
        if grp.shared:
            assert abs(dlp[off:off + grp.n_cfg].sum()) < 1e-10
        else:
            blk = dlp[off:off + grp.n_potentials].reshape(grp.n_fac, grp.n_cfg)
            assert np.abs(blk.sum(1)).max() < 1e-10
        off += grp.n_potentials


def test_grad_rejects_wide_logical_and_max_product():
    """The oracle's logical adjoint enumerates parent configurations: fan-in above 20
    (the deconvolution's OR factors reach 180) is refused, as is max-product."""
    p = W.deconvolution(1, n_img=1, n_iters=3)
    with pytest.raises(ValueError):
        oracle.grad(p.graph, p.log_pot, p.evidence, 1.0, 0.5, 3, np.zeros(p.graph.n_var_states))
    q = W.ising_grid(3, 3, 1)
    with pytest.raises(ValueError):
        oracle.grad(q.graph, q.log_pot, q.evidence, 0.0, 0.5, 3, np.zeros(q.graph.n_var_states))
