"""Pins for the FP64 oracle against facts the mathematics fixes (CPU only).

* LBP is exact on trees (Pearl 1988): with damping 0 and as many iterations as the tree
  has variables, normalised beliefs equal the exact log-marginals (sum-product, T=1)
  and the max-marginals (max-product, T=0), computed here by enumerating the joint.
* One flooding iteration on loopy graphs equals the dense-tensor definition with raw
  (unnormalised) messages and raw damping: the normalised beliefs are invariant to the
  per-edge constants that normalisation removes.
* The closed-form OR / AND updates (linear in the fan-in, Sec. 3) equal brute-force
  enumeration over all parent configurations, for T in {0, 0.5, 1}.
* Special cases: one parent copies the child's log-odds and vice versa; no parents
  forces the child to 0 (OR) or 1 (AND); a 2-variable Ising pair has a closed form.
* Large sparse configuration lists (40-state chain, pairs within 3 listed): the
  beliefs equal the forward-backward (max-)marginals of the chain.
* MAP decode on random 30-unit RBMs (the protocol of Sec. 5.1) never beats the
  brute-force MAP and is checked against it.
"""
import numpy as np
import pytest

import oracle
from paper_2202_04110_gb300 import workloads as W
from tests import _brute as B


def _tree_cases():
    cases = []
    for seed in range(12):
        cases.append(dict(seed=seed, logical=True, shared=(seed % 3 == 0), xor=False))
    seed = 300
    while sum(c["xor"] for c in cases) < 6:  # trees that also hold XOR (parity) factors
        g, _, _ = W.random_factor_tree(seed, n_vars=9, logical=True, xor=True)
        if any(lg.kind == W.XOR for lg in g.logic_groups):
            cases.append(dict(seed=seed, logical=True, shared=(seed % 2 == 0), xor=True))
        seed += 1
    return cases


@pytest.mark.parametrize("case", _tree_cases(), ids=lambda c: f"tree{c['seed']}")
@pytest.mark.parametrize("T", [1.0, 0.0])
def test_tree_exact(case, T):
    g, lp, ev = W.random_factor_tree(case["seed"], n_vars=9, shared=case["shared"],
                                     logical=case["logical"], xor=case["xor"])
    if case["xor"]:
        assert any(lg.kind == W.XOR for lg in g.logic_groups), "the tree should hold an XOR factor"
    msgs, fl = oracle.run_bp(g, lp, ev, T, 0.0, g.n_vars + 1)
    _, nb, dec, fl2 = oracle.beliefs(g, ev, msgs)
    assert fl == 0 and fl2 == 0
    exact = B.exact_log_marginals(g, lp, ev, T)
    if T == 1.0:
        np.testing.assert_allclose(nb, exact, atol=1e-10)
    else:
        # max-marginals are defined up to one constant per variable
        ks = g.num_states
        vs = np.concatenate([[0], np.cumsum(ks)])
        for v in range(g.n_vars):
            a = nb[vs[v]:vs[v + 1]]
            b = exact[vs[v]:vs[v + 1]]
            np.testing.assert_allclose(a - a.max(), b - b.max(), atol=1e-10)
        # MAP: the decode of max-product on a tree maximises the joint when unique
        x_map, best = B.brute_map(g, lp, ev)
        J = B.joint_scores(g, lp, ev)
        assert np.isclose(J[tuple(dec)], best, atol=1e-9)


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("T", [1.0, 0.0])
def test_tree_exact_with_damping(seed, T):
    """Damping changes the path, not the fixed point: 300 damped iterations on a tree
    also give the exact marginals."""
    g, lp, ev = W.random_factor_tree(100 + seed, n_vars=8)
    msgs, _ = oracle.run_bp(g, lp, ev, T, 0.5, 300)
    _, nb, _, _ = oracle.beliefs(g, ev, msgs)
    exact = B.exact_log_marginals(g, lp, ev, T)
    vs = np.concatenate([[0], np.cumsum(g.num_states)])
    for v in range(g.n_vars):
        a, b = nb[vs[v]:vs[v + 1]], exact[vs[v]:vs[v + 1]]
        np.testing.assert_allclose(a - a.max(), b - b.max(), atol=1e-8)


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("T", [1.0, 0.0, 0.5])
@pytest.mark.parametrize("damping", [0.0, 0.5])
def test_loopy_matches_dense_definition(seed, T, damping):
    g, lp, ev = W.random_graph(seed, n_vars=9, max_K=3, n_pair=8, n_triple=2, n_or=2, n_and=2,
                               sparse=True, shared=(seed % 2 == 1), n_xor=(2 if seed >= 4 else 0))
    n_it = 7
    msgs, fl = oracle.run_bp(g, lp, ev, T, damping, n_it)
    _, nb, _, _ = oracle.beliefs(g, ev, msgs)
    ref, _ = B.dense_lbp(g, lp, ev, T, damping, n_it)
    assert fl == 0
    np.testing.assert_allclose(nb, ref, atol=1e-9)


@pytest.mark.parametrize("seed", range(4))
def test_warm_start_composes(seed):
    """Messages are the explicit state: a runs then b runs equals a+b runs."""
    g, lp, ev = W.random_graph(seed, n_vars=8)
    m1, _ = oracle.run_bp(g, lp, ev, 1.0, 0.5, 5)
    m2, _ = oracle.run_bp(g, lp, ev, 1.0, 0.5, 6, msgs=m1)
    m3, _ = oracle.run_bp(g, lp, ev, 1.0, 0.5, 11)
    np.testing.assert_array_equal(m2, m3)


@pytest.mark.parametrize("kind", [W.OR, W.AND, W.XOR])
@pytest.mark.parametrize("T", [0.0, 0.5, 1.0])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 8, 11])
def test_logical_closed_form_vs_enumeration(kind, T, n):
    rng = np.random.default_rng(1000 * n + 10 * kind + int(4 * T))
    for trial in range(6):
        scale = [0.3, 1.0, 4.0, 12.0, 1.0, 1.0][trial]
        v2f = rng.normal(0, scale, size=(n + 1, 2))
        if trial == 4:  # strongly negative parents: small A_{-i}
            v2f[:-1, 1] = v2f[:-1, 0] - rng.uniform(8, 15, n)
        if trial == 5:  # decisive child
            v2f[-1] = [0.0, 9.0]
        closed = oracle.logic_update(kind, v2f, T, brute=False)
        ref = B.logic_dense(kind, v2f, T)
        np.testing.assert_allclose(closed, ref, atol=1e-9, rtol=1e-9)
        brute = oracle.logic_update(kind, v2f, T, brute=True)
        np.testing.assert_allclose(brute, ref, atol=1e-9, rtol=1e-9)


@pytest.mark.parametrize("T", [0.0, 0.5, 1.0])
def test_xor_special_cases(T):
    # one parent: XOR(p) = p, so each side receives the other's log-odds
    v2f = np.array([[0.0, 1.3], [0.2, -0.5]])
    out = oracle.logic_update(W.XOR, v2f, T)
    assert np.isclose(out[0, 1] - out[0, 0], -0.7)
    assert np.isclose(out[1, 1] - out[1, 0], 1.3)
    # no parents: XOR of nothing is 0
    out = oracle.logic_update(W.XOR, np.array([[0.4, -0.1]]), T)
    assert out[0, 0] == 0.0 and out[0, 1] == -np.inf
    # a parent with even odds (log-odds 0) makes every other member's message flat
    v2f = np.array([[0.3, 0.3], [0.0, 2.0], [1.0, -1.5]])
    out = oracle.logic_update(W.XOR, v2f, T)
    assert np.allclose(out[1], 0.0) and np.allclose(out[2], 0.0)
    # all others certain: the member receives their parity with certainty
    v2f = np.array([[-np.inf, 0.0], [-np.inf, 0.0], [0.1, 0.2]])  # parents 1, 1 -> child 0
    out = oracle.logic_update(W.XOR, v2f, T)
    assert out[2, 0] == 0.0 and out[2, 1] == -np.inf
    ref = B.logic_dense(W.XOR, v2f, T)
    np.testing.assert_allclose(out, ref, atol=1e-12)
    # the two-member parity (child = one parent) at T = 1 is the pairwise equality factor
    if T == 1.0:
        x = 0.8
        v2f = np.array([[0.0, x], [0.0, 0.0]])
        out = oracle.logic_update(W.XOR, v2f, T)
        assert np.isclose(out[1, 1] - out[1, 0], x)
    # three members at T = 1: the parity check's product rule tanh(out/2) = -prod tanh(-x/2)
    if T == 1.0:
        x1, x2 = 0.9, -1.7
        v2f = np.array([[0.0, x1], [0.0, x2], [0.0, 0.0]])
        out = oracle.logic_update(W.XOR, v2f, T)
        d = np.tanh(-x1 / 2) * np.tanh(-x2 / 2)
        assert np.isclose(out[2, 1] - out[2, 0], np.log((1 - d) / (1 + d)))


@pytest.mark.parametrize("T", [0.0, 1.0])
def test_logical_special_cases(T):
    # one parent: OR(p) = p, so each side receives the other's log-odds
    v2f = np.array([[0.0, 1.3], [0.2, -0.5]])  # parent x=1.3, child x=-0.7
    out = oracle.logic_update(W.OR, v2f, T)
    assert np.isclose(out[0, 1] - out[0, 0], -0.7)
    assert np.isclose(out[1, 1] - out[1, 0], 1.3)
    # no parents: OR of nothing is 0, AND of nothing is 1
    out = oracle.logic_update(W.OR, np.array([[0.4, -0.1]]), T)
    assert out[0, 0] == 0.0 and out[0, 1] == -np.inf
    out = oracle.logic_update(W.AND, np.array([[0.4, -0.1]]), T)
    assert out[0, 0] == -np.inf and out[0, 1] == 0.0
    # child certainly on (evidence +inf): the only possibly-on parent must be on
    v2f = np.array([[0.0, -2.0], [0.0, -np.inf], [-np.inf, 0.0]])
    out = oracle.logic_update(W.OR, v2f, T)
    ref = B.logic_dense(W.OR, v2f, T)
    np.testing.assert_allclose(out, ref, atol=1e-12)
    # a parent certainly on: the others receive a flat message
    v2f = np.array([[-np.inf, 0.0], [0.0, 0.7], [0.1, 0.3]])
    out = oracle.logic_update(W.OR, v2f, T)
    ref = B.logic_dense(W.OR, v2f, T)
    np.testing.assert_allclose(out, ref, atol=1e-12)
    assert np.allclose(out[1], 0.0)


def test_ising_pair_closed_form():
    """Two spins: p(s1, s2) ~ exp(J s1 s2 + h1 s1 + h2 s2). P(s1 = +1) in closed form."""
    J, h1, h2 = 0.7, -0.3, 1.1
    g = W.FactorGraph(np.array([2, 2], np.int32),
                      [W.EnumGroup(W.PAIR2_CFG.copy(), np.array([[0, 1]], np.int32))], [])
    lp = np.array([J, -J, -J, J])
    ev = np.array([-h1, h1, -h2, h2])
    for T in (1.0, 0.0):
        msgs, _ = oracle.run_bp(g, lp, ev, T, 0.0, 3)
        _, nb, dec, _ = oracle.beliefs(g, ev, msgs)
        w = {(a, b): np.exp(J * a * b + h1 * a + h2 * b) for a in (-1, 1) for b in (-1, 1)}
        if T == 1.0:
            p1 = (w[(1, 1)] + w[(1, -1)]) / sum(w.values())
            assert np.isclose(np.exp(nb[1]), p1, atol=1e-12)
        else:
            best = max(w, key=w.get)
            assert tuple(2 * dec - 1) == best


def test_sizes_of_workloads():
    p = W.ising_small(0)
    s = oracle.sizes(p.graph)
    assert s == dict(V=100, VS=200, E=360, ES=720, P=720)
    big = W.ising_grid(1000, 1000, 0, n_iters=1)
    assert big.graph.n_factors == 1_998_000
    assert big.graph.n_edge_states == 7_992_000
    d = W.deconvolution(0, n_iters=1)
    assert d.graph.n_vars == 180 + 50_000 + 1_800_000 + 22_500
    assert d.graph.n_edges == 7_222_500
    assert d.graph.n_edge_states == 14_445_000
    fan = np.diff(d.graph.logic_groups[1].par_off)
    assert fan.min() == 5 and fan.max() == 180
    s = oracle.sizes(d.graph)
    assert s["ES"] == 14_445_000


def test_rbm_map_protocol():
    """Sec. 5.1 protocol: 20 random 30-unit RBMs (15 visible + 15 hidden), 200
    max-product iterations with damping 0.5, MAP quality = log-potential of the decoded
    configuration, ground truth by enumeration. The decode can never beat the brute-force
    MAP; how often it recovers it depends on the RBM distribution, which the paper does
    not state (so the recovery count is reported, not pinned)."""
    recovered = 0
    for s in range(20):
        p = W.rbm(15, 15, seed=500 + s, w_std=1.0, T=0.0, damping=0.5, n_iters=200)
        _, dec, _, _ = oracle.infer(p)
        nv, nh = 15, 15
        Wm = p.log_pot.reshape(nv, nh, 4)[:, :, 3].astype(np.float64)
        b = p.evidence.reshape(-1, 2)[:, 1].astype(np.float64)
        vis = ((np.arange(2 ** nv)[:, None] >> np.arange(nv)) & 1).astype(np.float64)
        act = b[nv:] + vis @ Wm
        best_per_v = vis @ b[:nv] + np.maximum(act, 0).sum(1)
        best = best_per_v.max()
        v, h = dec[:nv].astype(np.float64), dec[nv:].astype(np.float64)
        got = v @ b[:nv] + h @ b[nv:] + v @ Wm @ h
        assert got <= best + 1e-9
        recovered += bool(np.isclose(got, best, atol=1e-9))
    assert recovered >= 10


def _chain_forward_backward(K, cfg, phis, ev, T):
    """Exact (max-)marginals of a chain x_0 - x_1 - ... by the forward-backward
    recursions (Rabiner 1989), in log space: phis[i] is the [K, K] table of the factor
    between x_i and x_{i+1} (-inf where a configuration is not listed), ev[i] the
    evidence of x_i. LSE for T = 1, max for T = 0. Returns unnormalised [n, K] scores."""
    def red(z, axis):
        if T == 0.0:
            return z.max(axis=axis)
        return B.lse(z, axis=axis)
    n = len(ev)
    alpha = [ev[0]]
    for i in range(n - 1):
        alpha.append(ev[i + 1] + red(alpha[i][:, None] + phis[i], 0))
    beta = [np.zeros(K)] * n
    for i in range(n - 2, -1, -1):
        beta[i] = red(phis[i] + (ev[i + 1] + beta[i + 1])[None, :], 1)
    return np.stack([alpha[i] + beta[i] for i in range(n)])


@pytest.mark.parametrize("T", [1.0, 0.0])
@pytest.mark.parametrize("shared", [True, False])
def test_large_sparse_factor_chain_exact(T, shared):
    """A chain of 40-state variables whose pairwise factors list only the pairs within 3
    of each other (a large, sparse configuration list, as in Sec. 5.2): LBP is exact on
    the chain, so the oracle's beliefs equal the forward-backward (max-)marginals."""
    K, n = 40, 7
    rng = np.random.default_rng(5)
    a, b = np.nonzero(np.abs(np.arange(K)[:, None] - np.arange(K)[None, :]) <= 3)
    cfg = np.stack([a, b], axis=1).astype(np.int32)
    pairs = np.stack([np.arange(n - 1), np.arange(1, n)], axis=1).astype(np.int32)
    n_pot = cfg.shape[0] * (1 if shared else n - 1)
    lp = rng.standard_normal(n_pot)
    ev = rng.standard_normal((n, K))
    g = W.FactorGraph(np.full(n, K, np.int32), [W.EnumGroup(cfg, pairs, shared)], [])
    phis = []
    for i in range(n - 1):
        t = np.full((K, K), -np.inf)
        t[cfg[:, 0], cfg[:, 1]] = lp if shared else lp[i * cfg.shape[0]:(i + 1) * cfg.shape[0]]
        phis.append(t)
    exact = _chain_forward_backward(K, cfg, phis, ev, T)
    msgs, fl = oracle.run_bp(g, lp, ev.ravel(), T, 0.0, n + 1)
    _, nb, dec, fl2 = oracle.beliefs(g, ev.ravel(), msgs)
    assert fl == 0 and fl2 == 0
    nb = nb.reshape(n, K)
    for v in range(n):  # defined up to one constant per variable
        np.testing.assert_allclose(nb[v] - nb[v].max(), exact[v] - exact[v].max(), atol=1e-10)
    if T == 0.0:
        np.testing.assert_array_equal(dec, exact.argmax(axis=1))
