"""GPU parity of the XOR (parity) logical factor against the FP64 oracle.

The XOR factor is the third kind of logical factor (Sec. 3 counts three kinds with
linear-time updates and names none; OR, AND and XOR are the three built). Its closed
form is the product rule of parity checks at T > 0 and the min-sum rule at T = 0
(oracle: xor_update); the oracle's closed form is pinned by enumeration on the CPU
(test_oracle_pins.py). Here the CUDA path -- the thread-per-factor kernel for fan-in up
to 4 and the warp-scan kernel above -- is held to the oracle at 1e-4 on random loopy
graphs, trees (where BP is exact), wide factors that span several 32-parent rounds,
hard evidence and contradictions, and the many-evidence launch.
"""
import numpy as np
import pytest

import oracle
from paper_2202_04110_gb300 import workloads as W
from tests._parity import assert_beliefs_close, assert_decode_ok, assert_within_envelope, oracle_envelope

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


def _infer(binding, graph, log_pot, evidence, T, damping, n_iters):
    import torch
    g = binding.Graph(graph)
    lp = torch.as_tensor(np.asarray(log_pot, np.float32)).cuda()
    ev = torch.as_tensor(np.asarray(evidence, np.float32)).cuda()
    m = g.new_msgs()
    g.run_bp(lp, ev, T, damping, n_iters, m)
    nb = g.beliefs(ev, m, True).cpu().numpy()
    dec = g.decode(ev, m).cpu().numpy()
    return g, m, nb, dec, g.flags(clear=True)


def _check(binding, graph, log_pot, evidence, T, damping, n_iters, what):
    _, m, nb, dec, flags = _infer(binding, graph, log_pot, evidence, T, damping, n_iters)
    om, ofl = oracle.run_bp(graph, log_pot, evidence, T, damping, n_iters)
    _, onb, _, ofl2 = oracle.beliefs(graph, evidence, om)
    assert_beliefs_close(nb, onb, what=what)
    assert_decode_ok(dec, onb, graph.num_states, what=what)
    assert bool(flags & 1) == bool((ofl | ofl2) & 1), (what, flags, ofl, ofl2)
    return m, om


def _xor_graph(fanins, seed, n_extra=0):
    """One XOR group, factor f with fanins[f] parents; parents and children are distinct
    fresh binary variables, plus n_extra pairwise factors tying random variables together
    (loops). Evidence mixes weak (N(0, 1)) and strong (N(+-4, 1)) log-odds."""
    rng = np.random.default_rng(seed)
    offs, pars, ch = [0], [], []
    v = 0
    for n in fanins:
        pars.extend(range(v, v + n))
        ch.append(v + n)
        v += n + 1
        offs.append(len(pars))
    n_var = v
    enum = []
    pots = []
    if n_extra:
        pairs = np.stack([rng.choice(n_var, 2, replace=False) for _ in range(n_extra)]).astype(np.int32)
        cfg = np.array([[0, 0], [0, 1], [1, 0], [1, 1]], np.int32)
        enum.append(W.EnumGroup(cfg, pairs, False))
        pots.append(rng.normal(0, 1, 4 * n_extra))
    fg = W.FactorGraph(np.full(n_var, 2, np.int32), enum,
                       [W.LogicGroup(W.XOR, np.asarray(offs, np.int32), np.asarray(pars, np.int32),
                                     np.asarray(ch, np.int32))])
    h = np.where(rng.random(n_var) < 0.5, rng.normal(0, 1, n_var), rng.normal(0, 1, n_var) + rng.choice([-4, 4], n_var))
    ev = np.stack([np.zeros(n_var), h], 1).ravel().astype(np.float32)
    lp = (np.concatenate(pots) if pots else np.zeros(0)).astype(np.float32)
    return fg, lp, ev


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("T", [0.0, 0.5, 1.0])
def test_random_loopy_with_xor_strict(gpu, seed, T):
    """Random loopy graphs with XOR next to OR / AND and enumeration factors, 4 iterations."""
    g, lp, ev = W.random_graph(seed, n_vars=40, max_K=4, n_pair=70, n_triple=6, n_or=3, n_and=3, n_xor=6,
                               sparse=True, shared=(seed % 2 == 1))
    assert any(lg.kind == W.XOR for lg in g.logic_groups)
    _check(gpu, g, lp, ev, T, 0.5, 4, f"random+xor seed={seed} T={T}")


@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("T", [0.0, 1.0])
def test_random_loopy_with_xor_envelope(gpu, seed, T):
    g, lp, ev = W.random_graph(seed, n_vars=40, max_K=4, n_pair=70, n_triple=6, n_or=3, n_and=3, n_xor=6,
                               sparse=True, shared=(seed % 2 == 1))
    _, _, nb, dec, _ = _infer(gpu, g, lp, ev, T, 0.5, 12)
    nb0, _, spread, unstable, _ = oracle_envelope(oracle, g, lp, ev, T, 0.5, 12, k=2)
    assert_within_envelope(nb, dec, nb0, spread, unstable, g.num_states, what=f"random+xor envelope seed={seed}")


def _xor_trees(count):
    out, seed = [], 300
    while len(out) < count:
        g, lp, ev = W.random_factor_tree(seed, n_vars=60, max_K=4, shared=(seed % 2 == 0), xor=True)
        if any(lg.kind == W.XOR and lg.n_fac > 0 for lg in g.logic_groups):
            out.append((seed, g, lp, ev))
        seed += 1
    return out


@pytest.mark.parametrize("T", [0.0, 1.0])
def test_xor_trees(gpu, T):
    """Trees with XOR factors: undamped BP converges to the exact marginals (max-marginals)
    within the diameter, so 61 iterations are a fixed point on both sides."""
    for seed, g, lp, ev in _xor_trees(4):
        _check(gpu, g, lp, ev, T, 0.0, 61, f"xor tree seed={seed} T={T}")


@pytest.mark.parametrize("T", [0.0, 0.5, 1.0])
def test_xor_fanin_paths(gpu, T):
    """Fan-in 0..4 (thread per factor) in one group and 5..70 (warp scans, up to three
    32-parent rounds) in another, on a loopy graph: both kernels against the oracle."""
    fg, lp, ev = _xor_graph([0, 1, 2, 3, 4, 4, 3, 2, 1, 0] * 30, seed=1, n_extra=150)
    _check(gpu, fg, lp, ev, T, 0.5, 6, f"xor fan-in <= 4, T={T}")
    fg, lp, ev = _xor_graph([5, 31, 32, 33, 64, 65, 70, 6, 17] * 8, seed=2, n_extra=100)
    _check(gpu, fg, lp, ev, T, 0.5, 6, f"xor fan-in 5..70, T={T}")


@pytest.mark.parametrize("T", [0.0, 1.0])
def test_wide_xor_factor(gpu, T):
    """A single XOR factor with 1000 parents (32 rounds of the warp scans)."""
    fg, lp, ev = _xor_graph([1000], seed=3)
    _check(gpu, fg, lp, ev, T, 0.5, 5, f"wide xor T={T}")


@pytest.mark.parametrize("T", [0.0, 1.0])
def test_xor_hard_evidence_and_contradiction(gpu, T):
    """Clamped parents (one state at -inf) fix the parity the child must take: the GPU
    decodes it and matches the oracle; clamping the child against it is a contradiction
    that both sides flag."""
    for fan in (3, 9):  # thread path, warp path
        fg, lp, ev = _xor_graph([fan], seed=4 + fan)
        e = ev.reshape(-1, 2).copy()
        bits = np.arange(fan) % 2  # parents clamped to 0, 1, 0, ...
        for j, bit in enumerate(bits):
            e[j, 1 - bit] = -np.inf
        _, _, nb, dec, flags = _infer(gpu, fg, lp, e.ravel(), T, 0.5, 4)
        assert dec[fan] == bits.sum() % 2
        _check(gpu, fg, lp, e.ravel(), T, 0.5, 4, f"xor clamped fan={fan}")
        assert flags & gpu.FLAG_CONTRADICTION == 0
        e[fan, bits.sum() % 2] = -np.inf  # child clamped to the wrong parity
        _, _, _, _, flags = _infer(gpu, fg, lp, e.ravel(), T, 0.5, 4)
        om, ofl = oracle.run_bp(fg, lp, e.ravel(), T, 0.5, 4)
        _, _, _, ofl2 = oracle.beliefs(fg, e.ravel(), om)
        assert (ofl | ofl2) & oracle.FLAG_CONTRADICTION
        assert flags & gpu.FLAG_CONTRADICTION


def test_xor_multi_evidence_matches_single_runs(gpu):
    """The many-evidence launch runs the same XOR kernels: bitwise equal to one-by-one runs."""
    import torch
    fg, lp, ev = _xor_graph([2, 3, 7, 40] * 10, seed=6, n_extra=40)
    g = gpu.Graph(fg)
    S = 5
    rng = np.random.default_rng(7)
    evs = np.stack([ev + rng.normal(0, 0.5, ev.size).astype(np.float32) for _ in range(S)])
    lpt = torch.as_tensor(lp).cuda()
    m = torch.zeros(S, g.info["n_edge_states"], device="cuda")
    for T in (0.0, 1.0):
        m.zero_()
        g.run_bp_multi(lpt, torch.as_tensor(evs).cuda(), T, 0.5, 8, m)
        for s in range(S):
            ms = g.new_msgs()
            g.run_bp(lpt, torch.as_tensor(evs[s]).cuda(), T, 0.5, 8, ms)
            assert torch.equal(ms, m[s]), (T, s)


def test_xor_gradient_not_supported(gpu):
    import torch
    fg, lp, ev = _xor_graph([3], seed=8)
    g = gpu.Graph(fg)
    with pytest.raises(gpu.PgmError) as ei:
        g.grad(torch.as_tensor(lp).cuda(), torch.as_tensor(ev).cuda(), 1.0, 0.5, 4, 2,
               torch.zeros(ev.size, device="cuda"))
    assert ei.value.status == -4


def test_xor_empty_and_single_factor_groups(gpu):
    """A group with no factors next to XOR groups of one factor (fan-in 0 and 1): the
    compiler keeps the empty group out of the launches, and the others match the oracle."""
    fg0, lp0, ev0 = _xor_graph([0], seed=21)
    fg1, lp1, ev1 = _xor_graph([1], seed=22)
    groups = [W.LogicGroup(W.XOR, np.array([0], np.int32), np.zeros(0, np.int32), np.zeros(0, np.int32))]
    groups += fg0.logic_groups
    g1 = fg1.logic_groups[0]
    n0 = fg0.num_states.size
    groups.append(W.LogicGroup(W.XOR, g1.par_off, g1.parents + n0, g1.child + n0))
    fg = W.FactorGraph(np.concatenate([fg0.num_states, fg1.num_states]), [], groups)
    ev = np.concatenate([ev0, ev1])
    for T in (0.0, 1.0):
        _check(gpu, fg, np.zeros(0, np.float32), ev, T, 0.5, 3, f"xor small groups T={T}")
