"""Variables with more than 64 factors (the block-per-variable and tile-split variable
passes): a factor forms such an edge's exact leave-one-out value from the variable's
per-state totals -- the float-float sum of the finite evidence and incoming entries and
the count of -inf ones -- and the edge's own entry. These stars put hard zeros (-inf
table entries and evidence) next to the hub, so that hub states carry -inf entries on
some edges: an edge whose own entry is the only -inf one must see the finite sum of the
others, every other edge -inf. Held to the FP64 oracle at 1e-4, and the multi-sample
launch (block per variable) to the single-sample one (tile split) bitwise.
"""
import numpy as np
import pytest

import oracle
from paper_2202_04110_gb300 import workloads as W
from tests._parity import assert_beliefs_close, assert_decode_ok

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


def _star(n_leaves, K, seed, p_zero, hub_zero=False, leaf_zero=0.0, one_zero=False):
    """Hub variable 0 (K states) joined to n_leaves leaves (K states) by pairwise factors
    with their own N(0, 1) tables, a fraction p_zero of table entries -inf (each row keeps
    one finite entry); a fraction leaf_zero of leaves with one state clamped off; with
    hub_zero the hub's state K-1 is clamped off. one_zero: leaf 1 is clamped to state 0 and
    its table forbids (hub 0, leaf 0), so exactly one edge sends the hub -inf on state 0."""
    rng = np.random.default_rng(seed)
    cfg = np.stack(np.meshgrid(np.arange(K), np.arange(K), indexing="ij"), -1).reshape(-1, 2).astype(np.int32)
    pairs = np.stack([np.zeros(n_leaves, np.int32), np.arange(1, n_leaves + 1, dtype=np.int32)], 1)
    lp = rng.normal(0, 1, (n_leaves, K, K))
    zero = rng.random((n_leaves, K, K)) < p_zero
    zero[:, np.arange(K), rng.integers(0, K, K)] = False
    lp[zero] = -np.inf
    ev = rng.normal(0, 1, (n_leaves + 1, K))
    clamp = rng.random(n_leaves) < leaf_zero
    ev[1:][clamp, rng.integers(0, K, clamp.sum())] = -np.inf
    if hub_zero:
        ev[0, K - 1] = -np.inf
    if one_zero:
        ev[1, 1:] = -np.inf
        lp[0, 0, 0] = -np.inf
    g = W.FactorGraph(np.full(n_leaves + 1, K, np.int32), [W.EnumGroup(cfg, pairs, False)], [])
    return g, lp.astype(np.float32).ravel(), ev.astype(np.float32).ravel()


def _run(binding, g, lp, ev, T, n_iters):
    import torch
    G = binding.Graph(g)
    lpt, evt = torch.as_tensor(lp).cuda(), torch.as_tensor(ev).cuda()
    m = G.new_msgs()
    G.run_bp(lpt, evt, T, 0.5, n_iters, m)
    return G, m, G.beliefs(evt, m, True).cpu().numpy(), G.decode(evt, m).cpu().numpy(), G.flags(clear=True)


@pytest.mark.parametrize("n_leaves", [100, 3000])  # one tile of 2048 edges, two tiles
@pytest.mark.parametrize("T", [0.0, 1.0])
@pytest.mark.parametrize("case", ["soft", "one_zero", "hard_tables", "hard_all"])
def test_star_hub_against_oracle(gpu, n_leaves, T, case):
    """soft: no -inf anywhere; one_zero: one -inf entry on one hub state (that edge sees the
    others' finite sum, every other edge -inf); hard_tables / hard_all: hundreds of -inf
    entries, hub states with counts of 2 and more, contradictions that both sides flag."""
    p_zero, hub_zero, leaf_zero = {"soft": (0.0, False, 0.0), "one_zero": (0.0, False, 0.0),
                                   "hard_tables": (0.6, False, 0.6), "hard_all": (0.3, True, 0.2)}[case]
    g, lp, ev = _star(n_leaves, 3, seed=n_leaves + len(case), p_zero=p_zero, hub_zero=hub_zero,
                      leaf_zero=leaf_zero, one_zero=case == "one_zero")
    _, m, nb, dec, flags = _run(gpu, g, lp, ev, T, 6)
    om, ofl = oracle.run_bp(g, lp, ev, T, 0.5, 6)
    _, onb, _, ofl2 = oracle.beliefs(g, ev, om)
    mg = m.cpu().numpy()
    om = np.asarray(om)
    assert (np.isneginf(mg) == np.isneginf(om)).all(), "-inf pattern of the messages"
    fin = np.isfinite(om)  # the messages themselves (a clamped leaf's belief hides its message)
    err = np.abs(mg[fin] - om[fin])
    assert (err <= 1e-4 + 2.0 ** -22 * np.abs(om[fin])).all(), f"messages differ by {err.max():.3e}"
    assert_beliefs_close(nb, onb, what=f"star {n_leaves} T={T} {case}")
    assert_decode_ok(dec, onb, g.num_states, what=f"star {n_leaves} T={T} {case}")
    assert bool(flags & 1) == bool((ofl | ofl2) & 1)


@pytest.mark.parametrize("T", [0.0, 1.0])
def test_star_multi_sample_equals_single(gpu, T):
    """The multi-sample launch runs the block-per-variable kernel, the single-sample run the
    tile split: the same totals in the same order, so the same bits."""
    import torch
    g, lp, ev = _star(3000, 3, seed=5, p_zero=0.3, hub_zero=False, leaf_zero=0.1)
    G = gpu.Graph(g)
    S = 3
    rng = np.random.default_rng(1)
    evs = np.stack([ev + rng.normal(0, 0.3, ev.size).astype(np.float32) for _ in range(S)])
    lpt = torch.as_tensor(lp).cuda()
    m = torch.zeros(S, G.info["n_edge_states"], device="cuda")
    G.run_bp_multi(lpt, torch.as_tensor(evs).cuda(), T, 0.5, 7, m)
    for s in range(S):
        ms = G.new_msgs()
        G.run_bp(lpt, torch.as_tensor(evs[s]).cuda(), T, 0.5, 7, ms)
        assert torch.equal(ms, m[s]), s


@pytest.mark.parametrize("n_leaves", [64, 65, 2048, 2049, 4097])
def test_star_degree_boundaries(gpu, n_leaves):
    """Hub degrees at the boundaries: 64 (thread per variable) and 65 (high-degree
    pass), one tile of 2048 edges exactly, one edge into a second tile, and three tiles
    with a one-edge tail; binary and 3-state hubs, T = 0 and 1."""
    for K in (2, 3):
        g, lp, ev = _star(n_leaves, K, seed=n_leaves + K, p_zero=0.2, leaf_zero=0.1)
        for T in (0.0, 1.0):
            _, m, nb, dec, flags = _run(gpu, g, lp, ev, T, 5)
            om, ofl = oracle.run_bp(g, lp, ev, T, 0.5, 5)
            _, onb, _, ofl2 = oracle.beliefs(g, ev, om)
            assert_beliefs_close(nb, onb, what=f"star {n_leaves} K={K} T={T}")
            assert_decode_ok(dec, onb, g.num_states, what=f"star {n_leaves} K={K} T={T}")
            assert bool(flags & 1) == bool((ofl | ofl2) & 1)
