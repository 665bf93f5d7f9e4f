"""Seeded random graphs that mix every kind of group the compiler knows -- dense pairwise
tables of mixed state counts, listed triple factors, OR / AND / XOR factors of fan-in
1..6 and one wide enough for the warp kernel, a hub with more than 64 factors, hard
evidence -- against the FP64 oracle (short horizon, strict 1e-4), and in one batch
against the same graphs run alone (bitwise).
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


def mixed_graph(seed: int):
    """80 variables (K in {2, 3, 5}), pairwise groups per state-count signature (dense
    tables, shared or per factor), one listed triple group, a binary hub joined to 70
    binary variables, logical groups over the binary variables, hard evidence on a tenth
    of the variables (multi-state ones)."""
    rng = np.random.default_rng(seed)
    n = 80
    K = rng.choice([2, 2, 3, 5], size=n).astype(np.int32)
    K[0] = 2
    binary = np.flatnonzero(K == 2)
    enum, pots = [], []
    # pairwise groups by signature
    by_sig = {}
    for _ in range(110):
        a, b = rng.choice(n, 2, replace=False)
        by_sig.setdefault((int(K[a]), int(K[b])), []).append((a, b))
    for (ka, kb), pairs in sorted(by_sig.items()):
        cfg = np.stack(np.meshgrid(np.arange(ka), np.arange(kb), indexing="ij"), -1).reshape(-1, 2).astype(np.int32)
        shared = bool(rng.random() < 0.4)
        enum.append(W.EnumGroup(cfg, np.asarray(pairs, np.int32), shared))
        pots.append(rng.normal(0, 1, cfg.shape[0] * (1 if shared else len(pairs))))
    # a listed triple group over one signature
    trip = rng.choice(n, 3, replace=False)
    sig = K[trip]
    full = np.stack(np.meshgrid(*[np.arange(k) for k in sig], indexing="ij"), -1).reshape(-1, 3)
    keep = rng.random(full.shape[0]) < 0.6
    keep[0] = True
    cfg = full[keep].astype(np.int32)
    triples = [trip]
    for _ in range(5):
        pick = [int(rng.choice(np.flatnonzero(K == k))) for k in sig]
        if len(set(pick)) == 3:
            triples.append(np.asarray(pick))
    enum.append(W.EnumGroup(cfg, np.asarray(triples, np.int32), False))
    pots.append(rng.normal(0, 1, cfg.shape[0] * len(triples)))
    # the hub: binary variable 0 with 70 binary neighbours (a block-per-tile variable pass)
    others = [v for v in binary if v != 0]
    nb = rng.choice(others, size=70, replace=True)  # (repeated pairs are separate factors)
    hub_pairs = np.stack([np.zeros(nb.size, np.int64), nb], 1).astype(np.int32)
    cfg2 = np.array([[0, 0], [0, 1], [1, 0], [1, 1]], np.int32)
    enum.append(W.EnumGroup(cfg2, hub_pairs, False))
    pots.append(rng.normal(0, 0.7, 4 * nb.size))
    # logical groups
    logic = []
    for kind in (W.OR, W.AND, W.XOR):
        offs, pars, ch = [0], [], []
        # fan-in 1..6 (a factor of no parents forces its child, and two such factors of
        # different kinds on one child are the undefined case above; tested elsewhere)
        fans = list(rng.integers(1, 7, size=4)) + ([40] if kind == W.OR else [])
        for fan in fans:
            sel = rng.choice(binary[1:], size=min(int(fan) + 1, binary.size - 1), replace=False)
            pars.extend(int(x) for x in sel[:-1])
            ch.append(int(sel[-1]))
            offs.append(len(pars))
        logic.append(W.LogicGroup(kind, np.asarray(offs, np.int32), np.asarray(pars, np.int32),
                                  np.asarray(ch, np.int32)))
    g = W.FactorGraph(K, enum, logic)
    ev = rng.normal(0, 1, int(K.sum()))
    off = np.concatenate([[0], np.cumsum(K)])
    # hard evidence (one state off) on a tenth of the variables, the multi-state ones: the
    # logical factors then see finite log-odds (two certain inputs of opposite sense would
    # make an OR update inf - inf, a case the method leaves undefined)
    multi = np.flatnonzero(K > 2)
    for v in rng.choice(multi, min(n // 10, multi.size), replace=False):
        ev[off[v] + rng.integers(0, K[v])] = -np.inf
    return g, np.concatenate(pots).astype(np.float32), ev.astype(np.float32)


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("T", [0.0, 0.7, 1.0])
def test_mixed_graph_against_oracle(gpu, seed, T):
    import torch
    g, lp, ev = mixed_graph(seed)
    G = gpu.Graph(g)
    lpt, evt = torch.as_tensor(lp).cuda(), torch.as_tensor(ev).cuda()
    m = G.new_msgs()
    G.run_bp(lpt, evt, T, 0.5, 3, m)
    nb = G.beliefs(evt, m, True).cpu().numpy()
    dec = G.decode(evt, m).cpu().numpy()
    flags = G.flags(clear=True)
    om, ofl = oracle.run_bp(g, lp, ev, T, 0.5, 3)
    _, onb, _, ofl2 = oracle.beliefs(g, ev, om)
    mg, om = m.cpu().numpy(), np.asarray(om)
    assert (np.isneginf(mg) == np.isneginf(om)).all(), "-inf pattern of the messages"
    assert_beliefs_close(nb, onb, what=f"mixed seed={seed} T={T}")
    assert_decode_ok(dec, onb, g.num_states, what=f"mixed seed={seed} T={T}")
    assert bool(flags & 1) == bool((ofl | ofl2) & 1)


def test_mixed_graphs_batched_equal_alone(gpu):
    """Six mixed graphs as one batch: each member's messages equal the graph run alone."""
    import torch
    graphs = [mixed_graph(100 + i) for i in range(6)]
    gb = gpu.Graph([g for g, _, _ in graphs])
    lp = torch.as_tensor(np.concatenate([x for _, x, _ in graphs])).cuda()
    ev = torch.as_tensor(np.concatenate([x for _, _, x in graphs])).cuda()
    for T in (0.0, 1.0):
        mb = gb.new_msgs()
        gb.run_bp(lp, ev, T, 0.5, 5, mb)
        for i, (g, lpi, evi) in enumerate(graphs):
            off = gb.member(i)
            G = gpu.Graph(g)
            m1 = G.new_msgs()
            G.run_bp(torch.as_tensor(lpi).cuda(), torch.as_tensor(evi).cuda(), T, 0.5, 5, m1)
            seg = mb[off["es_off"]: off["es_off"] + off["n_edge_states"]]
            assert torch.equal(seg, m1), (T, i)
