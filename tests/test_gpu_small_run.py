"""The one-launch run of small binary pairwise graphs (PGM_OPT_SMALL_RUN).

One thread block (up to 700 variables), or a cluster of blocks sharing their shared
memories (16 blocks on a GB300: up to 16,384 variables), runs every iteration of the log-ratio scheme (Sec. 3's
parallel damped updates on binary 2 x 2 factors) with the exchanged arrays in shared
memory. Its per-item arithmetic is that of the multi-launch iterations, so its messages are
held bitwise to the multi-launch run with the option off, and its beliefs to the FP64
oracle at the strict bound: on grids from 2 x 2 to the size limits, chains, a grid whose
variables are numbered at random (so that most factors reach into other blocks of the
cluster), hard and contradictory evidence, tables with -inf entries, shared tables, damping
0, warm starts, T = 0 and T > 0, with and without CUDA graphs.
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


def _run(binding, graph, lp, ev, T, damping, n_iters, small, m0=None, cuda_graph=1):
    import torch
    g = binding.Graph(graph)
    g.set_option(binding.OPT_SMALL_RUN, small)
    g.set_option(binding.OPT_CUDA_GRAPH, cuda_graph)
    lpt = torch.as_tensor(np.asarray(lp, np.float32)).cuda()
    evt = torch.as_tensor(np.asarray(ev, np.float32)).cuda()
    m = g.new_msgs() if m0 is None else torch.as_tensor(np.asarray(m0, np.float32)).cuda().clone()
    g.run_bp(lpt, evt, T, damping, n_iters, m)
    g.run_bp(lpt, evt, T, damping, n_iters, m.zero_() if m0 is None else m.copy_(
        torch.as_tensor(np.asarray(m0, np.float32)).cuda()))  # a replay of the recorded run
    nb = g.beliefs(evt, m, True).cpu().numpy()
    dec = g.decode(evt, m).cpu().numpy()
    return g, m.cpu().numpy(), nb, dec, g.flags(clear=True)


def _both(binding, graph, lp, ev, T, damping, n_iters, m0=None, cuda_graph=1, expect_small=True, mode=1):
    """The one-launch run (mode 1: one block or the cluster by size; 2: the cluster) against
    the multi-launch run (0): bitwise equal messages, equal flags."""
    gm, mm, _, _, fm = _run(binding, graph, lp, ev, T, damping, n_iters, 0, m0, cuda_graph)
    assert gm.get_option(binding.OPT_SMALL_RUN) == 0
    gs, ms, nbs, decs, fs = _run(binding, graph, lp, ev, T, damping, n_iters, mode, m0, cuda_graph)
    assert gs.get_option(binding.OPT_SMALL_RUN) == (mode if expect_small else 0)
    assert np.array_equal(ms, mm, equal_nan=True), f"max diff {np.nanmax(np.abs(ms - mm))}"
    assert fs == fm, (fs, fm)
    return ms, nbs, decs, fs


def _oracle_check(graph, lp, ev, T, damping, n_iters, nb, dec, what, m0=None):
    if m0 is None:
        om, _ = oracle.run_bp(graph, lp, ev, T, damping, n_iters)
    else:
        om, _ = oracle.run_bp(graph, lp, ev, T, damping, n_iters, msgs=m0)
    _, onb, _, _ = oracle.beliefs(graph, ev, om)
    assert_beliefs_close(nb, onb, what=what)
    assert_decode_ok(dec, onb, graph.num_states, what=what)


@pytest.mark.parametrize("T", [1.0, 0.0])
def test_ising10x10(gpu, T):
    """The 10 x 10 Ising grid (180 factors), 50 iterations: bitwise equal to the
    multi-launch run, and the oracle at 1e-4."""
    p = W.ising_small(0)
    _, nb, dec, _ = _both(gpu, p.graph, p.log_pot, p.evidence, T, 0.5, 50)
    _oracle_check(p.graph, p.log_pot, p.evidence, T, 0.5, 50, nb, dec, f"ising10x10 T={T}")


@pytest.mark.parametrize("shape", [(1, 2), (2, 2), (1, 50), (3, 7), (23, 23), (24, 24), (26, 27), (31, 31),
                                   (32, 32), (8, 128), (1, 1024), (33, 33), (1, 1025), (45, 45), (64, 64),
                                   (90, 90), (64, 128), (1, 8192), (91, 91), (128, 128), (1, 16384)])
def test_sizes_up_to_the_limit(gpu, shape):
    """From one factor to the limits: one block with one factor per thread or two (23 x 23:
    1,012 factors; 24 x 24: 1,104) up to 700 variables; then the cluster (16 blocks on a
    GB300) from 702 variables (26 x 27) through 1,024 and 8,192 (64 x 128: 16,192 factors)
    to 16,384 (128 x 128: 32,512 factors, two per thread; a chain of 16,384)."""
    r, c = shape
    p = W.ising_grid(r, c, seed=r * 100 + c, T=1.0)
    for T in (1.0, 0.0):
        _, nb, dec, _ = _both(gpu, p.graph, p.log_pot, p.evidence, T, 0.5, 20)
        _oracle_check(p.graph, p.log_pot, p.evidence, T, 0.5, 20, nb, dec, f"ising{r}x{c} T={T}")


@pytest.mark.parametrize("shape", [(129, 128), (1, 16385)])
def test_above_the_limit_keeps_the_launches(gpu, shape):
    """16,512 and 16,385 variables: above the limit, the multi-launch form."""
    r, c = shape
    p = W.ising_grid(r, c, seed=3, T=1.0)
    _both(gpu, p.graph, p.log_pot, p.evidence, 1.0, 0.5, 10, expect_small=False)


def _hard(ev, frac, seed, both=False):
    """-inf evidence on one state of a fraction of the variables (both states: a
    contradiction)."""
    rng = np.random.default_rng(seed)
    e = np.asarray(ev, np.float32).reshape(-1, 2).copy()
    rows = np.flatnonzero(rng.random(e.shape[0]) < frac)
    e[rows, rng.integers(0, 2, rows.size)] = -np.inf
    if both and rows.size:
        e[rows[0]] = -np.inf
    return e.ravel()


@pytest.mark.parametrize("T", [1.0, 0.0])
def test_hard_evidence(gpu, T):
    """Clamped variables take the explicit-sum path (lr_var_slow's sums in global lam,
    read by the factor pass after the barrier)."""
    p = W.ising_grid(20, 20, seed=7, T=T)
    ev = _hard(p.evidence, 0.15, 8)
    _, nb, dec, _ = _both(gpu, p.graph, p.log_pot, ev, T, 0.5, 30)
    _oracle_check(p.graph, p.log_pot, ev, T, 0.5, 30, nb, dec, f"hard evidence T={T}")


@pytest.mark.parametrize("T", [1.0, 0.0])
def test_contradiction_flag(gpu, T):
    """A variable with both states at -inf: both forms raise the same flags and store the
    same messages."""
    p = W.ising_grid(12, 12, seed=9, T=T)
    ev = _hard(p.evidence, 0.1, 10, both=True)
    _, _, _, flags = _both(gpu, p.graph, p.log_pot, ev, T, 0.5, 15)
    assert flags & gpu.FLAG_CONTRADICTION


def test_tables_with_neg_inf_entries_and_shared_tables(gpu):
    """Per-factor tables with a forbidden configuration (-inf entry: the exact path of the
    factor update), and a group sharing one table, in one graph."""
    rng = np.random.default_rng(11)
    p = W.ising_grid(15, 15, seed=11, T=1.0)
    lp = p.log_pot.reshape(-1, 4).copy()
    bad = rng.choice(lp.shape[0], 40, replace=False)
    lp[bad, rng.integers(0, 4, bad.size)] = -np.inf
    pairs = p.graph.enum_groups[0].vars
    half = pairs.shape[0] // 2
    cfg = W.PAIR2_CFG.copy()
    graph = W.FactorGraph(p.graph.num_states, [W.EnumGroup(cfg, pairs[:half], False),
                                               W.EnumGroup(cfg, pairs[half:], True)], [])
    lp2 = np.concatenate([lp[:half].ravel(), np.array([0.4, -0.4, -0.4, 0.4], np.float32)])
    for T in (1.0, 0.0):
        _, nb, dec, _ = _both(gpu, graph, lp2, p.evidence, T, 0.5, 25)
        _oracle_check(graph, lp2, p.evidence, T, 0.5, 25, nb, dec, f"-inf tables T={T}")


def test_damping_zero_warm_start_and_no_cuda_graph(gpu):
    """Damping 0, a run continued from the messages of an earlier run, and kernels
    launched one by one."""
    p = W.ising_grid(24, 24, seed=12, T=1.0)
    _, _, _, _, _ = _run(gpu, p.graph, p.log_pot, p.evidence, 1.0, 0.5, 10, 1)
    m0 = _run(gpu, p.graph, p.log_pot, p.evidence, 1.0, 0.5, 10, 0)[1]
    _, nb, dec, _ = _both(gpu, p.graph, p.log_pot, p.evidence, 1.0, 0.0, 12, m0=m0, cuda_graph=0)
    _oracle_check(p.graph, p.log_pot, p.evidence, 1.0, 0.0, 12, nb, dec, "damping 0, warm start", m0=m0)
    _both(gpu, p.graph, p.log_pot, p.evidence, 0.0, 0.5, 12, m0=m0, cuda_graph=1)


def test_qualifying_graphs(gpu):
    """The option reports the single-block form only for binary pairwise graphs in the
    4-slot layout within the limits; short runs below the log-ratio threshold keep the
    edge-state iterations either way."""
    import torch
    p = W.ising_small(0)
    g = gpu.Graph(p.graph)
    assert g.get_option(gpu.OPT_SMALL_RUN) == 1
    g.set_option(gpu.OPT_SMALL_RUN, 0)
    assert g.get_option(gpu.OPT_SMALL_RUN) == 0
    with pytest.raises(gpu.PgmError):
        g.set_option(gpu.OPT_SMALL_RUN, 3)
    pk = W.potts_grid(8, 4, seed=1, T=1.0)
    assert gpu.Graph(pk.graph).get_option(gpu.OPT_SMALL_RUN) == 0  # not binary
    # a hub variable with 6 factors: the CSR log-ratio layout, not the 4-slot one
    pairs = np.array([[0, i] for i in range(1, 7)], np.int32)
    hub = W.FactorGraph(np.full(7, 2, np.int32), [W.EnumGroup(W.PAIR2_CFG.copy(), pairs, False)], [])
    gh = gpu.Graph(hub)
    assert gh.get_option(gpu.OPT_SMALL_RUN) == 0
    # 3 iterations (below the default log-ratio threshold of 4): edge-state iterations
    gs, ms, nb, dec, _ = _run(gpu, p.graph, p.log_pot, p.evidence, 1.0, 0.5, 3, 1)
    _, mm, _, _, _ = _run(gpu, p.graph, p.log_pot, p.evidence, 1.0, 0.5, 3, 0)
    assert np.array_equal(ms, mm)
    _oracle_check(p.graph, p.log_pot, p.evidence, 1.0, 0.5, 3, nb, dec, "3 iterations")


def _permuted(p, seed):
    """The same grid with its variables numbered at random: a factor's two variables, and
    a variable's four slots, then mostly live in other blocks of the cluster."""
    rng = np.random.default_rng(seed)
    n = p.graph.num_states.size
    perm = rng.permutation(n).astype(np.int32)
    g0 = p.graph.enum_groups[0]
    graph = W.FactorGraph(p.graph.num_states, [W.EnumGroup(g0.cfg, perm[g0.vars], False)], [])
    ev = np.empty_like(p.evidence.reshape(-1, 2))
    ev[perm] = p.evidence.reshape(-1, 2)
    return graph, ev.ravel()


@pytest.mark.parametrize("T", [1.0, 0.0])
def test_cluster_random_numbering_and_hard_evidence(gpu, T):
    """A 60 x 60 grid (3,600 variables: a cluster) numbered at random, plain and with hard
    and contradictory evidence: bitwise equal to the multi-launch run, and the oracle."""
    p = W.ising_grid(60, 60, seed=21, T=T)
    graph, ev = _permuted(p, 22)
    _, nb, dec, _ = _both(gpu, graph, p.log_pot, ev, T, 0.5, 25)
    _oracle_check(graph, p.log_pot, ev, T, 0.5, 25, nb, dec, f"permuted 60x60 T={T}")
    evh = _hard(ev, 0.1, 23)
    _, nb, dec, _ = _both(gpu, graph, p.log_pot, evh, T, 0.5, 25)
    _oracle_check(graph, p.log_pot, evh, T, 0.5, 25, nb, dec, f"permuted 60x60 hard T={T}")
    evc = _hard(ev, 0.05, 24, both=True)
    _, _, _, flags = _both(gpu, graph, p.log_pot, evc, T, 0.5, 10)
    assert flags & gpu.FLAG_CONTRADICTION


def test_cluster_tables_damping_and_warm_start(gpu):
    """The cluster with -inf table entries and a shared table group, damping 0 from warm
    messages, kernels launched one by one."""
    rng = np.random.default_rng(31)
    p = W.ising_grid(50, 70, seed=31, T=1.0)
    lp = p.log_pot.reshape(-1, 4).copy()
    bad = rng.choice(lp.shape[0], 300, replace=False)
    lp[bad, rng.integers(0, 4, bad.size)] = -np.inf
    pairs = p.graph.enum_groups[0].vars
    half = pairs.shape[0] // 2
    cfg = W.PAIR2_CFG.copy()
    graph = W.FactorGraph(p.graph.num_states, [W.EnumGroup(cfg, pairs[:half], False),
                                               W.EnumGroup(cfg, pairs[half:], True)], [])
    lp2 = np.concatenate([lp[:half].ravel(), np.array([0.3, -0.3, -0.3, 0.3], np.float32)])
    _, nb, dec, _ = _both(gpu, graph, lp2, p.evidence, 1.0, 0.5, 20)
    _oracle_check(graph, lp2, p.evidence, 1.0, 0.5, 20, nb, dec, "cluster -inf tables")
    m0 = _run(gpu, graph, lp2, p.evidence, 1.0, 0.5, 10, 0)[1]
    _, nb, dec, _ = _both(gpu, graph, lp2, p.evidence, 1.0, 0.0, 12, m0=m0, cuda_graph=0)
    _oracle_check(graph, lp2, p.evidence, 1.0, 0.0, 12, nb, dec, "cluster damping 0, warm start", m0=m0)


@pytest.mark.parametrize("shape", [(1, 2), (2, 2), (2, 3), (3, 7), (10, 10), (24, 24), (32, 32)])
def test_cluster_forced_on_small_graphs(gpu, shape):
    """Setting 2 runs the cluster at any size it takes: with fewer variables than blocks
    (1 x 2, 2 x 2, 2 x 3), blocks that own no variable or no factor still take part in
    every barrier; bitwise equal to the multi-launch run, and the oracle."""
    r, c = shape
    p = W.ising_grid(r, c, seed=r * 10 + c + 5, T=1.0)
    for T in (1.0, 0.0):
        _, nb, dec, _ = _both(gpu, p.graph, p.log_pot, p.evidence, T, 0.5, 16, mode=2)
        _oracle_check(p.graph, p.log_pot, p.evidence, T, 0.5, 16, nb, dec, f"cluster {r}x{c} T={T}")
    evh = _hard(p.evidence, 0.2, r + c)
    _both(gpu, p.graph, p.log_pot, evh, 1.0, 0.5, 16, mode=2)
