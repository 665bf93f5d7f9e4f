"""Log-ratio iterations of binary pairwise graphs (PGM_OPT_LOG_RATIO).

A max-normalised binary message (Sec. 3) has one entry exactly 0, so the iterations may
keep d = m(1) - m(0) per edge; the variable-to-factor values are kept the same way, as
exact leave-one-out sums. The iteration map is unchanged, so:

* "strict" runs match the FP64 oracle to 1e-4 (the same criteria as the edge-state path);
* "stepwise": with the option set to 1, single log-ratio iterations from the GPU's own
  messages match one oracle iteration, including hard (-inf) potentials, couplings of
  several hundred and contradictory evidence;
* warm starts (normalised or not), batches of binary grids and the launch counts behave
  as documented; graphs that do not qualify report the option as 0.
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


def _binary_pairwise(seed, n_vars, n_fac, hard_frac=0.0, big_frac=0.0, max_deg=40):
    """Random binary pairwise graph, variable degrees <= max_deg, with a fraction of
    hard (-inf) table entries and of large couplings (|J| up to 300)."""
    rng = np.random.default_rng(seed)
    deg = np.zeros(n_vars, np.int64)
    pairs = []
    while len(pairs) < n_fac:
        a, b = rng.integers(0, n_vars, 2)
        if a == b or deg[a] >= max_deg or deg[b] >= max_deg:
            continue
        deg[a] += 1
        deg[b] += 1
        pairs.append((a, b))
    pairs = np.asarray(pairs, np.int32)
    J = rng.uniform(-1.5, 1.5, n_fac)
    J[rng.random(n_fac) < big_frac] *= 200.0
    pot = np.stack([J, -J, -J, J], axis=1)
    hard = rng.random(n_fac) < hard_frac
    pot[hard, rng.integers(0, 4, hard.sum())] = -np.inf
    ev = rng.standard_normal((n_vars, 2))
    g = W.FactorGraph(np.full(n_vars, 2, np.int32), [W.EnumGroup(W.PAIR2_CFG.copy(), pairs, False)], [])
    return g, pot.astype(np.float32).ravel(), ev.astype(np.float32).ravel()


def _tensors(lp, ev):
    import torch
    return (torch.as_tensor(np.asarray(lp, np.float32)).cuda(),
            torch.as_tensor(np.asarray(ev, np.float32)).cuda())


def _run(binding, g, lp, ev, T, n_iters, lr_min=4, msgs0=None, damping=0.5, cuda_graph=True):
    import torch
    G = binding.Graph(g)
    G.set_option(binding.OPT_LOG_RATIO, lr_min)
    G.set_option(binding.OPT_CUDA_GRAPH, 1 if cuda_graph else 0)
    lpt, evt = _tensors(lp, ev)
    m = G.new_msgs() if msgs0 is None else torch.as_tensor(np.asarray(msgs0, np.float32)).cuda()
    G.run_bp(lpt, evt, T, damping, n_iters, m)
    nb = G.beliefs(evt, m, True)
    dec = G.decode(evt, m)
    return G, m.cpu().numpy(), nb.cpu().numpy(), dec.cpu().numpy(), G.flags(clear=True)


def _check(binding, g, lp, ev, T, n_iters, what, **kw):
    G, m, nb, dec, flags = _run(binding, g, lp, ev, T, n_iters, **kw)
    om, ofl = oracle.run_bp(g, lp, ev, T, kw.get("damping", 0.5), n_iters,
                            msgs=kw.get("msgs0"))
    _, onb, _, ofl2 = oracle.beliefs(g, ev, om)
    assert_beliefs_close(nb, onb, what=what)
    assert_decode_ok(dec, onb, g.num_states, what=what)
    assert bool(flags & 1) == bool((ofl | ofl2) & 1), (what, flags, ofl, ofl2)
    return G, m, om


def _stepwise(binding, g, lp, ev, T, points, what, damping=0.5, atol=1e-4, rtol=1e-6):
    """Single log-ratio iterations (option = 1) from the GPU's own messages at each of
    `points` against one FP64 oracle iteration from the same messages."""
    G = binding.Graph(g)
    G.set_option(binding.OPT_LOG_RATIO, 1)
    assert G.get_option(binding.OPT_LOG_RATIO) == 1
    lpt, evt = _tensors(lp, ev)
    msgs = G.new_msgs()
    done = 0
    for t in sorted(points):
        if t > done:
            G.run_bp(lpt, evt, T, damping, t - done, msgs)
            done = t
        m_t = msgs.cpu().numpy().astype(np.float64)
        G.run_bp(lpt, evt, T, damping, 1, msgs)
        done += 1
        m_gpu = msgs.cpu().numpy().astype(np.float64)
        nb_gpu = G.beliefs(evt, msgs, True).cpu().numpy().astype(np.float64)
        m_ora, _ = oracle.run_bp(g, lp, ev, T, damping, 1, msgs=m_t)
        _, nb_ora, _, _ = oracle.beliefs(g, ev, m_ora)
        for name, a, o in (("messages", m_gpu, m_ora), ("beliefs", nb_gpu, nb_ora)):
            assert not np.isnan(a).any(), f"{what} step {t}: NaN in GPU {name}"
            assert (np.isneginf(a) == np.isneginf(o)).all(), f"{what} step {t}: -inf pattern of {name}"
            fin = np.isfinite(o)
            err = np.abs(a[fin] - o[fin])
            tol = atol + rtol * np.abs(o[fin])
            if err.size:
                k = int(np.argmax(err - tol))
                assert (err <= tol).all(), f"{what} step {t}: {name} differ by {err[k]:.3e} (oracle {o[fin][k]:.6g})"


def _cases(T):
    it = 40 if T > 0 else 20
    p = W.ising_grid(37, 53, 11)
    yield "ising37x53", p.graph, p.log_pot, p.evidence, it
    g, lp, ev = _binary_pairwise(12, 3000, 9000)
    yield "sparse-deg40", g, lp, ev, (it if T > 0 else 10)
    p = W.ising_grid(1, 2, 14)
    yield "one-factor", p.graph, p.log_pot, p.evidence, it


@pytest.mark.parametrize("T", [1.0, 0.0])
@pytest.mark.parametrize("cuda_graph", [True, False])
def test_strict_parity(gpu, T, cuda_graph):
    for name, g, lp, ev, it in _cases(T):
        G, _, _ = _check(gpu, g, lp, ev, T, it, f"{name} T={T}", cuda_graph=cuda_graph)
        assert G.get_option(gpu.OPT_LOG_RATIO) == 4, name


def _contradictory_grid():
    p = W.ising_grid(8, 9, 15)
    ev = p.evidence.copy()
    ev[2 * 20: 2 * 20 + 2] = -np.inf  # variable 20: both states impossible
    return p.graph, p.log_pot, ev


@pytest.mark.parametrize("T", [1.0, 0.0])
def test_stepwise(gpu, T):
    p = W.ising_grid(37, 53, 11)
    _stepwise(gpu, p.graph, p.log_pot, p.evidence, T, [0, 3, 17, 60], f"ising T={T}")
    g, lp, ev = _binary_pairwise(13, 2000, 5000, hard_frac=0.02, big_frac=0.05)
    _stepwise(gpu, g, lp, ev, T, [0, 3, 17], f"hard-and-large T={T}")
    g, lp, ev = _contradictory_grid()
    _stepwise(gpu, g, lp, ev, T, [0, 2, 9], f"contradiction T={T}")
    _stepwise(gpu, g, lp, ev, T, [0, 4], f"no damping T={T}", damping=0.0)


def test_contradiction_flag(gpu):
    g, lp, ev = _contradictory_grid()
    for T in (1.0, 0.0):
        G, m, nb, _, flags = _run(gpu, g, lp, ev, T, 12)
        assert G.get_option(gpu.OPT_LOG_RATIO) == 4
        assert flags & 1 and not np.isnan(m).any()
        assert np.isneginf(nb[40:42]).all()


def test_warm_starts(gpu):
    # from a previous run (max-normalised messages): 9 + 25 iterations = 34
    p = W.ising_grid(24, 29, 31)
    _, m_a, _, _, _ = _run(gpu, p.graph, p.log_pot, p.evidence, 1.0, 9)
    _check(gpu, p.graph, p.log_pot, p.evidence, 1.0, 25, "warm 9+25", msgs0=m_a)
    om, _ = oracle.run_bp(p.graph, p.log_pot, p.evidence, 1.0, 0.5, 34)
    _, m_b, _, _, _ = _run(gpu, p.graph, p.log_pot, p.evidence, 1.0, 25, msgs0=m_a)
    np.testing.assert_allclose(m_b, om, atol=1e-4, rtol=0)
    # from messages that are not max-normalised (neither entry 0)
    rng = np.random.default_rng(32)
    m_init = rng.normal(0.0, 2.0, oracle.sizes(p.graph)["ES"]).astype(np.float32)
    for T in (1.0, 0.0):
        _check(gpu, p.graph, p.log_pot, p.evidence, T, 6, f"unnormalised warm T={T}", msgs0=m_init)


def test_short_runs_and_zero_iterations(gpu):
    p = W.ising_grid(16, 16, 41)
    for n_it in (1, 3, 4, 5):  # below the default minimum: edge-state path
        _check(gpu, p.graph, p.log_pot, p.evidence, 1.0, n_it, f"{n_it} iterations")
    rng = np.random.default_rng(42)
    m_init = rng.normal(0.0, 1.0, oracle.sizes(p.graph)["ES"]).astype(np.float32)
    _, m, _, _, _ = _run(gpu, p.graph, p.log_pot, p.evidence, 1.0, 0, lr_min=1, msgs0=m_init)
    assert np.array_equal(m, m_init)  # n_iters = 0 leaves msgs untouched


def test_option_values_and_ineligible_graphs(gpu):
    potts = W.potts_grid(8, 3, 1)
    rbm = W.rbm(80, 70, 2)  # variables with more than 64 factors
    g, _, _ = W.random_graph(3, n_vars=20, max_K=2, n_pair=20, n_triple=2, n_or=2, n_and=1)
    for graph in (potts.graph, rbm.graph, g):
        G = gpu.Graph(graph)
        assert G.get_option(gpu.OPT_LOG_RATIO) == 0
        G.set_option(gpu.OPT_LOG_RATIO, 1)
        assert G.get_option(gpu.OPT_LOG_RATIO) == 0
    G = gpu.Graph(W.ising_grid(4, 4, 3).graph)
    assert G.get_option(gpu.OPT_LOG_RATIO) == 4
    assert G.get_option(gpu.OPT_CUDA_GRAPH) == 1
    G.set_option(gpu.OPT_LOG_RATIO, 0)
    assert G.get_option(gpu.OPT_LOG_RATIO) == 0
    with pytest.raises(gpu.PgmError):
        G.set_option(gpu.OPT_LOG_RATIO, -1)
    with pytest.raises(gpu.PgmError):
        G.get_option(99)


def test_batch_of_binary_grids(gpu):
    """Members alone and inside a batch of binary grids run the same log-ratio
    arithmetic (bitwise equal) and match the oracle."""
    import torch
    members = [W.ising_grid(9 + 3 * i, 14 + 5 * i, 50 + i) for i in range(6)]
    batch = W.union(members)
    G = gpu.Graph([p.graph for p in members])
    assert G.get_option(gpu.OPT_LOG_RATIO) == 4
    lpt, evt = _tensors(batch.log_pot, batch.evidence)
    m = G.new_msgs()
    G.run_bp(lpt, evt, 1.0, 0.5, 30, m)
    nb = G.beliefs(evt, m, True).cpu().numpy()
    m = m.cpu().numpy()
    for i, p in enumerate(members):
        off = G.member(i)
        _, m1, nb1, _, _ = _run(gpu, p.graph, p.log_pot, p.evidence, 1.0, 30)
        assert np.array_equal(m[off["es_off"]: off["es_off"] + off["n_edge_states"]], m1)
        nbi = nb[off["vs_off"]: off["vs_off"] + off["n_var_states"]]
        assert np.array_equal(nbi, nb1)
        onb, _, _, _ = oracle.infer(p, n_iters=30, T=1.0)
        assert_beliefs_close(nbi, onb)
