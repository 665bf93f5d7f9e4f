"""Dense K-state pairwise factors (Potts, Sec. 5.2's enumeration factors over full
tables): the kernel forms of the factor pass give the same results.

The K / 4-lane form (four states per lane, for tables shared by a group), the
direction form (a thread per factor and direction) -- alternatives the autotuner may
pick -- and the thread-per-factor form (the default) run the same arithmetic in the same
order, so their messages are bitwise equal: with the linear-domain form of a shared table (range within
60 T), with the exact form (a table range above 60 T), at T = 0, with hard evidence (the
rare path), in batches whose members start at any offset, and for many samples at once.
Both are held to the FP64 oracle as well.
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


def _run_form(binding, graph, lp, ev, T, n_iters, form, damping=0.5, samples=0):
    import torch
    g = binding.Graph(graph)
    g.set_option(binding.OPT_PAIR_FORM, form)
    lpt = torch.as_tensor(np.asarray(lp, np.float32)).cuda()
    if samples:
        evt = torch.as_tensor(np.asarray(ev, np.float32)).cuda()
        m = torch.zeros(samples, g.info["n_edge_states"], device="cuda")
        g.run_bp_multi(lpt, evt, T, damping, n_iters, m)
        return g, m.cpu().numpy()
    evt = torch.as_tensor(np.asarray(ev, np.float32)).cuda()
    m = g.new_msgs()
    g.run_bp(lpt, evt, T, damping, n_iters, m)
    return g, m.cpu().numpy()


def _hard(p, frac, seed):
    """Clamp a fraction of the variables to one state with -inf evidence."""
    rng = np.random.default_rng(seed)
    K = int(p.graph.num_states[0])
    ev = p.evidence.reshape(-1, K).copy()
    rows = np.flatnonzero(rng.random(ev.shape[0]) < frac)
    keep = rng.integers(0, K, rows.size)
    ev[rows] = -np.inf
    ev[rows, keep] = 0.0
    p.evidence = ev.ravel()
    return p


@pytest.mark.parametrize("K", [8, 16])
@pytest.mark.parametrize("T", [1.0, 0.0, 0.4])
@pytest.mark.parametrize("case", ["plain", "wide_table", "hard"])
def test_quad_equals_thread_form(gpu, K, T, case):
    side = 37
    w = 40.0 if case == "wide_table" else None  # range 80 > 60 T: the exact (non-linear) form
    p = W.potts_grid(side, K, seed=K + 3, T=T, n_iters=15, w=w)
    if case == "hard":
        p = _hard(p, 0.1, 5)
    g_q, m_q = _run_form(gpu, p.graph, p.log_pot, p.evidence, T, 15, 3)
    assert g_q.launches()[-1][1] == (11 if K == 8 else 12)
    _, m_t = _run_form(gpu, p.graph, p.log_pot, p.evidence, T, 15, 1)
    assert np.array_equal(m_q, m_t, equal_nan=True), f"max diff {np.nanmax(np.abs(m_q - m_t))}"
    import torch
    evt = torch.as_tensor(p.evidence).cuda()
    mt = torch.as_tensor(m_q).cuda()
    nb = g_q.beliefs(evt, mt, True).cpu().numpy()
    dec = g_q.decode(evt, mt).cpu().numpy()
    if case == "wide_table":
        # log-beliefs reach 324 (one FP32 ulp: 3e-5) and FP32 message storage alone moves
        # the FP64 run by 9e-5: held to the oracle's ensemble envelope instead of 1e-4
        nb0, _, spread, unstable, _ = oracle_envelope(oracle, p.graph, p.log_pot, p.evidence, T, 0.5, 15)
        assert_within_envelope(nb, dec, nb0, spread, unstable, p.graph.num_states, factor=10.0,
                               what=f"K={K} T={T} {case}")
        return
    om, _ = oracle.run_bp(p.graph, p.log_pot, p.evidence, T, 0.5, 15)
    _, onb, _, _ = oracle.beliefs(p.graph, p.evidence, om)
    assert_beliefs_close(nb, onb, what=f"K={K} T={T} {case}")
    assert_decode_ok(dec, onb, p.graph.num_states, what=f"K={K} T={T} {case}")


def test_quad_in_batch_at_any_offset(gpu):
    """Members of 2, 4 and 8 states before the 16-state grids put their messages and
    beliefs at offsets that are not multiples of four floats; the batched run equals the
    thread form and each member alone."""
    ms = [W.potts_grid(13, 2, 1, T=1.0), W.potts_grid(17, 16, 2, T=1.0), W.potts_grid(11, 4, 3, T=1.0),
          W.potts_grid(9, 8, 4, T=1.0), W.ising_grid(3, 5, 5, T=1.0), W.potts_grid(21, 16, 6, T=1.0)]
    batch = W.union(ms)
    graphs = [p.graph for p in ms]
    g_q, m_q = _run_form(gpu, graphs, batch.log_pot, batch.evidence, 1.0, 12, 3)
    _, m_t = _run_form(gpu, graphs, batch.log_pot, batch.evidence, 1.0, 12, 1)
    assert np.array_equal(m_q, m_t)
    for i, p in enumerate(ms):
        off = g_q.member(i)
        g1 = gpu.Graph(p.graph)
        g1.set_option(gpu.OPT_LOG_RATIO, 0)
        import torch
        m1 = g1.new_msgs()
        g1.run_bp(torch.as_tensor(p.log_pot).cuda(), torch.as_tensor(p.evidence).cuda(), 1.0, 0.5, 12, m1)
        seg = m_q[off["es_off"]: off["es_off"] + off["n_edge_states"]]
        assert np.array_equal(seg, m1.cpu().numpy()), p.name


@pytest.mark.parametrize("T", [1.0, 0.0])
def test_quad_multi_sample(gpu, T):
    p = W.potts_grid(29, 16, 9, T=T, n_iters=10)
    S = 5
    rng = np.random.default_rng(3)
    ev = (p.evidence[None, :] + rng.standard_normal((S, p.evidence.size))).astype(np.float32)
    _, mq = _run_form(gpu, p.graph, p.log_pot, ev, T, 10, 3, samples=S)
    _, mt = _run_form(gpu, p.graph, p.log_pot, ev, T, 10, 1, samples=S)
    assert np.array_equal(mq, mt)
    for s in range(S):
        _, m1 = _run_form(gpu, p.graph, p.log_pot, ev[s], T, 10, 0)
        assert np.array_equal(mq[s], m1), s


def _per_factor_tables(p, seed):
    """The Potts grid with its own table per factor: the shared table plus N(0, 0.3)."""
    rng = np.random.default_rng(seed)
    g0 = p.graph.enum_groups[0]
    n_fac = g0.vars.shape[0]
    lp = (np.tile(p.log_pot, n_fac) + rng.normal(0, 0.3, n_fac * p.log_pot.size)).astype(np.float32)
    graph = W.FactorGraph(p.graph.num_states, [W.EnumGroup(g0.cfg, g0.vars, False)], [])
    return graph, lp


@pytest.mark.parametrize("K", [4, 8, 16])
@pytest.mark.parametrize("T", [1.0, 0.0, 0.4])
@pytest.mark.parametrize("case", ["plain", "wide_table", "hard", "per_factor"])
def test_direction_form_equals_thread_form(gpu, K, T, case):
    """A thread per factor and direction (form 4) against the thread form: bitwise, on
    shared tables (linear and exact forms), hard evidence (the rare path, finished by the
    even warp) and per-factor tables; and the oracle at 1e-4 on the plain case."""
    side = 37
    w = 40.0 if case == "wide_table" else None
    p = W.potts_grid(side, K, seed=K + 7, T=T, n_iters=15, w=w)
    if case == "hard":
        p = _hard(p, 0.1, 6)
    graph, lp = (p.graph, p.log_pot) if case != "per_factor" else _per_factor_tables(p, K)
    g_d, m_d = _run_form(gpu, graph, lp, p.evidence, T, 15, 4)
    assert g_d.launches()[-1][1] == {4: 13, 8: 14, 16: 15}[K]
    _, m_t = _run_form(gpu, graph, lp, p.evidence, T, 15, 1)
    assert np.array_equal(m_d, m_t, equal_nan=True), f"max diff {np.nanmax(np.abs(m_d - m_t))}"
    if case == "plain":
        import torch
        evt = torch.as_tensor(p.evidence).cuda()
        nb = g_d.beliefs(evt, torch.as_tensor(m_d).cuda(), True).cpu().numpy()
        om, _ = oracle.run_bp(graph, lp, p.evidence, T, 0.5, 15)
        _, onb, _, _ = oracle.beliefs(graph, p.evidence, om)
        assert_beliefs_close(nb, onb, what=f"direction form K={K} T={T}")


def test_direction_form_batch_and_samples(gpu):
    """The direction form in a batch whose members start at any offset, and for many
    samples at once: bitwise equal to the thread form."""
    ms = [W.potts_grid(13, 2, 1, T=1.0), W.potts_grid(17, 16, 2, T=1.0), W.potts_grid(11, 4, 3, T=1.0),
          W.potts_grid(9, 8, 4, T=1.0), W.ising_grid(3, 5, 5, T=1.0), W.potts_grid(21, 16, 6, T=1.0)]
    batch = W.union(ms)
    graphs = [p.graph for p in ms]
    _, m_d = _run_form(gpu, graphs, batch.log_pot, batch.evidence, 1.0, 12, 4)
    _, m_t = _run_form(gpu, graphs, batch.log_pot, batch.evidence, 1.0, 12, 1)
    assert np.array_equal(m_d, m_t)
    p = W.potts_grid(29, 8, 9, T=0.0, n_iters=10)
    rng = np.random.default_rng(4)
    ev = (p.evidence[None, :] + rng.standard_normal((4, p.evidence.size))).astype(np.float32)
    _, md = _run_form(gpu, p.graph, p.log_pot, ev, 0.0, 10, 4, samples=4)
    _, mt = _run_form(gpu, p.graph, p.log_pot, ev, 0.0, 10, 1, samples=4)
    assert np.array_equal(md, mt)
