"""Large listed-configuration factors: the block-per-factor form (launch variant 10).

Groups whose state sum is above 64 or whose list is longer than 256 configurations run
with a block per run of factors and the group's table staged in shared memory. Checked
against the FP64 oracle (normalised beliefs within 1e-4 plus the spread of an ensemble of
FP64 runs perturbed at FP32 resolution, decodes except at ties and unstable states), and
against the thread-per-factor form on groups both can run (PGM_OPT_ENUM_BLOCK): the same
bits.
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


def _t(a):
    import torch
    return torch.as_tensor(np.asarray(a, np.float32)).cuda()


def _variants(g):
    return [variant for kind, variant, _, _ in g.launches() if kind == 1]


def _run(gpu, p, T, n_iters, option=None, autotune=False):
    g = gpu.Graph(p.graph)
    if option is not None:
        g.set_option(gpu.OPT_ENUM_BLOCK, option)
    lp, ev = _t(p.log_pot), _t(p.evidence)
    if autotune:
        g.autotune(lp, ev, T, p.damping)
    m = g.new_msgs()
    g.run_bp(lp, ev, T, p.damping, n_iters, m)
    nb = g.beliefs(ev, m, True).cpu().numpy()
    dec = g.decode(ev, m).cpu().numpy()
    return g, m.cpu().numpy(), nb, dec


def _oracle(p, T, n_iters):
    om, fl = oracle.run_bp(p.graph, p.log_pot, p.evidence, T, p.damping, n_iters)
    _, onb, odec, fl2 = oracle.beliefs(p.graph, p.evidence, om)
    return om, onb, fl | fl2


CASES = {
    # RCN-like lateral factors: 49 states, 361 of 49 x 49 pairs listed (state sum 98)
    "pool49": lambda: W.pool_grid(6, 3, 1, 3, n_iters=25),
    "pool49_per_factor": lambda: W.pool_grid(5, 3, 1, 4, n_iters=25, shared=False),
    # 121 states, 2401 pairs (long lists: several lanes per output state)
    "pool121": lambda: W.pool_grid(4, 5, 2, 5, n_iters=20),
    # dense 48 x 48 pairs given as a list (state sum 96)
    "dense48": lambda: W.random_enum_factors(6, 30, 48, 2, 60, 48 * 48, n_iters=20),
    # 8-ary factors over 16-state variables, 3000 listed configurations (state sum 128)
    # (a sparse random list over 16^8 configurations; more factors per variable make the
    # run chaotic at FP32 resolution, which the oracle ensemble below measures)
    "arity8": lambda: W.random_enum_factors(7, 100, 16, 8, 12, 4000, n_iters=10, scale=0.5),
    # 3-ary, 40 states, a list of 5000 of 64000 (per-factor tables)
    "arity3_per_factor": lambda: W.random_enum_factors(8, 50, 40, 3, 40, 5000, shared=False, n_iters=15),
}


@pytest.mark.parametrize("T", [1.0, 0.0])
@pytest.mark.parametrize("name", sorted(CASES))
def test_large_factors_match_oracle(gpu, name, T):
    p = CASES[name]()
    n = p.n_iters
    g, m, nb, dec = _run(gpu, p, T, n)
    assert 10 in _variants(g)  # the block-per-factor form
    nb0, _, spread, unstable, fl = oracle_envelope(oracle, p.graph, p.log_pot, p.evidence, T, p.damping, n)
    assert fl == 0
    assert_within_envelope(nb, dec, nb0, spread, unstable, p.graph.num_states, what=f"{name} T={T}")
    assert g.flags() == 0


@pytest.mark.parametrize("T", [0.0, 1.0])
@pytest.mark.parametrize("seed", range(4))
def test_block_form_equals_thread_form(gpu, seed, T):
    """Small listed-configuration groups run in both forms (the block form with one
    thread per output state, the thread form's order): the same bits."""
    g0, lp, ev = W.random_graph(seed, n_vars=10, max_K=4, n_pair=12, n_triple=3, sparse=True,
                                shared=(seed % 2 == 0))
    p = W.Problem("rg", g0, lp, ev, T, 0.5, 12)
    ga, ma, nba, _ = _run(gpu, p, T, 12)
    gb, mb, nbb, _ = _run(gpu, p, T, 12, option=1)
    assert 4 in _variants(ga) and 10 in _variants(gb) and 4 not in _variants(gb)
    assert gb.get_option(gpu.OPT_ENUM_BLOCK) == 1
    assert np.array_equal(ma, mb)
    # and back
    gb.set_option(gpu.OPT_ENUM_BLOCK, 0)
    assert 4 in _variants(gb)
    m2 = gb.new_msgs()
    gb.run_bp(_t(lp), _t(ev), T, 0.5, 12, m2)
    assert np.array_equal(m2.cpu().numpy(), ma)


def test_many_factors_per_block_and_table_in_place(gpu):
    """A 40 x 40 pool grid (3120 factors: several per block, table staged) and a
    256-state pair group whose table (30000 listed pairs) is too large to stage (read in
    place), in one graph; T = 0, plus an autotuned run with the same bits."""
    a = W.pool_grid(40, 3, 1, 11, T=0.0, n_iters=12)
    b = W.random_enum_factors(12, 30, 256, 2, 20, 30000, T=0.0, n_iters=12)
    p = W.union([a, b])
    g, m, nb, dec = _run(gpu, p, 0.0, 12)
    _, onb, fl = _oracle(p, 0.0, 12)
    assert_beliefs_close(nb, onb, what="pool40 + pair256")
    assert_decode_ok(dec, onb, p.graph.num_states, what="pool40 + pair256")
    _, m2, _, _ = _run(gpu, p, 0.0, 12, autotune=True)
    assert np.array_equal(m, m2)
    # T = 1: the shapes the autotuner picks do not change the bits either
    _, m3, _, _ = _run(gpu, p, 1.0, 12)
    _, m4, _, _ = _run(gpu, p, 1.0, 12, autotune=True)
    assert np.array_equal(m3, m4)


def test_hard_evidence_and_contradiction(gpu):
    """Evidence at -inf removes states; a variable with every state removed makes its
    factors' messages contradictory (the flag is set, the oracle agrees)."""
    p = W.pool_grid(5, 3, 1, 13, T=1.0, n_iters=10)
    ev = p.evidence.reshape(25, 49).copy()
    ev[3, :40] = -np.inf      # variable 3: 9 states left
    ev[7, :] = -np.inf        # variable 7: contradiction
    p = W.Problem(p.name, p.graph, p.log_pot, ev.ravel(), 1.0, 0.5, 10)
    g, m, nb, dec = _run(gpu, p, 1.0, 10)
    om, fl = oracle.run_bp(p.graph, p.log_pot, p.evidence, 1.0, 0.5, 10)
    assert fl != 0 and (g.flags() & 1)
    np.testing.assert_allclose(m, om, atol=1e-4, rtol=0)


def test_batch_members_bit_identical(gpu):
    """Two pool grids and a dense-48 group batched into one graph give each member's
    messages bit for bit as alone."""
    probs = [W.pool_grid(5, 3, 1, 21, T=1.0), W.pool_grid(7, 3, 1, 22, T=1.0),
             W.random_enum_factors(23, 20, 48, 2, 30, 2304, T=1.0)]
    bg = gpu.Graph([p.graph for p in probs])
    lp = _t(np.concatenate([p.log_pot for p in probs]))
    ev = _t(np.concatenate([p.evidence for p in probs]))
    m = bg.new_msgs()
    bg.run_bp(lp, ev, 1.0, 0.5, 15, m)
    mm = m.cpu().numpy()
    for k, p in enumerate(probs):
        _, ma, _, _ = _run(gpu, p, 1.0, 15)
        info = bg.member(k)
        assert np.array_equal(mm[info["es_off"]:info["es_off"] + info["n_edge_states"]], ma)
