"""Batched uneven graphs (pgm_build_batch) and the launch machinery around them.

* Every member's messages and beliefs are bitwise identical alone and inside a mixed
  batch: the per-factor and per-variable arithmetic does not depend on the batch.
* A seeded subset of the 256-Potts-grid + RBM workload (T=1, 100 iterations) matches the
  FP64 oracle to 1e-4.
* The launch-shape autotuner and CUDA-graph replay change no result.
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


def _mixed_members():
    ms = [W.potts_grid(19, 4, 1, T=1.0), W.ising_grid(23, 31, 2, T=1.0), W.potts_grid(33, 16, 3, T=1.0),
          W.rbm(70, 90, 4, T=1.0), W.potts_grid(16, 2, 5, T=1.0), W.potts_grid(40, 8, 6, T=1.0),
          W.deconvolution(7, n_img=2, T=1.0)]
    g, lp, ev = W.random_graph(8, n_vars=30, max_K=4, n_pair=50, n_triple=4, n_or=4, n_and=4)
    ms.append(W.Problem("random", g, lp, ev, 1.0, 0.5, 20))
    return ms


def _run(binding, graph_or_list, lp, ev, T, n_iters, damping=0.5):
    import torch
    g = binding.Graph(graph_or_list)
    # the edge-state arithmetic throughout: a binary grid alone would otherwise take the
    # log-ratio iterations (compared alone vs batched in test_gpu_log_ratio.py)
    g.set_option(binding.OPT_LOG_RATIO, 0)
    lpt = torch.as_tensor(np.asarray(lp, np.float32)).cuda()
    evt = torch.as_tensor(np.asarray(ev, np.float32)).cuda()
    m = g.new_msgs()
    g.run_bp(lpt, evt, T, damping, n_iters, m)
    nb = g.beliefs(evt, m, True)
    dec = g.decode(evt, m)
    return g, m.cpu().numpy(), nb.cpu().numpy(), dec.cpu().numpy()


@pytest.mark.parametrize("T", [1.0, 0.0])
def test_members_alone_equal_in_batch(gpu, T):
    members = _mixed_members()
    batch = W.union(members)
    gb, mb, nbb, decb = _run(gpu, [p.graph for p in members], batch.log_pot, batch.evidence, T, 17)
    assert gb.info["n_members"] == len(members)
    for i, p in enumerate(members):
        off = gb.member(i)
        _, m1, nb1, dec1 = _run(gpu, p.graph, p.log_pot, p.evidence, T, 17)
        assert off["n_edge_states"] == m1.size and off["n_var_states"] == nb1.size
        ms = mb[off["es_off"]: off["es_off"] + off["n_edge_states"]]
        np.testing.assert_array_equal(ms, m1, err_msg=f"messages of member {i} ({p.name})")
        np.testing.assert_array_equal(nbb[off["vs_off"]: off["vs_off"] + off["n_var_states"]], nb1)
        np.testing.assert_array_equal(decb[off["var_off"]: off["var_off"] + off["n_vars"]], dec1)


def test_batch_union_layout_matches_single_graph(gpu):
    """The batch lays members out exactly as one graph built from their disjoint union."""
    members = _mixed_members()[:4]
    batch = W.union(members)
    _, mb, nbb, _ = _run(gpu, [p.graph for p in members], batch.log_pot, batch.evidence, 1.0, 9)
    _, mu, nbu, _ = _run(gpu, batch.graph, batch.log_pot, batch.evidence, 1.0, 9)
    np.testing.assert_array_equal(mb, mu)
    np.testing.assert_array_equal(nbb, nbu)


def test_potts_rbm_subset_vs_oracle(gpu):
    """A seeded subset of the batched workload: 16 Potts grids (side 16..64, K in
    {2,4,8,16}) plus the 784x500 RBM, T=1, damping 0.5, 100 iterations."""
    members = W.potts_batch_members(seed=0, n_grids=16, hi=64, n_iters=100)
    members.append(W.rbm(784, 500, 1, w_std=0.1, T=1.0, damping=0.5, n_iters=100))
    batch = W.union(members)
    _, m, nb, dec = _run(gpu, [p.graph for p in members], batch.log_pot, batch.evidence, 1.0, 100)
    om, _ = oracle.run_bp(batch.graph, batch.log_pot, batch.evidence, 1.0, 0.5, 100)
    _, onb, _, _ = oracle.beliefs(batch.graph, batch.evidence, om)
    assert_beliefs_close(nb, onb, what="potts+rbm subset")
    assert_decode_ok(dec, onb, batch.graph.num_states, what="potts+rbm subset")


def test_autotune_and_cuda_graph_do_not_change_results(gpu):
    import torch
    members = _mixed_members()
    batch = W.union(members)
    graphs = [p.graph for p in members]
    lp = torch.as_tensor(batch.log_pot).cuda()
    ev = torch.as_tensor(batch.evidence).cuda()
    g = gpu.Graph(graphs)
    g.set_option(gpu.OPT_CUDA_GRAPH, 0)
    ref = g.new_msgs()
    g.run_bp(lp, ev, 1.0, 0.5, 13, ref)
    before = g.launches()
    g.autotune(lp, ev, 1.0, 0.5)
    after = g.launches()
    assert len(before) == len(after)
    for k in (0, 1):
        g.set_option(gpu.OPT_CUDA_GRAPH, k)
        for rep in range(2):  # second call replays the cached CUDA graph
            m = g.new_msgs()
            g.run_bp(lp, ev, 1.0, 0.5, 13, m)
            assert torch.equal(m, ref), (k, rep, before, after)


@pytest.mark.parametrize("cuda_graph", [1, 0])
def test_pass_timing(gpu, cuda_graph):
    """pgm_set_profiling / pgm_pass_times: every period-th iteration's passes are timed,
    inside the cached CUDA graph when graphs are on; results are unchanged."""
    import torch
    p = W.ising_grid(64, 80, 7)
    for lr_min in (4, 0):  # log-ratio and edge-state iterations
        g = gpu.Graph(p.graph)
        g.set_option(gpu.OPT_CUDA_GRAPH, cuda_graph)
        g.set_option(gpu.OPT_LOG_RATIO, lr_min)
        lp = torch.as_tensor(p.log_pot).cuda()
        ev = torch.as_tensor(p.evidence).cuda()
        ref = g.new_msgs()
        g.run_bp(lp, ev, 1.0, 0.5, 30, ref)
        g.set_profiling(7)
        for rep in range(3):  # replays of the same cached graph
            m = g.new_msgs()
            g.run_bp(lp, ev, 1.0, 0.5, 30, m)
            assert torch.equal(m, ref)
        var_ms, fac_ms, n_var, n_fac = g.pass_times()
        per_call = 30 // 7  # iterations 6, 13, 20, 27
        assert g.info["launches_per_iter"] == 2  # one variable and one factor launch
        assert n_var == n_fac == 3 * per_call
        assert var_ms > 0 and fac_ms > 0
        assert g.pass_times()[2] == 0  # reset
        g.set_profiling(0)


def _alone(binding, p, T, damping, n_iters):
    import torch
    g = binding.Graph(p.graph)
    g.set_option(binding.OPT_LOG_RATIO, 0)
    m = g.new_msgs()
    g.run_bp(torch.as_tensor(p.log_pot).cuda(), torch.as_tensor(p.evidence).cuda(), T, damping, n_iters, m)
    return m.cpu().numpy()


@pytest.mark.parametrize("seed", [0, 1])
def test_batch_per_member_parameters(gpu, seed):
    """pgm_run_bp_batch: every member with its own T (0, 0.5 or 1), damping (0, 0.3, 0.5)
    and iteration count (0..12) in one batched run; each member's messages equal the
    member run alone with its parameters, bitwise, and its beliefs match the oracle."""
    import torch
    members = _mixed_members()
    rng = np.random.default_rng(seed)
    n = len(members)
    Ts = rng.choice([0.0, 0.5, 1.0], n).astype(np.float32)
    ds = rng.choice([0.0, 0.3, 0.5], n).astype(np.float32)
    its = rng.integers(0, 13, n).astype(np.int32)
    its[0] = 0
    its[-1] = 12
    batch = W.union(members)
    gb = gpu.Graph([p.graph for p in members])
    lp = torch.as_tensor(batch.log_pot).cuda()
    ev = torch.as_tensor(batch.evidence).cuda()
    m = gb.new_msgs()
    gb.run_bp_batch(lp, ev, Ts, ds, its, m)
    mb = m.cpu().numpy()
    for i, p in enumerate(members):
        off = gb.member(i)
        seg = mb[off["es_off"]: off["es_off"] + off["n_edge_states"]]
        ref = _alone(gpu, p, float(Ts[i]), float(ds[i]), int(its[i]))
        assert np.array_equal(seg, ref), (p.name, Ts[i], ds[i], its[i])
        om, _ = oracle.run_bp(p.graph, p.log_pot, p.evidence, float(Ts[i]), float(ds[i]), int(its[i]))
        _, onb, _, _ = oracle.beliefs(p.graph, p.evidence, om)
        g1 = gpu.Graph(p.graph)
        nb = g1.beliefs(torch.as_tensor(p.evidence).cuda(), torch.as_tensor(seg).cuda(), True).cpu().numpy()
        assert_beliefs_close(nb, onb, what=f"{p.name} T={Ts[i]} d={ds[i]} it={its[i]}")


def test_batch_per_member_warm_start_and_errors(gpu):
    """Two calls continue where the first stopped (warm start per member); bad
    per-member values are rejected with the member named."""
    import torch
    members = _mixed_members()[:4]
    batch = W.union(members)
    gb = gpu.Graph([p.graph for p in members])
    lp = torch.as_tensor(batch.log_pot).cuda()
    ev = torch.as_tensor(batch.evidence).cuda()
    Ts = np.array([1.0, 0.0, 1.0, 0.0], np.float32)
    ds = np.full(4, 0.5, np.float32)
    a = gb.new_msgs()
    gb.run_bp_batch(lp, ev, Ts, ds, np.array([2, 3, 0, 5], np.int32), a)
    gb.run_bp_batch(lp, ev, Ts, ds, np.array([4, 2, 6, 1], np.int32), a)
    b = gb.new_msgs()
    gb.run_bp_batch(lp, ev, Ts, ds, np.array([6, 5, 6, 6], np.int32), b)
    # a member's iterations split over two calls equal one run of the sum (ping-pong
    # buffers hold the same values; results are bitwise equal)
    assert torch.equal(a, b)
    for bad_T, bad_d, bad_n, word in ((-1.0, 0.5, 3, "T[2]"), (1.0, 1.0, 3, "damping[2]"), (1.0, 0.5, -1, "n_iters[2]")):
        T2, d2, n2 = Ts.copy(), ds.copy(), np.array([1, 1, 1, 1], np.int32)
        T2[2], d2[2], n2[2] = bad_T, bad_d, bad_n
        with pytest.raises(gpu.PgmError) as ei:
            gb.run_bp_batch(lp, ev, T2, d2, n2, a)
        assert ei.value.status == -1 and word in str(ei.value)
