"""Runs with an early exit (pgm_run_bp_until).

The run stops after the first checked iteration whose residual max |m_t - m_{t-1}| is
<= tol. The reported residual is recomputed here from an independent replay (t - 1
iterations, a copy, one more iteration); the messages equal those of the same
iterations run with pgm_run_bp, and track the FP64 oracle.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2202_04110_gb300 import workloads as W
from tests._parity import assert_beliefs_close

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


def test_early_exit_residual_and_messages(gpu):
    p = W.potts_grid(20, 4, 2, T=1.0)  # edge-state iterations: chunking changes nothing
    g = gpu.Graph(p.graph)
    lp, ev = _t(p.log_pot), _t(p.evidence)
    m = g.new_msgs()
    done, res = g.run_bp_until(lp, ev, 1.0, 0.5, 400, 1e-5, 10, m)
    assert done % 10 == 0 and 10 <= done < 400 and 0.0 <= res <= 1e-5
    # the residual of the last checked iteration, recomputed
    r = g.new_msgs()
    g.run_bp(lp, ev, 1.0, 0.5, done - 1, r)
    prev = r.cpu().numpy()
    g.run_bp(lp, ev, 1.0, 0.5, 1, r)
    assert np.array_equal(r.cpu().numpy(), m.cpu().numpy())
    d = np.abs(r.cpu().numpy().astype(np.float64) - prev)
    assert np.float32(d.max()) == np.float32(res)
    # the previous check had not converged
    if done == 10:
        return
    q = g.new_msgs()
    g.run_bp(lp, ev, 1.0, 0.5, done - 11, q)
    prev = q.cpu().numpy()
    g.run_bp(lp, ev, 1.0, 0.5, 1, q)
    assert np.abs(q.cpu().numpy() - prev).max() > 1e-5


def test_early_exit_log_ratio_graph_tracks_oracle(gpu):
    p = W.ising_grid(40, 50, 9, T=1.0)
    g = gpu.Graph(p.graph)
    m = g.new_msgs()
    done, res = g.run_bp_until(_t(p.log_pot), _t(p.evidence), 1.0, 0.5, 300, 1e-6, 25, m)
    assert done < 300 and res <= 1e-6
    om, _ = oracle.run_bp(p.graph, p.log_pot, p.evidence, 1.0, 0.5, done)
    _, onb, _, _ = oracle.beliefs(p.graph, p.evidence, om)
    nb = g.beliefs(_t(p.evidence), m, True).cpu().numpy()
    assert_beliefs_close(nb, onb, what=f"ising after {done} iterations")


def test_no_convergence_and_arguments(gpu):
    p = W.ising_grid(12, 12, 4, T=0.0)
    g = gpu.Graph(p.graph)
    lp, ev = _t(p.log_pot), _t(p.evidence)
    m = g.new_msgs()
    done, res = g.run_bp_until(lp, ev, 0.0, 0.5, 37, 0.0, 8, m)  # tol 0: runs to the end unless exact
    assert done == 37 or res == 0.0
    m = g.new_msgs()
    assert g.run_bp_until(lp, ev, 1.0, 0.5, 0, 1e-3, 5, m)[0] == 0
    assert math.isnan(g.run_bp_until(lp, ev, 1.0, 0.5, 0, 1e-3, 5, m)[1])
    for bad in ((1e-3, 0), (-1.0, 5), (float("nan"), 5)):
        with pytest.raises(gpu.PgmError):
            g.run_bp_until(lp, ev, 1.0, 0.5, 10, bad[0], bad[1], m)


@pytest.mark.parametrize("which", ["potts", "ising"])
def test_device_loop_equals_host_checked(gpu, which):
    """With CUDA graphs on, the full chunks run in a conditional while node (no host round
    trip per chunk); with them off, the host checks each chunk. Same iterations, same
    residual, bitwise the same messages; also when max_iters leaves a shorter last chunk
    and when the loop runs to its limit."""
    p = W.potts_grid(20, 4, 2, T=1.0) if which == "potts" else W.ising_grid(40, 50, 9, T=1.0)
    lp, ev = _t(p.log_pot), _t(p.evidence)
    for max_iters, tol, ck in ((400, 1e-5, 10), (47, 1e-5, 10), (33, 0.0, 8), (7, 1e-3, 10)):
        out = []
        for graphs in (1, 0):
            g = gpu.Graph(p.graph)
            g.set_option(gpu.OPT_CUDA_GRAPH, graphs)
            m = g.new_msgs()
            done, res = g.run_bp_until(lp, ev, 1.0, 0.5, max_iters, tol, ck, m)
            m2 = g.new_msgs()  # a second call replays the cached graph
            done2, res2 = g.run_bp_until(lp, ev, 1.0, 0.5, max_iters, tol, ck, m2)
            assert (done2, np.float32(res2)) == (done, np.float32(res))
            assert np.array_equal(m.cpu().numpy(), m2.cpu().numpy())
            out.append((done, np.float32(res), m.cpu().numpy()))
        assert out[0][0] == out[1][0] and out[0][1] == out[1][1], (which, max_iters, out[0][:2], out[1][:2])
        assert np.array_equal(out[0][2], out[1][2])


def _members():
    ms = [W.ising_grid(20, 30, 1, T=1.0), W.potts_grid(16, 4, 2, T=1.0), W.ising_grid(9, 9, 3, T=1.0),
          W.potts_grid(12, 8, 4, T=1.0), W.rbm(12, 9, 5, T=1.0)]
    g, lp, ev = W.random_graph(6, n_vars=12, max_K=3, n_pair=14, n_triple=2)
    ms.append(W.Problem("random", g, lp, ev, 1.0, 0.5, 10))
    ms.append(W.pool_grid(5, 3, 1, 8, T=1.0))  # block-form factors, warp variable pass
    return ms


@pytest.mark.parametrize("graphs", [1, 0])
@pytest.mark.parametrize("case", [(300, 1e-5, 10), (57, 1e-4, 8), (40, 0.0, 10)])
def test_members_stop_on_their_own(gpu, graphs, case):
    """pgm_run_bp_until_members on a batch: every member's iterations, residual and
    messages equal pgm_run_bp_until of that member alone (log-ratio iterations off), so
    a stopped member keeps its messages while the others go on."""
    import torch
    max_iters, tol, ck = case
    ms = _members()
    T = 1.0
    bg = gpu.Graph([p.graph for p in ms])
    bg.set_option(gpu.OPT_CUDA_GRAPH, graphs)
    lp = _t(np.concatenate([p.log_pot for p in ms]))
    ev = _t(np.concatenate([p.evidence for p in ms]))
    for rep in range(2):  # the second call replays the cached graph
        m = bg.new_msgs()
        done, res = bg.run_bp_until_members(lp, ev, T, 0.5, max_iters, tol, ck, m)
        mm = m.cpu().numpy()
        for k, p in enumerate(ms):
            g = gpu.Graph(p.graph)
            g.set_option(gpu.OPT_LOG_RATIO, 0)
            a = g.new_msgs()
            d1, r1 = g.run_bp_until(_t(p.log_pot), _t(p.evidence), T, 0.5, max_iters, tol, ck, a)
            info = bg.member(k)
            assert (done[k], np.float32(res[k])) == (d1, np.float32(r1)), (k, p.name, done[k], res[k], d1, r1)
            assert np.array_equal(mm[info["es_off"]:info["es_off"] + info["n_edge_states"]], a.cpu().numpy()), p.name
    if tol > 0 and max_iters == 300:
        assert len(set(done.tolist())) > 1  # members stopped at different iterations
    # a normal run afterwards skips nothing
    m1 = bg.new_msgs()
    bg.run_bp(lp, ev, T, 0.5, 7, m1)
    for k, p in enumerate(ms):
        g = gpu.Graph(p.graph)
        g.set_option(gpu.OPT_LOG_RATIO, 0)  # the batch is not a binary pairwise graph
        a = g.new_msgs()
        g.run_bp(_t(p.log_pot), _t(p.evidence), T, 0.5, 7, a)
        info = bg.member(k)
        assert np.array_equal(m1.cpu().numpy()[info["es_off"]:info["es_off"] + info["n_edge_states"]], a.cpu().numpy())


def test_members_arguments(gpu):
    ms = _members()[:2]
    bg = gpu.Graph([p.graph for p in ms])
    lp = _t(np.concatenate([p.log_pot for p in ms]))
    ev = _t(np.concatenate([p.evidence for p in ms]))
    m = bg.new_msgs()
    done, res = bg.run_bp_until_members(lp, ev, 1.0, 0.5, 0, 1e-3, 5, m)
    assert (done == 0).all() and np.isnan(res).all()
    for bad in ((1e-3, 0), (-1.0, 5), (float("nan"), 5)):
        with pytest.raises(gpu.PgmError):
            bg.run_bp_until_members(lp, ev, 1.0, 0.5, 10, bad[0], bad[1], m)
