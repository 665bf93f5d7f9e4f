"""Serving loop (pgm_serve_*): continuous admission, each result equal to the request run
alone, the memory budget, errors reported per request, bounded waits."""
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


def _requests(n=40, seed=0):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        kind = i % 6
        T = float(rng.choice([0.0, 1.0]))
        it = int(rng.integers(10, 61))
        if kind == 0:
            p = W.ising_grid(int(rng.integers(8, 80)), int(rng.integers(8, 80)), i, T=T)
        elif kind == 1:
            p = W.potts_grid(int(rng.integers(8, 60)), 4, i, T=T)
        elif kind == 2:
            p = W.potts_grid(int(rng.integers(8, 40)), 16, i, T=T)
        elif kind == 3:
            p = W.rbm(int(rng.integers(20, 90)), int(rng.integers(20, 90)), i, T=T)
        elif kind == 4:
            p = W.deconvolution(i, n_img=1, T=T)
        else:
            g, lp, ev = W.random_graph(i, n_vars=30, max_K=4, n_pair=50, n_triple=4, n_or=3, n_and=3)
            p = W.Problem("random", g, lp, ev, T, 0.5, it)
        out.append((p, T, it))
    return out


def _alone(binding, p, T, it):
    import torch
    g = binding.Graph(p.graph)
    lp = torch.as_tensor(np.asarray(p.log_pot, np.float32)).cuda()
    ev = torch.as_tensor(np.asarray(p.evidence, np.float32)).cuda()
    m = g.new_msgs()
    g.run_bp(lp, ev, T, 0.5, it, m)
    return g.beliefs(ev, m, True).cpu().numpy(), g.decode(ev, m).cpu().numpy()


@pytest.mark.parametrize("slots", [4, 1])
def test_results_equal_alone(gpu, slots):
    reqs = _requests()
    srv = gpu.Server(memory_budget_bytes=48 << 20, max_in_flight=slots)
    ids = [srv.submit(p.graph, p.log_pot, p.evidence, T, 0.5, it) for p, T, it in reqs]
    results = [srv.wait(i, 120.0) for i in ids]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["peak_bytes"] <= 48 << 20
    # the latency splits into queue, host compile, admission wait and device work
    stages = st["queue_s"] + st["compile_s"] + st["admit_s"] + st["run_s"]
    total = sum(r[2] for r in results)
    assert st["compile_s"] > 0 and st["run_s"] > 0
    assert abs(stages - total) <= 1e-3 * len(reqs) + 1e-3 * total, (stages, total)
    for (p, T, it), (bel, dec, lat) in zip(reqs, results):
        b1, d1 = _alone(gpu, p, T, it)
        np.testing.assert_array_equal(bel, b1, err_msg=p.name)
        np.testing.assert_array_equal(dec, d1, err_msg=p.name)
        assert lat > 0


def test_served_results_match_oracle(gpu):
    srv = gpu.Server(memory_budget_bytes=1 << 30, max_in_flight=3)
    ps = [W.ising_grid(30, 41, 3, T=1.0), W.potts_grid(25, 4, 4, T=1.0), W.rbm(40, 30, 5, T=1.0)]
    ids = [srv.submit(p.graph, p.log_pot, p.evidence, 1.0, 0.5, 30) for p in ps]
    for p, i in zip(ps, ids):
        bel, dec, _ = srv.wait(i, 60.0)
        om, _ = oracle.run_bp(p.graph, p.log_pot, p.evidence, 1.0, 0.5, 30)
        _, onb, _, _ = oracle.beliefs(p.graph, p.evidence, om)
        assert_beliefs_close(bel, onb, what=p.name)
    srv.close()


def test_errors_are_per_request(gpu):
    srv = gpu.Server(memory_budget_bytes=1 << 20, max_in_flight=2)
    big = W.ising_grid(300, 300, 1)
    small = W.ising_grid(10, 10, 2)
    bad = W.FactorGraph(np.array([2, 2], np.int32), [W.EnumGroup(W.PAIR2_CFG.copy(), np.array([[0, 5]], np.int32))])
    i_big = srv.submit(big.graph, big.log_pot, big.evidence, 1.0, 0.5, 5)
    i_bad = srv.submit(bad, np.zeros(4, np.float32), np.zeros(4, np.float32), 1.0, 0.5, 5)
    i_ok = srv.submit(small.graph, small.log_pot, small.evidence, 1.0, 0.5, 5)
    with pytest.raises(gpu.PgmError) as ei:
        srv.wait(i_big, 60.0)
    assert ei.value.status == -2  # PGM_ENOMEM: alone above the budget
    with pytest.raises(gpu.PgmError) as ei:
        srv.wait(i_bad, 60.0)
    assert ei.value.status == -1  # PGM_EINVAL from the build
    assert srv.wait(i_ok, 60.0) is not None
    st = srv.stats()
    assert st["failed"] == 2 and st["completed"] == 1
    srv.close()


def test_bounded_wait_times_out(gpu):
    srv = gpu.Server(memory_budget_bytes=1 << 30, max_in_flight=1)
    p = W.ising_grid(400, 400, 1)
    i = srv.submit(p.graph, p.log_pot, p.evidence, 1.0, 0.5, 400)
    with pytest.raises(gpu.PgmError) as ei:
        srv.wait(i, 0.0)
    assert ei.value.status == -6  # PGM_ETIMEDOUT, the request keeps running
    assert srv.wait(i, 120.0) is not None
    srv.close()


def _alone_until(binding, p, T, it, tol, ck):
    import torch
    g = binding.Graph(p.graph)
    lp = torch.as_tensor(np.asarray(p.log_pot, np.float32)).cuda()
    ev = torch.as_tensor(np.asarray(p.evidence, np.float32)).cuda()
    m = g.new_msgs()
    done, _ = g.run_bp_until(lp, ev, T, 0.5, it, tol, ck, m)
    return g.beliefs(ev, m, True).cpu().numpy(), g.decode(ev, m).cpu().numpy(), done, g.info["n_edge_states"]


@pytest.mark.parametrize("slots", [4, 1])
def test_early_exit_requests_equal_alone(gpu, slots):
    """Requests with a residual tolerance (pgm_serve_submit_until) stop early; each result
    equals pgm_run_bp_until of the same request alone, and the server counts only the
    iterations run."""
    reqs = _requests(n=18, seed=3)
    tol, ck = 1e-4, 10
    srv = gpu.Server(memory_budget_bytes=48 << 20, max_in_flight=slots)
    ids = [srv.submit(p.graph, p.log_pot, p.evidence, T, 0.5, 4 * it, tol=tol, check_every=ck) for p, T, it in reqs]
    results = [srv.wait(i, 120.0) for i in ids]
    st = srv.stats()
    srv.close()
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["peak_bytes"] <= 48 << 20
    upd, full = 0, 0
    for (p, T, it), (bel, dec, lat) in zip(reqs, results):
        b1, d1, done, ES = _alone_until(gpu, p, T, 4 * it, tol, ck)
        np.testing.assert_array_equal(bel, b1, err_msg=p.name)
        np.testing.assert_array_equal(dec, d1, err_msg=p.name)
        upd += done * ES
        full += 4 * it * ES
    assert st["updates_done"] == upd
    assert upd < full  # some requests converged before their limit
    with pytest.raises(gpu.PgmError):
        srv2 = gpu.Server(memory_budget_bytes=1 << 20, max_in_flight=1)
        try:
            p = reqs[0][0]
            srv2.submit(p.graph, p.log_pot, p.evidence, 1.0, 0.5, 10, tol=1e-3, check_every=0)
        finally:
            srv2.close()


def test_large_factor_requests_equal_alone(gpu):
    """Requests with large listed-configuration factors (pool grids of 49 and 121 states:
    the block-form factor kernel, the warp variable pass and its belief residuals) served
    alongside Ising grids: each result equals the request run alone."""
    reqs = [(W.pool_grid(6, 3, 1, 31, T=0.0), 0.0, 20), (W.ising_grid(20, 25, 32), 1.0, 30),
            (W.pool_grid(4, 5, 2, 33, T=1.0), 1.0, 15), (W.pool_grid(5, 3, 1, 34, T=1.0, shared=False), 1.0, 12)]
    srv = gpu.Server(memory_budget_bytes=256 << 20, max_in_flight=3)
    ids = [srv.submit(p.graph, p.log_pot, p.evidence, T, 0.5, it) for p, T, it in reqs]
    results = [srv.wait(i, 120.0) for i in ids]
    srv.close()
    for (p, T, it), (bel, dec, _) in zip(reqs, results):
        b1, d1 = _alone(gpu, p, T, it)
        np.testing.assert_array_equal(bel, b1, err_msg=p.name)
        np.testing.assert_array_equal(dec, d1, err_msg=p.name)


@pytest.mark.parametrize("tol", [None, 1e-4])
def test_borrowed_requests_equal_copied(gpu, tol):
    """pgm_serve_submit_borrowed (no copies at submission) gives the results of the
    copying submissions, with and without an early exit; a borrowed request with a bad
    description fails on its own."""
    reqs = _requests(n=12, seed=5)
    out = []
    for borrow in (False, True):
        srv = gpu.Server(memory_budget_bytes=64 << 20, max_in_flight=4)
        keep = [(np.asarray(p.log_pot, np.float32), np.asarray(p.evidence, np.float32)) for p, _, _ in reqs]
        ids = [srv.submit(p.graph, lp, ev, T, 0.5, it, tol=tol, borrow=borrow)
               for (p, T, it), (lp, ev) in zip(reqs, keep)]
        out.append([srv.wait(i, 120.0) for i in ids])
        srv.close()
    for (b0, d0, _), (b1, d1, _) in zip(out[0], out[1]):
        np.testing.assert_array_equal(b0, b1)
        np.testing.assert_array_equal(d0, d1)
    srv = gpu.Server(memory_budget_bytes=1 << 20, max_in_flight=1)
    bad = W.FactorGraph(np.array([2, 2], np.int32), [W.EnumGroup(W.PAIR2_CFG.copy(), np.array([[0, 5]], np.int32))])
    i_bad = srv.submit(bad, np.zeros(4, np.float32), np.zeros(4, np.float32), 1.0, 0.5, 5, borrow=True)
    with pytest.raises(gpu.PgmError) as ei:
        srv.wait(i_bad, 60.0)
    assert ei.value.status == -1
    srv.close()
