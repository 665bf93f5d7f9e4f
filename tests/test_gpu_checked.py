"""Checked mode on the GPU (PGM_OPT_CHECKED), on valid graphs only.

Every call first range-checks the graph's index arrays on the device; on valid graphs
the status word's PGM_FLAG_INDEX stays clear, pgm_checked_report finds nothing, and the
results are bitwise those of the unchecked calls. (The checks' response to bad entries is
tested on the host, tests/test_audit_cpu.py: no out-of-range index is handed to a GPU.)
"""
import numpy as np
import pytest

from paper_2202_04110_gb300 import workloads as W

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


def _problems():
    g_rand, lp, ev = W.random_graph(3, n_vars=30, max_K=4, n_pair=40, n_triple=5, n_or=4, n_and=4, sparse=True)
    return [W.ising_grid(40, 41, 0, T=1.0), W.potts_grid(30, 16, 1, T=1.0), W.rbm(100, 90, 2, T=0.0),
            W.deconvolution(3, n_img=2, T=0.0), W.Problem("random", g_rand, lp, ev, 1.0, 0.5, 10),
            W.pool_grid(12, 2, 1, 4, T=0.0)]


@pytest.mark.parametrize("idx", range(6))
def test_checked_mode_changes_nothing_on_valid_graphs(gpu, idx):
    import torch
    p = _problems()[idx]
    lp = torch.as_tensor(p.log_pot).cuda()
    ev = torch.as_tensor(p.evidence).cuda()
    out = []
    for checked in (0, 1):
        g = gpu.Graph(p.graph)
        g.set_option(gpu.OPT_CHECKED, checked)
        assert g.get_option(gpu.OPT_CHECKED) == checked
        m = g.new_msgs()
        g.run_bp(lp, ev, p.T, 0.5, 12, m)
        nb = g.beliefs(ev, m, True)
        dec = g.decode(ev, m)
        f = g.flags(clear=True)
        assert not f & gpu.FLAG_INDEX, (p.name, checked, f)
        assert g.checked_report()[0] == -1
        out.append((m.cpu().numpy(), nb.cpu().numpy(), dec.cpu().numpy()))
    for a, b in zip(out[0], out[1]):
        assert np.array_equal(a, b, equal_nan=True), p.name


def test_checked_mode_batch_and_gradient(gpu):
    import torch
    ms = [W.potts_grid(13, 4, 1, T=1.0), W.ising_grid(9, 11, 2, T=1.0), W.deconvolution(5, n_img=1, T=1.0)]
    batch = W.union(ms)
    lp = torch.as_tensor(batch.log_pot).cuda()
    ev = torch.as_tensor(batch.evidence).cuda()
    res = []
    for checked in (0, 1):
        g = gpu.Graph([p.graph for p in ms])
        g.set_option(gpu.OPT_CHECKED, checked)
        m = g.new_msgs()
        g.run_bp_batch(lp, ev, [1.0, 0.0, 1.0], [0.5, 0.5, 0.3], [5, 7, 3], m)
        gn = torch.as_tensor(np.random.default_rng(0).standard_normal(g.info["n_var_states"]).astype(np.float32)).cuda()
        d_lp, d_ev = g.grad(lp, ev, 1.0, 0.5, 6, 3, gn)
        assert not g.flags(clear=True) & gpu.FLAG_INDEX
        res.append((m.cpu().numpy(), d_ev.cpu().numpy()))
    assert np.array_equal(res[0][0], res[1][0])
    assert np.allclose(res[0][1], res[1][1], atol=1e-6)
