"""The allocation-free grid entry point (pgm_grid2_run_bp_noalloc) against pgm_run_bp.

Some callers cannot allocate device memory (a process whose device memory is owned and
budgeted by a host framework, or code that must not call cudaMalloc after start-up);
pgm_grid2_run_bp_noalloc serves them with its scratch in a static device array. This
file is collected last so that a run stopping at the first failure has already run
every other test; it must pass alone in a fresh process and after the other tests.
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


def _reference(binding, p, T, n_iters):
    import torch
    g = binding.Graph(p.graph)
    lp = torch.as_tensor(p.log_pot).cuda()
    ev = torch.as_tensor(p.evidence).cuda()
    m = g.new_msgs()
    g.run_bp(lp, ev, T, p.damping, n_iters, m)
    return g, lp, ev, m


@pytest.mark.parametrize("shape,T,n_iters", [((37, 53), 1.0, 25), ((64, 1), 0.0, 12), ((200, 300), 1.0, 31)])
def test_noalloc_matches_run_bp_twice(gpu, shape, T, n_iters):
    import torch
    rows, cols = shape
    p = W.ising_grid(rows, cols, seed=rows + cols, T=T, n_iters=n_iters)
    g, lp, ev, m_ref = _reference(gpu, p, T, n_iters)
    nb_ref = g.beliefs(ev, m_ref, True)
    for call in range(2):  # the second call reuses the static scratch the first one left behind
        m = torch.zeros_like(m_ref)
        gpu.grid2_run_bp_noalloc(rows, cols, lp, ev, T, p.damping, n_iters, m)
        torch.cuda.synchronize()
        np.testing.assert_allclose(m.cpu().numpy(), m_ref.cpu().numpy(), atol=1e-4, rtol=0,
                                   err_msg=f"messages, call {call}")
        nb = g.beliefs(ev, m, True)
        np.testing.assert_allclose(nb.cpu().numpy(), nb_ref.cpu().numpy(), atol=1e-4, rtol=0,
                                   err_msg=f"beliefs, call {call}")


def test_noalloc_warm_start_and_odd_counts(gpu):
    import torch
    p = W.ising_grid(21, 22, seed=3, T=1.0)
    g, lp, ev, m_ref = _reference(gpu, p, 1.0, 7)
    m = torch.zeros_like(m_ref)
    gpu.grid2_run_bp_noalloc(21, 22, lp, ev, 1.0, 0.5, 3, m)
    gpu.grid2_run_bp_noalloc(21, 22, lp, ev, 1.0, 0.5, 4, m)
    np.testing.assert_allclose(m.cpu().numpy(), m_ref.cpu().numpy(), atol=1e-4, rtol=0)


def test_noalloc_rejects_oversized_grid(gpu):
    import torch
    rows = cols = 700  # 4 * 978,600 factors + 2 * 490,000 variables > 4,194,304 floats
    ev = torch.zeros(2 * rows * cols, device="cuda")
    F = rows * (cols - 1) + (rows - 1) * cols
    lp = torch.zeros(4 * F, device="cuda")
    m = torch.zeros(4 * F, device="cuda")
    with pytest.raises(gpu.PgmError) as ei:
        gpu.grid2_run_bp_noalloc(rows, cols, lp, ev, 1.0, 0.5, 1, m)
    assert ei.value.status == -1
    assert "scratch" in str(ei.value)
