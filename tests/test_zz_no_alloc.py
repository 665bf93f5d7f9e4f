"""The allocation-free grid entry point (pgm_grid2_run_bp_noalloc) against pgm_run_bp and
the FP64 oracle.

Some callers cannot allocate device memory (a process whose device memory is owned and
budgeted by a host framework, or code that must not call cudaMalloc after start-up);
pgm_grid2_run_bp_noalloc serves them with its scratch in a static device array. This
file is collected last so that a run stopping at the first failure has already run
every other test; it must pass alone in a fresh process and after the other tests.
"""
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


def _reference(binding, p, T, n_iters):
    import torch
    g = binding.Graph(p.graph)
    lp = torch.as_tensor(p.log_pot).cuda()
    ev = torch.as_tensor(p.evidence).cuda()
    m = g.new_msgs()
    g.run_bp(lp, ev, T, p.damping, n_iters, m)
    return g, lp, ev, m


def _oracle_nb(p, T, n_iters):
    om, ofl = oracle.run_bp(p.graph, p.log_pot, p.evidence, T, p.damping, n_iters)
    _, onb, _, ofl2 = oracle.beliefs(p.graph, p.evidence, om)
    return onb, ofl | ofl2


@pytest.mark.parametrize("shape,T,n_iters", [((37, 53), 1.0, 25), ((64, 1), 0.0, 12), ((200, 300), 1.0, 31)])
def test_noalloc_matches_run_bp_twice(gpu, shape, T, n_iters):
    import torch
    rows, cols = shape
    p = W.ising_grid(rows, cols, seed=rows + cols, T=T, n_iters=n_iters)
    g, lp, ev, m_ref = _reference(gpu, p, T, n_iters)
    nb_ref = g.beliefs(ev, m_ref, True)
    onb, _ = _oracle_nb(p, T, n_iters)
    for call in range(2):  # the second call reuses the static scratch the first one left behind
        m = torch.zeros_like(m_ref)
        gpu.grid2_run_bp_noalloc(rows, cols, lp, ev, T, p.damping, n_iters, m)
        torch.cuda.synchronize()
        np.testing.assert_allclose(m.cpu().numpy(), m_ref.cpu().numpy(), atol=1e-4, rtol=0,
                                   err_msg=f"messages, call {call}")
        nb = g.beliefs(ev, m, True).cpu().numpy()
        np.testing.assert_allclose(nb, nb_ref.cpu().numpy(), atol=1e-4, rtol=0, err_msg=f"beliefs, call {call}")
        assert_beliefs_close(nb, onb, what=f"noalloc vs oracle, call {call}")
        assert gpu.grid2_noalloc_flags(clear=True) == 0


def _hard_grid(rows, cols, seed, scale):
    """An Ising grid with couplings scale * U[-1, 1] and fields scale * N(0, 1), a fifth
    of the cells clamped by hard evidence (one state at -inf). With scale > 128 the
    stored messages exceed the kernels' threshold for b - m, so every factor takes its
    variable-to-factor values from explicit leave-one-out sums."""
    p = W.ising_grid(rows, cols, seed=seed, T=1.0)
    rng = np.random.default_rng(seed + 1)
    lp = (p.log_pot * scale).astype(np.float32)
    ev = (p.evidence * scale).reshape(-1, 2)
    clamp = rng.random(rows * cols) < 0.2
    state = rng.integers(0, 2, rows * cols)
    ev[clamp, 1 - state[clamp]] = -np.inf
    p.log_pot = lp
    p.evidence = ev.astype(np.float32).ravel()
    return p


@pytest.mark.parametrize("T", [0.0, 1.0])
@pytest.mark.parametrize("scale", [1.0, 300.0])
def test_noalloc_hard_evidence_and_large_messages(gpu, T, scale):
    """-inf evidence on a fifth of the cells; with scale 300 the messages exceed 128, the
    recompute branch of the factor kernel. Against the oracle and pgm_run_bp, twice. At
    scale 300 the raw beliefs reach 2,500, and a normalised log-belief b - LSE(b) formed
    from them in FP32 is exact only to their ulp (2.4e-4 at 2,500), so there the tolerance
    is 1e-4 plus two FP32 ulps of the raw belief rather than of the normalised value. Each
    CUDA path is held to that bound against the oracle; the two paths round in different
    orders, so against each other they are held to the sum of their two bounds."""
    import torch
    rows, cols, n_iters = 29, 31, 20
    p = _hard_grid(rows, cols, 11, scale)
    g, lp, ev, m_ref = _reference(gpu, p, T, n_iters)
    nb_ref = g.beliefs(ev, m_ref, True).cpu().numpy()
    om, ofl = oracle.run_bp(p.graph, p.log_pot, p.evidence, T, 0.5, n_iters)
    braw, onb, _, ofl2 = oracle.beliefs(p.graph, p.evidence, om)
    ofl |= ofl2
    fin = np.isfinite(braw)
    rtol_raw = np.where(fin, 2.0 ** -21 * np.abs(np.where(fin, braw, 0.0)), 0.0)

    fin_o = np.isfinite(onb)
    tol_o = 1e-4 + 2.0 ** -22 * np.abs(np.where(fin_o, onb, 0.0)) + rtol_raw

    def close(a, ref, tol, what):
        a = np.asarray(a, np.float64)
        assert (np.isneginf(a) == np.isneginf(ref)).all(), what
        f = np.isfinite(ref)
        err = np.abs(a[f] - ref[f])
        assert (err <= tol[f]).all(), f"{what}: max excess {np.max(err - tol[f]):.3e}"

    close(nb_ref, onb, tol_o, "pgm_run_bp vs oracle")
    for call in range(2):
        m = torch.zeros_like(m_ref)
        gpu.grid2_run_bp_noalloc(rows, cols, lp, ev, T, 0.5, n_iters, m)
        nb = g.beliefs(ev, m, True).cpu().numpy()
        close(nb, onb, tol_o, f"noalloc vs oracle, call {call}")
        close(nb, np.asarray(nb_ref, np.float64), 2.0 * tol_o, f"noalloc vs pgm_run_bp, call {call}")
        assert gpu.grid2_noalloc_flags(clear=True) == (ofl & oracle.FLAG_CONTRADICTION), call


def test_noalloc_contradiction_flag(gpu):
    """A 3 x 3 grid whose centre is forced to 0 by its upper neighbour and to 1 by its left
    neighbour (hard evidence and hard equality couplings): the centre's message towards its
    right neighbour has both states at -inf, a contradiction that pgm_run_bp, the oracle and
    the allocation-free call all report."""
    import torch
    p = W.ising_grid(3, 3, seed=0, T=1.0)
    pairs = p.graph.enum_groups[0].vars
    lp = np.tile(np.array([0.0, 0.3, -0.2, 0.1], np.float32), (pairs.shape[0], 1))
    eq = np.array([0.0, -np.inf, -np.inf, 0.0], np.float32)
    for f, (a, b) in enumerate(pairs):
        if (a, b) in ((1, 4), (3, 4)):
            lp[f] = eq
    ev = np.zeros((9, 2), np.float32)
    ev[1] = [0.0, -np.inf]   # (0, 1) forced to 0
    ev[3] = [-np.inf, 0.0]   # (1, 0) forced to 1
    p.log_pot, p.evidence = lp.ravel(), ev.ravel()
    g, lp_d, ev_d, m_ref = _reference(gpu, p, 1.0, 6)
    assert g.flags(clear=True) & gpu.FLAG_CONTRADICTION
    onb, ofl = _oracle_nb(p, 1.0, 6)
    assert ofl & oracle.FLAG_CONTRADICTION
    gpu.grid2_noalloc_flags(clear=True)
    m = torch.zeros_like(m_ref)
    gpu.grid2_run_bp_noalloc(3, 3, lp_d, ev_d, 1.0, 0.5, 6, m)
    assert gpu.grid2_noalloc_flags() & gpu.FLAG_CONTRADICTION
    np.testing.assert_array_equal(np.isneginf(m.cpu().numpy()), np.isneginf(m_ref.cpu().numpy()))
    fin = np.isfinite(m_ref.cpu().numpy())
    np.testing.assert_allclose(m.cpu().numpy()[fin], m_ref.cpu().numpy()[fin], atol=1e-4, rtol=0)
    # the next call starts from a clear status word
    p2 = W.ising_grid(3, 3, seed=1, T=1.0)
    gpu.grid2_run_bp_noalloc(3, 3, torch.as_tensor(p2.log_pot).cuda(), torch.as_tensor(p2.evidence).cuda(),
                             1.0, 0.5, 6, torch.zeros_like(m_ref))
    assert gpu.grid2_noalloc_flags(clear=True) == 0


def test_noalloc_warm_start_and_odd_counts(gpu):
    import torch
    p = W.ising_grid(21, 22, seed=3, T=1.0)
    g, lp, ev, m_ref = _reference(gpu, p, 1.0, 7)
    m = torch.zeros_like(m_ref)
    gpu.grid2_run_bp_noalloc(21, 22, lp, ev, 1.0, 0.5, 3, m)
    gpu.grid2_run_bp_noalloc(21, 22, lp, ev, 1.0, 0.5, 4, m)
    np.testing.assert_allclose(m.cpu().numpy(), m_ref.cpu().numpy(), atol=1e-4, rtol=0)


def test_noalloc_size_limit(gpu):
    """4 * (2 r c - r - c) + 2 r c <= 4,194,304 floats: 648 x 648 (4,193,856) runs and
    matches pgm_run_bp; 649 x 649 (4,206,818) is rejected."""
    import torch
    p = W.ising_grid(648, 648, seed=5, T=1.0, n_iters=4)
    g, lp, ev, m_ref = _reference(gpu, p, 1.0, 4)
    m = torch.zeros_like(m_ref)
    gpu.grid2_run_bp_noalloc(648, 648, lp, ev, 1.0, 0.5, 4, m)
    np.testing.assert_allclose(m.cpu().numpy(), m_ref.cpu().numpy(), atol=1e-4, rtol=0)
    rows = cols = 649
    F = rows * (cols - 1) + (rows - 1) * cols
    ev = torch.zeros(2 * rows * cols, device="cuda")
    lp = torch.zeros(4 * F, device="cuda")
    m = torch.zeros(4 * F, device="cuda")
    with pytest.raises(gpu.PgmError) as ei:
        gpu.grid2_run_bp_noalloc(rows, cols, lp, ev, 1.0, 0.5, 1, m)
    assert ei.value.status == -1
    assert "scratch" in str(ei.value)
