"""Many evidence / potential sets on one graph (pgm_run_bp_multi).

The samples of a binary grid run together (sample index innermost); each sample's
messages must be bitwise those of pgm_run_bp on that sample alone (the per-sample
arithmetic is the same), and match the FP64 oracle. Other graphs run sample by sample.
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


def _samples(p, S, seed, per_sample_pot=False):
    """S evidence sets (fields h ~ N(0, 1) as [-h, h]); optionally S coupling sets."""
    rng = np.random.default_rng(seed)
    V = p.graph.n_vars
    h = rng.standard_normal((S, V))
    ev = np.stack([-h, h], axis=2).reshape(S, -1).astype(np.float32)
    if per_sample_pot:
        F = p.log_pot.size // 4
        J = rng.uniform(-1.0, 1.0, (S, F))
        lp = np.stack([J, -J, -J, J], axis=2).reshape(S, -1).astype(np.float32)
    else:
        lp = p.log_pot.astype(np.float32)
    return lp, ev


def _multi(gpu, graph, lp, ev, T, n_iters, msgs0=None):
    import torch
    g = gpu.Graph(graph)
    lpt = torch.as_tensor(lp).cuda()
    evt = torch.as_tensor(ev).cuda()
    S = ev.shape[0]
    ES = g.info["n_edge_states"]
    m = torch.zeros(S, ES, device="cuda") if msgs0 is None else torch.as_tensor(msgs0).cuda().clone()
    g.run_bp_multi(lpt, evt, T, 0.5, n_iters, m)
    return g, m.cpu().numpy()


def _single(gpu, graph, lp, ev, T, n_iters, msgs0=None):
    import torch
    g = gpu.Graph(graph)
    out = []
    for s in range(ev.shape[0]):
        lps = torch.as_tensor(lp[s] if lp.ndim == 2 else lp).cuda()
        evs = torch.as_tensor(ev[s]).cuda()
        m = g.new_msgs() if msgs0 is None else torch.as_tensor(msgs0[s]).cuda().clone()
        g.run_bp(lps, evs, T, 0.5, n_iters, m)
        out.append(m.cpu().numpy())
    return np.stack(out)


def _same(a, b):
    both_nan = np.isnan(a) & np.isnan(b)
    assert np.array_equal(a[~both_nan], b[~both_nan])


@pytest.mark.parametrize("T", [1.0, 0.0])
@pytest.mark.parametrize("per_sample_pot", [False, True])
def test_samples_equal_single_runs(gpu, T, per_sample_pot):
    p = W.ising_grid(37, 53, 11)
    lp, ev = _samples(p, 5, 7, per_sample_pot)
    g, mm = _multi(gpu, p.graph, lp, ev, T, 30)
    assert g.get_option(gpu.OPT_LOG_RATIO) == 4  # the joint path
    ms = _single(gpu, p.graph, lp, ev, T, 30)
    _same(mm, ms)


def test_samples_match_oracle(gpu):
    p = W.ising_grid(24, 31, 3)
    lp, ev = _samples(p, 4, 9, per_sample_pot=True)
    _, mm = _multi(gpu, p.graph, lp, ev, 1.0, 40)
    for s in (0, 3):
        om, _ = oracle.run_bp(p.graph, lp[s], ev[s], 1.0, 0.5, 40)
        _, onb, _, _ = oracle.beliefs(p.graph, ev[s], om)
        _, gnb, _, _ = oracle.beliefs(p.graph, ev[s], mm[s].astype(np.float64))
        assert_beliefs_close(gnb, onb, what=f"sample {s}")
        np.testing.assert_allclose(mm[s], om, atol=1e-4, rtol=0)


def test_hard_evidence_and_warm_start(gpu):
    p = W.ising_grid(16, 21, 5)
    lp, ev = _samples(p, 3, 4)
    ev[1, 2 * 40: 2 * 40 + 2] = -np.inf  # sample 1: variable 40 contradictory
    ev[2, 2 * 7] = -np.inf              # sample 2: variable 7 forced to state 1
    rng = np.random.default_rng(8)
    m0 = rng.normal(0.0, 1.0, (3, oracle.sizes(p.graph)["ES"])).astype(np.float32)
    for msgs0 in (None, m0):
        for T in (1.0, 0.0):
            _, mm = _multi(gpu, p.graph, lp, ev, T, 12, msgs0)
            ms = _single(gpu, p.graph, lp, ev, T, 12, msgs0)
            _same(mm, ms)


def test_growing_sample_count_and_short_runs(gpu):
    import torch
    p = W.ising_grid(9, 13, 2)
    g = gpu.Graph(p.graph)
    ES = g.info["n_edge_states"]
    for S, it in ((2, 10), (6, 10), (3, 2)):  # buffers grow; 2 iterations: sample by sample
        lp, ev = _samples(p, S, S)
        m = torch.zeros(S, ES, device="cuda")
        g.run_bp_multi(torch.as_tensor(lp).cuda(), torch.as_tensor(ev).cuda(), 1.0, 0.5, it, m)
        _same(m.cpu().numpy(), _single(gpu, p.graph, lp, ev, 1.0, it))
    with pytest.raises(gpu.PgmError):
        gpu.check(gpu.load_library().pgm_run_bp_multi(g.handle, 0, None, 0, None, 1.0, 0.5, 1, None, None))


def _other(name):
    if name == "potts4":
        return W.potts_grid(12, 4, 1, T=1.0)
    if name == "potts16":
        return W.potts_grid(10, 16, 2, T=1.0)
    if name == "rbm":  # visible variables of degree 150: block-per-variable pass, exact sums
        return W.rbm(40, 150, 3)
    if name == "deconv":  # OR / AND factors, degree up to 200
        return W.deconvolution(4, n_img=1, n_iters=10)
    if name == "pool":  # 49-state variables (warp pass, residuals), block-form factors
        return W.pool_grid(6, 3, 1, 5, T=1.0)
    g, lp, ev = W.random_graph(9, n_vars=14, max_K=4, n_pair=16, n_triple=3, n_or=2, n_and=2)
    return W.Problem("random", g, lp, ev, 1.0, 0.5, 10)


@pytest.mark.parametrize("T", [1.0, 0.0])
@pytest.mark.parametrize("per_sample_pot", [False, True])
@pytest.mark.parametrize("name", ["potts4", "potts16", "rbm", "deconv", "pool", "random"])
def test_other_graphs_samples_side_by_side(gpu, name, per_sample_pot, T):
    """Graphs without the joint log-ratio path run their samples as the second grid
    dimension of every edge-state launch; each sample's messages are bitwise those of
    pgm_run_bp on that sample alone."""
    p = _other(name)
    S = 5
    rng = np.random.default_rng(3)
    ev = (np.asarray(p.evidence, np.float32)[None, :] +
          rng.standard_normal((S, p.graph.n_var_states)).astype(np.float32))
    if per_sample_pot and p.graph.n_potentials > 0:
        lp = (np.asarray(p.log_pot, np.float32)[None, :] +
              0.3 * rng.standard_normal((S, p.graph.n_potentials)).astype(np.float32))
    else:
        lp = np.asarray(p.log_pot, np.float32)
    for it in (7, 8):  # odd and even: the result in the scratch buffer or in place
        _, mm = _multi(gpu, p.graph, lp, ev, T, it)
        _same(mm, _single(gpu, p.graph, lp, ev, T, it))


def test_chunks_of_samples(gpu):
    """Per-sample exchange arrays of ~21 MB: half the L2 holds 2 samples, so 3 samples run
    as a chunk of 2 and a chunk of 1 (offsets into every sample-major array)."""
    p = W.ising_grid(820, 820, 6)
    lp, ev = _samples(p, 3, 12, per_sample_pot=True)
    _, mm = _multi(gpu, p.graph, lp, ev, 1.0, 6)
    _same(mm, _single(gpu, p.graph, lp, ev, 1.0, 6))


def _gumbel(rng, shape):
    return (-np.log(-np.log(rng.uniform(1e-12, 1.0, shape)))).astype(np.float32)


@pytest.mark.parametrize("which", ["ising", "deconvolution"])
def test_perturb_and_max_product_samples(gpu, which):
    """pgm_pmp_sample: each sample is the MAP decode of max-product on the model with
    Gumbel-perturbed evidence; checked against the oracle run on the same perturbed
    evidence (decodes equal except at oracle ties), and against pgm_run_bp + decode."""
    import torch
    from tests._parity import assert_decode_ok
    if which == "ising":
        p = W.ising_grid(16, 21, 5)  # joint path
        n_it = 15
    else:
        p = W.deconvolution(3, n_img=2, n_iters=8)  # logical factors: sample by sample
        n_it = 8
    S = 4
    rng = np.random.default_rng(21)
    noise = _gumbel(rng, (S, p.graph.n_var_states))
    g = gpu.Graph(p.graph)
    lpt = torch.as_tensor(p.log_pot.astype(np.float32)).cuda()
    evt = torch.as_tensor(p.evidence.astype(np.float32)).cuda()
    samples, _ = g.pmp_sample(lpt, evt, torch.as_tensor(noise).cuda(), 0.5, n_it)
    samples = samples.cpu().numpy()
    assert len({tuple(x) for x in samples}) > 1  # the perturbations change the samples
    for s in range(S):
        pev = p.evidence.astype(np.float32) + noise[s]
        om, _ = oracle.run_bp(p.graph, p.log_pot, pev, 0.0, 0.5, n_it)
        _, onb, _, _ = oracle.beliefs(p.graph, pev, om)
        assert_decode_ok(samples[s], onb, p.graph.num_states, what=f"{which} sample {s}")
        m = g.new_msgs()
        pevt = torch.as_tensor(pev).cuda()
        g.run_bp(lpt, pevt, 0.0, 0.5, n_it, m)
        assert np.array_equal(g.decode(pevt, m).cpu().numpy(), samples[s])
