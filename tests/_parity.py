"""Comparison helpers for GPU-vs-oracle parity (test code only)."""
import numpy as np

# Normalised log-beliefs (b - LSE_1(b)) of the FP32 GPU path must agree with the FP64
# oracle to 1e-4 absolute after the same iteration count; MAP decodes must be equal
# except where the oracle's two best states are within 1e-6 (several answers correct).
ATOL = 1e-4
# Two FP32 ulps of the value itself: a log-belief of magnitude above ~840 cannot be
# represented in FP32 to 1e-4 absolute (one ulp of 1024 is 1.2e-4).
RTOL = 2.0 ** -22
TIE = 1e-6


def assert_beliefs_close(gpu, ora, atol=ATOL, rtol=RTOL, what=""):
    g = np.asarray(gpu, np.float64)
    o = np.asarray(ora, np.float64)
    assert g.shape == o.shape, (g.shape, o.shape)
    assert not np.isnan(g).any(), f"{what}: NaN in GPU beliefs"
    ninf_g, ninf_o = np.isneginf(g), np.isneginf(o)
    assert (ninf_g == ninf_o).all(), f"{what}: -inf pattern differs at {np.flatnonzero(ninf_g != ninf_o)[:10]}"
    fin = ~ninf_o
    if fin.any():
        err = np.abs(g[fin] - o[fin])
        tol = atol + rtol * np.abs(o[fin])
        worst = int(np.argmax(err - tol))
        assert (err <= tol).all(), (f"{what}: |gpu - oracle| = {err[worst]:.3e} at {np.flatnonzero(fin)[worst]} "
                                    f"(oracle {o[fin][worst]:.6g}, tolerance {tol[worst]:.3e})")
        return float(err.max())
    return 0.0


def assert_decode_ok(gpu_dec, ora_nb, num_states, tie=TIE, what=""):
    """GPU decode must be the oracle's argmax, or within `tie` of the oracle's best."""
    dec = np.asarray(gpu_dec)
    nb = np.asarray(ora_nb, np.float64)
    vs = np.concatenate([[0], np.cumsum(num_states)])
    bad = []
    for v in range(len(num_states)):
        b = nb[vs[v]:vs[v + 1]]
        d = int(dec[v])
        if not (0 <= d < len(b)):
            bad.append(v)
            continue
        if b[d] < b.max() - tie:
            bad.append(v)
    assert not bad, f"{what}: decode differs at variables {bad[:10]} (of {len(bad)})"


def oracle_envelope(oracle, graph, log_pot, evidence, T, damping, n_iters, k=2, rel=1e-6, seed=12345):
    """The oracle's normalised log-beliefs and decode, plus their spread over an ensemble
    of nearby FP64 runs: one that rounds its messages to FP32 after every iteration
    (the storage model of any FP32-message implementation) and `k` whose log-potentials
    and evidence are multiplied by (1 + rel * N(0,1)) (about 8 FP32 ulps). Max-product
    and long loopy runs amplify such changes far beyond 1e-4; the spread measures how far
    an FP32 evaluation can land from the FP64 result."""
    rng = np.random.default_rng(seed)
    m0, fl = oracle.run_bp(graph, log_pot, evidence, T, damping, n_iters)
    _, nb0, dec0, fl2 = oracle.beliefs(graph, evidence, m0)
    spread = np.zeros_like(nb0)
    unstable = np.zeros(dec0.shape, bool)
    members = [(log_pot, evidence, True)]
    for _ in range(k):
        lp = np.asarray(log_pot, np.float64) * (1 + rel * rng.standard_normal(np.size(log_pot)))
        ev = np.asarray(evidence, np.float64) * (1 + rel * rng.standard_normal(np.size(evidence)))
        members.append((lp, ev, False))
    for lp, ev, r32 in members:
        m1, _ = oracle.run_bp(graph, lp, ev, T, damping, n_iters, round_f32=r32)
        _, nb1, dec1, _ = oracle.beliefs(graph, evidence, m1)
        with np.errstate(invalid="ignore"):
            d = np.abs(nb1 - nb0)
        d[np.isneginf(nb0) & np.isneginf(nb1)] = 0.0
        spread = np.maximum(spread, np.nan_to_num(d, nan=np.inf, posinf=np.inf))
        unstable |= dec1 != dec0
    return nb0, dec0, spread, unstable, fl | fl2


def assert_within_envelope(gpu_nb, gpu_dec, nb0, spread, unstable, num_states, atol=ATOL,
                           rtol=1e-6, factor=3.0, tie=TIE, what=""):
    """|gpu - oracle| <= atol + rtol |oracle| + factor * spread, per entry; decodes equal
    except where the perturbed oracle runs disagree among themselves or at ties."""
    g = np.asarray(gpu_nb, np.float64)
    assert not np.isnan(g).any(), f"{what}: NaN in GPU beliefs"
    both_ninf = np.isneginf(g) & np.isneginf(nb0)
    tol = atol + rtol * np.abs(np.where(np.isfinite(nb0), nb0, 0.0)) + factor * spread
    with np.errstate(invalid="ignore"):
        err = np.abs(g - nb0)
    err[both_ninf] = 0.0
    bad = np.flatnonzero(~(err <= tol))
    assert bad.size == 0, (f"{what}: {bad.size} entries outside the envelope, e.g. index {bad[0]}: "
                           f"gpu {g[bad[0]]:.6g} oracle {nb0[bad[0]]:.6g} spread {spread[bad[0]]:.3g}")
    vs = np.concatenate([[0], np.cumsum(num_states)])
    dec = np.asarray(gpu_dec)
    wrong = []
    for v in np.flatnonzero(dec != np.asarray(_argmax(nb0, vs))):
        b = nb0[vs[v]:vs[v + 1]]
        d = int(dec[v])
        if unstable[v] or (0 <= d < b.size and b[d] >= b.max() - tie):
            continue
        wrong.append(int(v))
    assert not wrong, f"{what}: decode differs at stable variables {wrong[:10]}"
    fin = np.isfinite(nb0)
    return float(err[fin].max()) if fin.any() else 0.0, float(spread[fin].max()) if fin.any() else 0.0


def _argmax(nb, vs):
    out = np.zeros(len(vs) - 1, np.int64)
    for v in range(len(vs) - 1):
        out[v] = int(np.argmax(nb[vs[v]:vs[v + 1]]))
    return out


def _factor_needed(err, spr, o):
    over = err - (ATOL + 1e-6 * np.abs(o))
    bad = over > 0
    if not bad.any():
        return 0.0
    with np.errstate(divide="ignore"):
        return float(np.max(over[bad] / spr[bad]))


def horizon_stats(gpu_nb, gpu_dec, nb0, spread, unstable, num_states, tie=TIE):
    """Figures of a long run against the oracle and its ensemble: |gpu - oracle| (max,
    99th percentile, median), the ensemble spread (max, median, fraction above 1e-4), the
    fraction of entries the GPU moves by more than 1e-4, and how many variables the GPU
    decodes differently from the FP64 oracle -- split into ensemble-unstable ones (the
    nearby FP64 runs disagree among themselves), oracle ties and stable ones."""
    g = np.asarray(gpu_nb, np.float64)
    fin = np.isfinite(nb0)
    with np.errstate(invalid="ignore"):
        err = np.abs(g - nb0)[fin]
    spr = spread[fin]
    vs = np.concatenate([[0], np.cumsum(num_states)])
    am = _argmax(nb0, vs)
    dec = np.asarray(gpu_dec)
    diff = np.flatnonzero(dec != am)
    n_unst = n_tie = n_stable = 0
    for v in diff:
        b = nb0[vs[v]:vs[v + 1]]
        d = int(dec[v])
        if unstable[v]:
            n_unst += 1
        elif 0 <= d < b.size and b[d] >= b.max() - tie:
            n_tie += 1
        else:
            n_stable += 1
    q = lambda a, f: float(np.quantile(a, f)) if a.size else 0.0
    return {"err_max": float(err.max()) if err.size else 0.0, "err_p99": q(err, 0.99), "err_median": q(err, 0.5),
            "err_frac_above_1e-4": float((err > 1e-4).mean()) if err.size else 0.0,
            "spread_max": float(spr.max()) if spr.size else 0.0, "spread_p99": q(spr, 0.99),
            "spread_median": q(spr, 0.5), "spread_frac_above_1e-4": float((spr > 1e-4).mean()) if spr.size else 0.0,
            "ratio_max": float(np.max(err / (1e-4 + spr))) if err.size else 0.0,
            # the smallest envelope factor that holds: max of (err - 1e-4 - 1e-6 |o|) / spread
            "factor_needed": _factor_needed(err, spr, nb0[fin]),
            "decode_diff": int(diff.size), "decode_diff_unstable": n_unst, "decode_diff_tie": n_tie,
            "decode_diff_stable": n_stable, "unstable_vars": int(np.asarray(unstable).sum()),
            "n_vars": int(len(num_states))}


def oracle_members(oracle, graph, log_pot, evidence, T, damping, n_iters, k=2, rel=1e-6, seed=12345):
    """The FP64 oracle run and an ensemble of nearby FP64 runs: one that rounds its
    messages to FP32 after every iteration (the storage model of an FP32-message
    implementation) and `k` with log-potentials and evidence multiplied by
    (1 + rel N(0,1)) (about 8 FP32 ulps). Returns (nb0, dec0, members), members a list of
    (normalised log-beliefs, decode) per ensemble run."""
    rng = np.random.default_rng(seed)
    m0, _ = oracle.run_bp(graph, log_pot, evidence, T, damping, n_iters)
    _, nb0, dec0, _ = oracle.beliefs(graph, evidence, m0)
    runs = [(log_pot, evidence, True)]
    for _ in range(k):
        lp = np.asarray(log_pot, np.float64) * (1 + rel * rng.standard_normal(np.size(log_pot)))
        ev = np.asarray(evidence, np.float64) * (1 + rel * rng.standard_normal(np.size(evidence)))
        runs.append((lp, ev, False))
    members = []
    for lp, ev, r32 in runs:
        m1, _ = oracle.run_bp(graph, lp, ev, T, damping, n_iters, round_f32=r32)
        _, nb1, dec1, _ = oracle.beliefs(graph, evidence, m1)
        members.append((nb1, dec1))
    return nb0, dec0, members


def deviation_figures(nb, dec, nb0, dec0, num_states, tie=TIE):
    """How far one run lies from the FP64 oracle run: quantiles of |nb - nb0| over the
    oracle's finite entries (a -inf entry on both sides counts 0, a NaN or a -inf on one
    side counts inf) and the number of variables decoded differently, oracle ties (two
    best states within `tie`) excepted."""
    g = np.asarray(nb, np.float64)
    fin = np.isfinite(nb0)
    with np.errstate(invalid="ignore"):
        e = np.abs(g - nb0)
    e = np.nan_to_num(e, nan=np.inf, posinf=np.inf)[fin]
    vs = np.concatenate([[0], np.cumsum(num_states)])
    n_diff = 0
    for v in np.flatnonzero(np.asarray(dec) != np.asarray(dec0)):
        b = nb0[vs[v]:vs[v + 1]]
        d = int(dec[v])
        if 0 <= d < b.size and b[d] >= b.max() - tie:
            continue
        n_diff += 1
    q = lambda f: float(np.quantile(e, f)) if e.size else 0.0
    return {"median": q(0.5), "p90": q(0.9), "p99": q(0.99), "max": float(e.max()) if e.size else 0.0,
            "frac_above_1e-4": float((e > 1e-4).mean()) if e.size else 0.0, "decode_diff": n_diff}


def assert_like_members(gpu_nb, gpu_dec, nb0, dec0, members, num_states, factor=3.0, atol=ATOL, what=""):
    """Long chaotic runs: FP32 message storage alone moves the FP64 result far beyond
    1e-4, so the GPU run is held to be one more member of the ensemble of nearby FP64 runs
    -- its deviation from the FP64 oracle run, at the median, 90th and 99th percentiles
    and at the maximum, and its number of differently decoded variables, at most `factor`
    times the largest member's (deviations plus atol). Returns (gpu figures, member
    figures)."""
    assert not np.isnan(np.asarray(gpu_nb, np.float64)).any(), f"{what}: NaN in GPU beliefs"
    fg = deviation_figures(gpu_nb, gpu_dec, nb0, dec0, num_states)
    fm = [deviation_figures(nb, dec, nb0, dec0, num_states) for nb, dec in members]
    for key in ("median", "p90", "p99", "max"):
        lim = atol + factor * max(f[key] for f in fm)
        assert fg[key] <= lim, f"{what}: GPU deviation {key} {fg[key]:.4g} above {lim:.4g} (members {[f[key] for f in fm]})"
    lim = factor * max(f["decode_diff"] for f in fm)
    assert fg["decode_diff"] <= lim, (f"{what}: GPU decodes {fg['decode_diff']} variables differently, above "
                                      f"{lim:.0f} (members {[f['decode_diff'] for f in fm]})")
    return fg, fm
