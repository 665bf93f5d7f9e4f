"""Comparison helpers for GPU-vs-oracle parity (test code only)."""
import numpy as np

# Normalised log-beliefs (b - LSE_1(b)) of the FP32 GPU path must agree with the FP64
# oracle to 1e-4 absolute after the same iteration count; MAP decodes must be equal
# except where the oracle's two best states are within 1e-6 (several answers correct).
ATOL = 1e-4
TIE = 1e-6


def assert_beliefs_close(gpu, ora, atol=ATOL, what=""):
    g = np.asarray(gpu, np.float64)
    o = np.asarray(ora, np.float64)
    assert g.shape == o.shape, (g.shape, o.shape)
    assert not np.isnan(g).any(), f"{what}: NaN in GPU beliefs"
    ninf_g, ninf_o = np.isneginf(g), np.isneginf(o)
    assert (ninf_g == ninf_o).all(), f"{what}: -inf pattern differs at {np.flatnonzero(ninf_g != ninf_o)[:10]}"
    fin = ~ninf_o
    if fin.any():
        err = np.abs(g[fin] - o[fin])
        worst = int(np.argmax(err))
        assert err.max() <= atol, f"{what}: max |gpu - oracle| = {err.max():.3e} at {np.flatnonzero(fin)[worst]}"
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
