"""C-ABI checks that need no GPU: the library loads, exports every symbol declared in
include/pgm.h, and its host graph compiler validates descriptions and reports exact
sizes (the flat layout of Sec. 4 of the paper: one value per edge-state)."""
import os
import re

import numpy as np
import pytest

from paper_2202_04110_gb300 import binding as B
from paper_2202_04110_gb300 import build as BUILD
from paper_2202_04110_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    BUILD.build()
    return B.load_library()


def declared_symbols():
    syms = set()
    for name in os.listdir(os.path.join(ROOT, "include")):
        if name.endswith(".h"):
            src = open(os.path.join(ROOT, "include", name)).read()
            syms |= set(re.findall(r"^\s*(?:pgm_status|void|const char \*)\s*\*?\s*(pgm_\w+)\s*\(", src, re.M))
    return syms


def test_exports_every_declared_symbol(lib):
    syms = declared_symbols()
    assert "pgm_run_bp" in syms and "pgm_build" in syms
    for s in sorted(syms):
        assert hasattr(lib, s), s
    assert set(B.EXPORTED) == syms


def test_sizes_match_workload_counts(lib):
    for p in (W.ising_small(0), W.ising_grid(37, 23, 1), W.potts_grid(20, 4, 2), W.rbm(30, 20, 3)):
        info = B.check_desc(p.graph)
        assert info["n_vars"] == p.graph.n_vars
        assert info["n_var_states"] == p.graph.n_var_states
        assert info["n_edges"] == p.graph.n_edges
        assert info["n_edge_states"] == p.graph.n_edge_states
        assert info["n_potentials"] == p.graph.n_potentials == p.log_pot.size
    d = W.deconvolution(0, n_img=4, n_iters=1)
    info = B.check_desc(d.graph)
    assert info["n_edge_states"] == d.graph.n_edge_states
    assert info["max_degree"] == 4 * 100  # each W variable is in n_img * 10 * 10 AND factors


def test_ising_large_exact_counts(lib):
    p = W.ising_grid(1000, 1000, 0, n_iters=1)
    info = B.check_desc(p.graph)
    assert info["n_factors"] == 1_998_000
    assert info["n_edges"] == 3_996_000
    assert info["n_edge_states"] == 7_992_000
    assert info["n_var_states"] == 2_000_000
    assert info["max_degree"] == 4


def _bad(fg, match):
    with pytest.raises(B.PgmError) as ei:
        B.check_desc(fg)
    assert ei.value.status == -1
    assert match in str(ei.value)


def test_validation_errors(lib):
    cfg = W.PAIR2_CFG.copy()
    ok = W.FactorGraph(np.array([2, 2], np.int32), [W.EnumGroup(cfg, np.array([[0, 1]], np.int32))])
    B.check_desc(ok)
    _bad(W.FactorGraph(np.array([2, 2], np.int32), [W.EnumGroup(cfg, np.array([[0, 2]], np.int32))]), "out of range")
    _bad(W.FactorGraph(np.array([2, 0], np.int32), []), "states")
    _bad(W.FactorGraph(np.array([2, 3], np.int32), [W.EnumGroup(np.array([[0, 3]], np.int32), np.array([[0, 1]], np.int32))]), "out of range")
    _bad(W.FactorGraph(np.array([2, 2, 3], np.int32), [W.EnumGroup(cfg, np.array([[0, 1], [0, 2]], np.int32))]), "differs")
    _bad(W.FactorGraph(np.array([2, 3], np.int32), [], [W.LogicGroup(W.OR, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([1], np.int32))]), "not binary")
    _bad(W.FactorGraph(np.array([2, 2], np.int32), [], [W.LogicGroup(W.OR, np.array([0, 2, 1], np.int32), np.array([0, 1], np.int32), np.array([1, 0], np.int32))]), "decreases")
    _bad(W.FactorGraph(np.array([2, 2], np.int32), [], [W.LogicGroup(7, np.array([0, 1], np.int32), np.array([0], np.int32), np.array([1], np.int32))]), "kind")
    big = np.full(9, 2, np.int32)
    _bad(W.FactorGraph(big, [W.EnumGroup(np.zeros((1, 9), np.int32), np.arange(9, dtype=np.int32)[None])]), "arity")


def test_zero_parent_logical_factor_accepted(lib):
    fg = W.FactorGraph(np.array([2, 2], np.int32), [], [W.LogicGroup(W.OR, np.array([0, 0], np.int32), np.zeros(0, np.int32), np.array([1], np.int32))])
    info = B.check_desc(fg)
    assert info["n_edges"] == 1 and info["n_edge_states"] == 2


def test_product_path_has_no_oracle_import():
    """The product modules never import the oracle."""
    pkg = os.path.join(ROOT, "paper_2202_04110_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in src and "from oracle" not in src, f
                assert "lbp_oracle" not in src, f


def test_large_enumeration_groups_accepted(lib):
    """State sums above 64 (up to 8 neighbours x 256 states) and long configuration lists
    compile on the host (the block-form kernels take them); sizes are exact."""
    K = 256
    cfg = np.stack([np.arange(K), (np.arange(K) + 1) % K], axis=1).astype(np.int32)
    fg = W.FactorGraph(np.full(3, K, np.int32), [W.EnumGroup(cfg, np.array([[0, 1], [1, 2]], np.int32))])
    info = B.check_desc(fg)
    assert info["n_edge_states"] == 2 * 2 * K and info["n_potentials"] == 2 * K
    big = np.zeros((3, 8), np.int32)
    big[1] = 255
    big[2] = np.arange(8)
    fg8 = W.FactorGraph(np.full(8, K, np.int32), [W.EnumGroup(big, np.arange(8, dtype=np.int32)[None], True)])
    info = B.check_desc(fg8)
    assert info["n_edge_states"] == 8 * K and info["n_potentials"] == 3
    p = W.pool_grid(16, 5, 2, 0)
    info = B.check_desc(p.graph)
    assert info["n_edge_states"] == 2 * (2 * 16 * 15) * 121
    assert info["n_potentials"] == 2401
