"""Checked mode's range checks (PGM_OPT_CHECKED), on the host and without a GPU.

pgm_audit_desc runs the rules the device audit applies, on the host copies of a
compiled description's index arrays: every valid workload passes, and one corrupted
entry in any array -- flat index arrays, configuration tables, lists by output state,
group records, variable lists -- is reported at exactly that array and position, while
the extreme values inside each range are accepted. No out-of-range index ever reaches a
GPU: the GPU tests run checked mode on valid graphs only.
"""
import numpy as np
import pytest

from paper_2202_04110_gb300 import workloads as W

VS_OFF, VIN_OFF, VIN_ES, EDGE_VS, EDGE_VAR, TAB4, LR_POS, PAROFF, CFG, BS, ENUM_REC, LOGIC_REC, VAR_LIST = range(13)


@pytest.fixture(scope="module")
def lib():
    from paper_2202_04110_gb300 import build
    build.build()
    from paper_2202_04110_gb300 import binding
    return binding


def _graphs():
    g_rand, _, _ = W.random_graph(3, n_vars=30, max_K=4, n_pair=40, n_triple=5, n_or=4, n_and=4, n_xor=4,
                                  sparse=True)
    return {"ising": W.ising_grid(7, 9, 0).graph, "potts": W.potts_grid(6, 8, 1).graph,
            "rbm": W.rbm(70, 80, 2).graph, "deconv": W.deconvolution(3, n_img=1).graph,
            "random": g_rand, "pool": W.pool_grid(5, 2, 1, 4).graph,
            "enum8": W.random_enum_factors(6, 20, 16, 8, 10, 300).graph}


def test_valid_graphs_pass(lib):
    for name, fg in _graphs().items():
        assert lib.audit_desc(fg) == (-1, -1), name


def _sizes(fg):
    E = fg.n_edges
    return fg.n_vars, fg.n_var_states, E, fg.n_edge_states


@pytest.mark.parametrize("name", ["ising", "potts", "rbm", "deconv", "random", "pool", "enum8"])
def test_corrupted_flat_arrays_are_found(lib, name):
    fg = _graphs()[name]
    V, VS, E, ES = _sizes(fg)
    rng = np.random.default_rng(len(name))
    # edge_vs: an edge of a high-degree variable carries its variable's first state with
    # the sign bit set (-2**31 is state 0 so marked; -1 would be state 2**31 - 1)
    cases = [(VS_OFF, V, VS + 1, VS), (VIN_OFF, V // 2, E + 1, E), (VIN_ES, E - 1, ES, ES - 1),
             (VIN_ES, 0, -1, 0), (EDGE_VS, E // 3, -1, -2 ** 31), (EDGE_VS, E - 1, VS, VS - 1),
             (EDGE_VS, 0, -2 ** 31 + VS, -2 ** 31 + VS - 1)]
    for arr, pos, bad, good in cases:
        pos = int(min(max(pos, 0), (V if arr in (VS_OFF, VIN_OFF) else E - 1)))
        assert lib.audit_desc(fg, arr, pos, bad) == (arr, pos), (name, arr, pos, bad)
        # the extreme value inside the range is accepted (where it keeps the arrays consistent
        # enough for the later checks, which read only what they range-check first)
        got = lib.audit_desc(fg, arr, pos, good)
        assert got[0] != arr, (name, arr, pos, good, got)
    del rng


def test_corrupted_specialised_arrays_are_found(lib):
    g = _graphs()
    # the 4-slot table and the log-ratio slot map of a binary grid
    fg = g["ising"]
    V, VS, E, ES = _sizes(fg)
    assert lib.audit_desc(fg, TAB4, 5, ES) == (TAB4, 5)
    assert lib.audit_desc(fg, TAB4, 6, -2) == (TAB4, 6)
    assert lib.audit_desc(fg, LR_POS, 7, 4 * V) == (LR_POS, 7)
    assert lib.audit_desc(fg, LR_POS, 7, 4 * V - 1) == (-1, -1)
    # per-edge variables and lists of a listed-configuration graph
    fg = g["pool"]
    V, VS, E, ES = _sizes(fg)
    assert lib.audit_desc(fg, EDGE_VAR, 3, V) == (EDGE_VAR, 3)
    assert lib.audit_desc(fg, EDGE_VAR, 3, V - 1) == (-1, -1)
    # parent offsets of logical groups
    fg = g["deconv"]
    V, VS, E, ES = _sizes(fg)
    assert lib.audit_desc(fg, PAROFF, 2, E + 1) == (PAROFF, 2)
    assert lib.audit_desc(fg, PAROFF, 2, -1) == (PAROFF, 2)


def test_corrupted_tables_lists_and_records_are_found(lib):
    g = _graphs()
    fg = g["random"]
    # a configuration entry naming a state beyond its neighbour's count
    assert lib.audit_desc(fg, CFG, 0, 200) == (CFG, 0)
    # lists by output state: an offset beyond the list and a configuration id beyond n_cfg
    for name in ("random", "pool", "enum8"):
        fg = g[name]
        assert lib.audit_desc(fg, BS, 0, -1) == (BS, 0), name
        assert lib.audit_desc(fg, BS, 1, 1 << 30) == (BS, 1), name
    # a group record whose edge-states would run past the message array
    fg = g["potts"]
    assert lib.audit_desc(fg, ENUM_REC, 0, fg.n_edge_states) == (ENUM_REC, 0)
    assert lib.audit_desc(fg, ENUM_REC, 0, -4) == (ENUM_REC, 0)
    fg = g["deconv"]
    assert lib.audit_desc(fg, LOGIC_REC, 1, 1 << 28) == (LOGIC_REC, 1)
    assert lib.audit_desc(fg, LOGIC_REC, 0, -1) == (LOGIC_REC, 0)


def test_corrupted_variable_list_is_found(lib):
    fg = _graphs()["random"]
    V = fg.n_vars
    assert lib.audit_desc(fg, VAR_LIST, 0, V) == (VAR_LIST, 0)
    assert lib.audit_desc(fg, VAR_LIST, 0, -1) == (VAR_LIST, 0)


def test_bad_requests_are_rejected(lib):
    fg = _graphs()["ising"]
    with pytest.raises(lib.PgmError):
        lib.audit_desc(fg, VIN_ES, 10 ** 9, 0)
    with pytest.raises(lib.PgmError):
        lib.audit_desc(fg, 99, 0, 0)


def test_logical_kinds(lib):
    """OR, AND and XOR groups compile; any other kind is rejected by the host compiler."""
    g, _, _ = W.random_graph(3, n_vars=30, max_K=2, n_pair=10, n_triple=0, n_or=2, n_and=2, n_xor=2)
    assert sorted(lg.kind for lg in g.logic_groups) == [W.OR, W.AND, W.XOR]
    assert lib.audit_desc(g) == (-1, -1)
    bad = W.FactorGraph(g.num_states, g.enum_groups,
                        [W.LogicGroup(3, lg.par_off, lg.parents, lg.child) for lg in g.logic_groups])
    with pytest.raises(lib.PgmError) as ei:
        lib.audit_desc(bad)
    assert ei.value.status == -1 and "kind" in str(ei.value)
