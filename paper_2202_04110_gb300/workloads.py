"""Seeded synthetic factor graphs and inputs.

This module only builds graph structure and draws random numbers; it holds none of
the belief-propagation arithmetic. The CUDA path and the FP64 oracle both consume
what it produces, so a workload is bit-identical on both sides.

Graph model (PGMax's model specification layer, Sec. 3, the package features: discrete
variables with a varying number of states, arbitrary topology, enumeration factors
given by their list of valid configurations, Sec. 5.2; logical factors, Sec. 3):

* ``num_states[v]``: number of states K_v of variable v.
* Enumeration group: factors that share an arity and a configuration list.
  ``cfg[c, j]`` is the state of the j-th neighbour in configuration c; ``vars[f, j]``
  is the j-th neighbour of factor f. Log-potentials are either one table per factor
  (``shared=False``: ``n_fac * n_cfg`` values, factor-major) or one table for the whole
  group (``shared=True``: ``n_cfg`` values).
* Logical group (OR / AND): ``child[f] = OP(parents[par_off[f]:par_off[f+1]])`` over
  binary variables.

Flat layouts (the message, evidence and log-potential arrays of the C-ABI):

* evidence / beliefs: variable-major, ``K_v`` log-space values per variable.
* log-potentials: enumeration groups in order, each as described above.
* messages (factor to variable): edges enumerated group by group (enumeration
  groups first, then logical groups), factor-major; an enumeration factor's edges in
  neighbour order, a logical factor's edges as its parents in order and then its
  child. Each edge holds ``K_v`` values of its variable.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

OR = 0
AND = 1
XOR = 2  # the child is the parity of the parents


@dataclass
class EnumGroup:
    cfg: np.ndarray  # int32 [n_cfg, arity]
    vars: np.ndarray  # int32 [n_fac, arity]
    shared: bool = False

    @property
    def arity(self) -> int:
        return int(self.cfg.shape[1])

    @property
    def n_cfg(self) -> int:
        return int(self.cfg.shape[0])

    @property
    def n_fac(self) -> int:
        return int(self.vars.shape[0])

    @property
    def n_potentials(self) -> int:
        return self.n_cfg if self.shared else self.n_fac * self.n_cfg


@dataclass
class LogicGroup:
    kind: int  # OR, AND or XOR
    par_off: np.ndarray  # int32 [n_fac + 1]
    parents: np.ndarray  # int32 [par_off[-1]]
    child: np.ndarray  # int32 [n_fac]

    @property
    def n_fac(self) -> int:
        return int(self.child.shape[0])


@dataclass
class FactorGraph:
    num_states: np.ndarray  # int32 [V]
    enum_groups: list = field(default_factory=list)
    logic_groups: list = field(default_factory=list)

    @property
    def n_vars(self) -> int:
        return int(self.num_states.shape[0])

    @property
    def n_var_states(self) -> int:
        return int(self.num_states.sum())

    @property
    def n_potentials(self) -> int:
        return int(sum(g.n_potentials for g in self.enum_groups))

    @property
    def n_factors(self) -> int:
        return int(sum(g.n_fac for g in self.enum_groups) + sum(g.n_fac for g in self.logic_groups))

    @property
    def n_edges(self) -> int:
        e = sum(g.n_fac * g.arity for g in self.enum_groups)
        e += sum(int(g.par_off[-1]) + g.n_fac for g in self.logic_groups)
        return int(e)

    @property
    def n_edge_states(self) -> int:
        k = self.num_states.astype(np.int64)
        es = sum(int(k[g.vars].sum()) for g in self.enum_groups)
        es += sum(2 * (int(g.par_off[-1]) + g.n_fac) for g in self.logic_groups)
        return int(es)


@dataclass
class Problem:
    """A factor graph plus the numeric inputs of one inference call."""

    name: str
    graph: FactorGraph
    log_pot: np.ndarray  # float32 [n_potentials]
    evidence: np.ndarray  # float32 [VS]
    T: float
    damping: float
    n_iters: int


# ---------------------------------------------------------------------------
# Building blocks
# ---------------------------------------------------------------------------

PAIR2_CFG = np.array([[0, 0], [0, 1], [1, 0], [1, 1]], dtype=np.int32)


def dense_pair_cfg(k0: int, k1: int) -> np.ndarray:
    """Every configuration of a (k0, k1) pairwise factor, row-major in (a, b)."""
    a, b = np.meshgrid(np.arange(k0), np.arange(k1), indexing="ij")
    return np.stack([a.ravel(), b.ravel()], axis=1).astype(np.int32)


def grid_pairs(rows: int, cols: int, base: int = 0) -> np.ndarray:
    """4-neighbour pairs of a row-major grid. For each cell: its right pair, then its
    down pair, so that consecutive cells touch consecutive factors."""
    r, c = np.meshgrid(np.arange(rows), np.arange(cols), indexing="ij")
    idx = (r * cols + c).ravel()
    right = (c < cols - 1).ravel()
    down = (r < rows - 1).ravel()
    # interleave: for each cell, [right, down] when present
    out = np.empty((idx.size, 2, 2), dtype=np.int64)
    out[:, 0, 0] = idx
    out[:, 0, 1] = idx + 1
    out[:, 1, 0] = idx
    out[:, 1, 1] = idx + cols
    keep = np.stack([right, down], axis=1).ravel()
    pairs = out.reshape(-1, 2)[keep]
    return (pairs + base).astype(np.int32)


def ising_grid(rows: int, cols: int, seed: int, T: float = 1.0, damping: float = 0.5,
               n_iters: int = 50, name: str | None = None) -> Problem:
    """2D Ising grid: couplings J~U[-1,1] as log-potentials [J,-J,-J,J] over the
    configurations (0,0),(0,1),(1,0),(1,1); field h~N(0,1) as evidence [-h, +h]."""
    rng = np.random.default_rng(seed)
    pairs = grid_pairs(rows, cols)
    n = rows * cols
    J = rng.uniform(-1.0, 1.0, size=pairs.shape[0])
    h = rng.standard_normal(n)
    pot = np.stack([J, -J, -J, J], axis=1).astype(np.float32).ravel()
    ev = np.stack([-h, h], axis=1).astype(np.float32).ravel()
    g = FactorGraph(np.full(n, 2, np.int32), [EnumGroup(PAIR2_CFG.copy(), pairs, False)], [])
    return Problem(name or f"ising{rows}x{cols}", g, pot, ev, T, damping, n_iters)


def potts_grid(side: int, K: int, seed: int, T: float = 1.0, damping: float = 0.5,
               n_iters: int = 100, w: float | None = None) -> Problem:
    """Potts grid with one truncated-linear table -w*min(|a-b|, 2) shared by all
    pairwise factors of the grid and N(0,1) log-evidence per state."""
    rng = np.random.default_rng(seed)
    if w is None:
        w = float(rng.uniform(0.5, 2.0))
    pairs = grid_pairs(side, side)
    cfg = dense_pair_cfg(K, K)
    table = (-w * np.minimum(np.abs(cfg[:, 0] - cfg[:, 1]), 2)).astype(np.float32)
    ev = rng.standard_normal(side * side * K).astype(np.float32)
    g = FactorGraph(np.full(side * side, K, np.int32), [EnumGroup(cfg, pairs, True)], [])
    return Problem(f"potts{side}K{K}", g, table, ev, T, damping, n_iters)


def rbm(n_vis: int, n_hid: int, seed: int, w_std: float = 0.1, T: float = 1.0,
        damping: float = 0.5, n_iters: int = 100) -> Problem:
    """Binary RBM: visible 0..n_vis-1, hidden after them, one dense pairwise factor per
    (visible, hidden) pair with log-potentials [0, 0, 0, W_ij], evidence [0, b]."""
    rng = np.random.default_rng(seed)
    W = rng.normal(0.0, w_std, size=(n_vis, n_hid))
    b = rng.standard_normal(n_vis + n_hid)
    vi, hj = np.meshgrid(np.arange(n_vis), np.arange(n_hid), indexing="ij")
    pairs = np.stack([vi.ravel(), n_vis + hj.ravel()], axis=1).astype(np.int32)
    pot = np.zeros((pairs.shape[0], 4), np.float32)
    pot[:, 3] = W.ravel()
    ev = np.zeros((n_vis + n_hid, 2), np.float32)
    ev[:, 1] = b
    g = FactorGraph(np.full(n_vis + n_hid, 2, np.int32), [EnumGroup(PAIR2_CFG.copy(), pairs, False)], [])
    return Problem(f"rbm{n_vis}x{n_hid}", g, pot.ravel(), ev.ravel(), T, damping, n_iters)


def deconvolution(seed: int, n_feat: int = 5, feat_side: int = 6, s_side: int = 10,
                  n_img: int = 100, p_w: float = 0.1, p_s: float = 0.02, flip: float = 0.05,
                  prior: float = -2.0, T: float = 0.0, damping: float = 0.5,
                  n_iters: int = 1000) -> Problem:
    """2D binary deconvolution with logical factors (the PGMax example notebook of
    Sec. 5.2, after Lazaro-Gredilla et al. 2021).

    Variables, numbered in this order: features W[k, dy, dx], activations
    S[n, k, py, px], one AND variable z per (n, k, p, d) with z = AND(W[k, d], S[n, k, p]),
    pixels X[n, y, x] = OR over every z that covers (y, x). Priors log-odds ``prior`` on
    W and S; X carries soft evidence of a seeded ground truth with ``flip`` bit flips.
    """
    rng = np.random.default_rng(seed)
    img = s_side + feat_side - 1
    nW = n_feat * feat_side * feat_side
    nS = n_img * n_feat * s_side * s_side
    W_gt = rng.random((n_feat, feat_side, feat_side)) < p_w
    S_gt = rng.random((n_img, n_feat, s_side, s_side)) < p_s
    # AND variables: index order (n, k, py, px, dy, dx)
    n, k, py, px, dy, dx = np.meshgrid(np.arange(n_img), np.arange(n_feat), np.arange(s_side),
                                       np.arange(s_side), np.arange(feat_side),
                                       np.arange(feat_side), indexing="ij")
    n, k, py, px, dy, dx = (a.ravel() for a in (n, k, py, px, dy, dx))
    nZ = n.size
    w_idx = k * feat_side * feat_side + dy * feat_side + dx
    s_idx = nW + ((n * n_feat + k) * s_side + py) * s_side + px
    z_idx = nW + nS + np.arange(nZ)
    pix = (n * img + (py + dy)) * img + (px + dx)  # flat pixel id
    nX = n_img * img * img
    x_idx = nW + nS + nZ + np.arange(nX)
    # AND group: parents (W, S), child z
    and_par = np.stack([w_idx, s_idx], axis=1).ravel().astype(np.int32)
    and_off = (np.arange(nZ + 1) * 2).astype(np.int32)
    # OR group: parents = z sorted by pixel (stable in z order), child X
    order = np.argsort(pix, kind="stable")
    counts = np.bincount(pix, minlength=nX)
    or_off = np.concatenate([[0], np.cumsum(counts)]).astype(np.int32)
    or_par = z_idx[order].astype(np.int32)
    # ground truth X and noisy observation
    z_gt = W_gt[k, dy, dx] & S_gt[n, k, py, px]
    X_gt = np.zeros(nX, bool)
    np.logical_or.at(X_gt, pix, z_gt)
    flips = rng.random(nX) < flip
    X_obs = X_gt ^ flips
    V = nW + nS + nZ + nX
    ev = np.zeros((V, 2), np.float32)
    ev[:nW + nS, 1] = prior
    lo = float(np.log((1 - flip) / flip))
    ev[nW + nS + nZ:, 1] = np.where(X_obs, lo, -lo)
    g = FactorGraph(np.full(V, 2, np.int32), [],
                    [LogicGroup(AND, and_off, and_par, z_idx.astype(np.int32)),
                     LogicGroup(OR, or_off, or_par, x_idx.astype(np.int32))])
    return Problem("deconv", g, np.zeros(0, np.float32), ev.ravel(), T, damping, n_iters)


def pool_offsets(radius: int) -> np.ndarray:
    """The (2 radius + 1)^2 states of a pool variable: 2-D offsets (dy, dx), row-major."""
    r = np.arange(-radius, radius + 1)
    dy, dx = np.meshgrid(r, r, indexing="ij")
    return np.stack([dy.ravel(), dx.ravel()], axis=1)


def pool_grid(side: int, radius: int, slack: int, seed: int, T: float = 0.0, damping: float = 0.5,
              n_iters: int = 50, shared: bool = True) -> Problem:
    """Grid of pool variables shaped like a recursive cortical network's (Sec. 5.2):
    each variable has K = (2 radius + 1)^2 states, one per 2-D offset of its feature
    within the pool; a lateral pairwise factor joins 4-neighbours and lists only the
    offset pairs that differ by at most `slack` in each coordinate (a sparse list of
    configurations, e.g. 361 of 49 x 49 for radius 3, slack 1). Log-potentials N(0, 1)
    per listed configuration (one table for the grid, or one per factor with
    shared=False); evidence N(0, 1) per state."""
    rng = np.random.default_rng(seed)
    off = pool_offsets(radius)
    K = off.shape[0]
    d = np.abs(off[:, None, :] - off[None, :, :]).max(axis=2)
    a, b = np.nonzero(d <= slack)
    cfg = np.stack([a, b], axis=1).astype(np.int32)
    pairs = grid_pairs(side, side)
    n_pot = cfg.shape[0] if shared else cfg.shape[0] * pairs.shape[0]
    pot = rng.standard_normal(n_pot).astype(np.float32)
    ev = rng.standard_normal(side * side * K).astype(np.float32)
    g = FactorGraph(np.full(side * side, K, np.int32), [EnumGroup(cfg, pairs, shared)], [])
    return Problem(f"pool{side}x{side}K{K}s{slack}", g, pot, ev, T, damping, n_iters)


def random_enum_factors(seed: int, n_vars: int, K: int, arity: int, n_fac: int, n_cfg: int,
                        shared: bool = True, T: float = 1.0, damping: float = 0.5,
                        n_iters: int = 20, scale: float = 1.0) -> Problem:
    """n_fac factors of `arity` distinct variables drawn at random among n_vars K-state
    variables, sharing one random list of n_cfg distinct configurations (at most K^arity);
    log-potentials and evidence N(0, scale^2)."""
    rng = np.random.default_rng(seed)
    total = K ** arity
    n_cfg = min(n_cfg, total)
    if total <= 1 << 22:
        codes = np.sort(rng.choice(total, size=n_cfg, replace=False))
    else:
        codes = np.unique(rng.integers(0, total, size=2 * n_cfg))[:n_cfg]
    cfg = np.stack([(codes // K ** (arity - 1 - j)) % K for j in range(arity)], axis=1).astype(np.int32)
    vars_ = np.stack([rng.choice(n_vars, size=arity, replace=False) for _ in range(n_fac)]).astype(np.int32)
    n_pot = cfg.shape[0] if shared else cfg.shape[0] * n_fac
    pot = (scale * rng.standard_normal(n_pot)).astype(np.float32)
    ev = (scale * rng.standard_normal(n_vars * K)).astype(np.float32)
    g = FactorGraph(np.full(n_vars, K, np.int32), [EnumGroup(cfg, vars_, shared)], [])
    return Problem(f"enum{arity}xK{K}c{cfg.shape[0]}", g, pot, ev, T, damping, n_iters)


def union(problems: list[Problem], name: str = "batch") -> Problem:
    """Disjoint union of several graphs: variables, groups, log-potentials and evidence
    concatenated in order. All members must share T and damping; the iteration count
    of the first member is kept."""
    ns, eg, lg, pots, evs = [], [], [], [], []
    base = 0
    for p in problems:
        g = p.graph
        ns.append(g.num_states)
        for e in g.enum_groups:
            eg.append(EnumGroup(e.cfg, (e.vars + base).astype(np.int32), e.shared))
        for l in g.logic_groups:
            lg.append(LogicGroup(l.kind, l.par_off, (l.parents + base).astype(np.int32),
                                 (l.child + base).astype(np.int32)))
        pots.append(p.log_pot)
        evs.append(p.evidence)
        base += g.n_vars
    g = FactorGraph(np.concatenate(ns).astype(np.int32), eg, lg)
    p0 = problems[0]
    return Problem(name, g, np.concatenate(pots).astype(np.float32),
                   np.concatenate(evs).astype(np.float32), p0.T, p0.damping, p0.n_iters)


# ---------------------------------------------------------------------------
# Workloads of the benchmark suite
# ---------------------------------------------------------------------------

def ising_small(seed: int = 0) -> Problem:
    """10x10 Ising grid, T=1, damping 0.5, 50 iterations (180 factors, 4 configs)."""
    return ising_grid(10, 10, seed, T=1.0, damping=0.5, n_iters=50, name="ising10x10")


def ising_large(seed: int = 0, T: float = 1.0, side: int = 1000, n_iters: int = 200) -> Problem:
    """1000x1000 Ising grid (1,998,000 pairwise factors), damping 0.5, 200 iterations."""
    return ising_grid(side, side, seed, T=T, damping=0.5, n_iters=n_iters,
                      name=f"ising{side}x{side}_T{T:g}")


def potts_batch_members(seed: int = 0, n_grids: int = 256, lo: int = 16, hi: int = 256,
                        Ks=(2, 4, 8, 16), n_iters: int = 100) -> list[Problem]:
    """Uneven Potts grids: side ~ U{lo..hi}, K ~ U(Ks), w ~ U[0.5, 2], evidence N(0,1)."""
    rng = np.random.default_rng(seed)
    sides = rng.integers(lo, hi + 1, size=n_grids)
    Kc = rng.choice(np.asarray(Ks), size=n_grids)
    ws = rng.uniform(0.5, 2.0, size=n_grids)
    seeds = rng.integers(0, 2**31 - 1, size=n_grids)
    return [potts_grid(int(s), int(k), int(sd), T=1.0, damping=0.5, n_iters=n_iters, w=float(w))
            for s, k, w, sd in zip(sides, Kc, ws, seeds)]


def potts_rbm_batch(seed: int = 0, n_grids: int = 256, n_iters: int = 100,
                    hi: int = 256, n_vis: int = 784, n_hid: int = 500) -> tuple[Problem, list[Problem]]:
    """256 uneven Potts grids plus a 784x500 RBM (W~N(0,0.1^2), biases N(0,1)), T=1."""
    members = potts_batch_members(seed, n_grids=n_grids, hi=hi, n_iters=n_iters)
    members.append(rbm(n_vis, n_hid, seed + 1, w_std=0.1, T=1.0, damping=0.5, n_iters=n_iters))
    return union(members, name="potts256+rbm"), members


def random_graph(seed: int, n_vars: int = 8, max_K: int = 3, n_pair: int = 6,
                 n_triple: int = 2, n_or: int = 1, n_and: int = 1, sparse: bool = True,
                 tree: bool = False, shared: bool = False, scale: float = 1.0,
                 n_xor: int = 0) -> tuple[FactorGraph, np.ndarray, np.ndarray]:
    """Small random factor graph with mixed state counts, pairwise and triple
    enumeration factors (optionally with sparse configuration lists) and logical
    factors over the binary variables. With ``tree=True`` only pairwise factors along
    a random spanning tree are drawn (LBP is exact there)."""
    rng = np.random.default_rng(seed)
    K = rng.integers(2, max_K + 1, size=n_vars).astype(np.int32)
    enum_groups, logic_groups, pots = [], [], []
    if tree:
        edges = [(int(rng.integers(0, i)), i) for i in range(1, n_vars)]
        by_shape: dict = {}
        for a, b in edges:
            by_shape.setdefault((int(K[a]), int(K[b])), []).append((a, b))
        for (ka, kb), lst in sorted(by_shape.items()):
            cfg = dense_pair_cfg(ka, kb)
            vars_ = np.asarray(lst, np.int32)
            n_pot = cfg.shape[0] if shared else cfg.shape[0] * len(lst)
            enum_groups.append(EnumGroup(cfg, vars_, shared))
            pots.append(rng.normal(0, scale, n_pot))
    else:
        # pairwise factors grouped by (K_a, K_b)
        by_shape = {}
        for _ in range(n_pair):
            a, b = rng.choice(n_vars, size=2, replace=False)
            by_shape.setdefault((int(K[a]), int(K[b])), []).append((int(a), int(b)))
        for (ka, kb), lst in sorted(by_shape.items()):
            cfg = dense_pair_cfg(ka, kb)
            if sparse and cfg.shape[0] > 2:
                keep = rng.random(cfg.shape[0]) < 0.75
                keep[rng.integers(0, cfg.shape[0])] = True
                cfg = cfg[keep]
            vars_ = np.asarray(lst, np.int32)
            n_pot = cfg.shape[0] if shared else cfg.shape[0] * len(lst)
            enum_groups.append(EnumGroup(cfg, vars_, shared))
            pots.append(rng.normal(0, scale, n_pot))
        # triple factors with a random configuration list (same K signature per group)
        if n_triple > 0:
            trip = rng.choice(n_vars, size=3, replace=False)
            sig = K[trip]
            full = np.stack(np.meshgrid(*[np.arange(k) for k in sig], indexing="ij"), -1).reshape(-1, 3)
            keep = rng.random(full.shape[0]) < (0.6 if sparse else 1.0)
            keep[0] = True
            cfg = full[keep].astype(np.int32)
            vars_ = [trip]
            cands = [v for v in range(n_vars)]
            for _ in range(n_triple - 1):
                # other triples with the same state signature, if available
                pick = []
                for k in sig:
                    opts = [v for v in cands if K[v] == k and v not in pick]
                    if not opts:
                        break
                    pick.append(int(rng.choice(opts)))
                if len(pick) == 3:
                    vars_.append(np.asarray(pick))
            vars_ = np.asarray(vars_, np.int32)
            n_pot = cfg.shape[0] if shared else cfg.shape[0] * vars_.shape[0]
            enum_groups.append(EnumGroup(cfg, vars_, shared))
            pots.append(rng.normal(0, scale, n_pot))
        # logical factors over binary variables
        binary = np.flatnonzero(K == 2)
        for kind, count in ((OR, n_or), (AND, n_and), (XOR, n_xor)):
            if count == 0 or binary.size < 2:
                continue
            offs, pars, ch = [0], [], []
            for _ in range(count):
                n_par = int(rng.integers(1, min(4, binary.size - 1) + 1))
                sel = rng.choice(binary, size=n_par + 1, replace=False)
                pars.extend(int(x) for x in sel[:-1])
                ch.append(int(sel[-1]))
                offs.append(len(pars))
            logic_groups.append(LogicGroup(kind, np.asarray(offs, np.int32),
                                           np.asarray(pars, np.int32), np.asarray(ch, np.int32)))
    g = FactorGraph(K, enum_groups, logic_groups)
    log_pot = (np.concatenate(pots) if pots else np.zeros(0)).astype(np.float32)
    evidence = rng.normal(0, scale, int(K.sum())).astype(np.float32)
    return g, log_pot, evidence


def random_factor_tree(seed: int, n_vars: int = 9, max_K: int = 3, shared: bool = False,
                       logical: bool = True, scale: float = 1.0,
                       xor: bool = False) -> tuple[FactorGraph, np.ndarray, np.ndarray]:
    """Random factor graph whose variable-factor graph is a tree: starting from one
    variable, each new factor joins one existing variable to 1-3 new ones. Factors are
    enumeration factors (dense or with a sparse configuration list) or, when all their
    variables are binary and ``logical`` is set, OR / AND factors (and XOR with ``xor``)."""
    rng = np.random.default_rng(seed)
    K = [int(rng.integers(2, max_K + 1))]
    enum_by_sig: dict = {}
    logic: dict = {OR: ([0], [], []), AND: ([0], [], []), XOR: ([0], [], [])}
    ENUM = -1
    while len(K) < n_vars:
        anchor = int(rng.integers(0, len(K)))
        n_new = int(min(rng.integers(1, 4), n_vars - len(K)))
        new = list(range(len(K), len(K) + n_new))
        if logical:
            draw = int(rng.integers(0, 4 if xor else 3))
            kind = {0: OR, 1: AND, 2: ENUM, 3: XOR}[draw]
        else:
            kind = ENUM
        if kind != ENUM:
            for _ in new:
                K.append(2)
            if K[anchor] != 2:
                kind = ENUM
        if kind == ENUM:
            for v in new:
                if len(K) <= v:
                    K.append(int(rng.integers(2, max_K + 1)))
            scope = [anchor] + new
            perm = rng.permutation(len(scope))
            scope = [scope[i] for i in perm]
            sig = tuple(K[v] for v in scope)
            enum_by_sig.setdefault(sig, []).append(scope)
        else:
            offs, pars, ch = logic[kind]
            scope = [anchor] + new
            c_pos = int(rng.integers(0, len(scope)))
            child = scope[c_pos]
            parents = [v for i, v in enumerate(scope) if i != c_pos]
            pars.extend(parents)
            ch.append(child)
            offs.append(len(pars))
    Karr = np.asarray(K, np.int32)
    enum_groups, pots = [], []
    for sig, scopes in sorted(enum_by_sig.items()):
        full = np.stack(np.meshgrid(*[np.arange(k) for k in sig], indexing="ij"), -1).reshape(-1, len(sig))
        keep = rng.random(full.shape[0]) < 0.7
        keep[int(rng.integers(0, full.shape[0]))] = True
        cfg = full[keep].astype(np.int32)
        vars_ = np.asarray(scopes, np.int32)
        enum_groups.append(EnumGroup(cfg, vars_, shared))
        n_pot = cfg.shape[0] if shared else cfg.shape[0] * vars_.shape[0]
        pots.append(rng.normal(0, scale, n_pot))
    logic_groups = []
    for kind in (OR, AND, XOR):
        offs, pars, ch = logic[kind]
        if ch:
            logic_groups.append(LogicGroup(kind, np.asarray(offs, np.int32),
                                           np.asarray(pars, np.int32), np.asarray(ch, np.int32)))
    g = FactorGraph(Karr, enum_groups, logic_groups)
    log_pot = (np.concatenate(pots) if pots else np.zeros(0)).astype(np.float32)
    evidence = rng.normal(0, scale, int(Karr.sum())).astype(np.float32)
    return g, log_pot, evidence


def serving_templates(seed: int = 0, n: int = 48, lo: int = 16, hi: int = 512, Ks=(2, 4, 16)):
    """Request templates of the serving workload: grids with side ~ U{lo..hi}, K ~ U(Ks)
    (K = 2: Ising, else Potts), T ~ U{0, 1}; damping 0.5."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        side = int(rng.integers(lo, hi + 1))
        K = int(rng.choice(np.asarray(Ks)))
        T = float(rng.choice([0.0, 1.0]))
        sd = int(rng.integers(0, 2**31 - 1))
        p = ising_grid(side, side, sd, T=T) if K == 2 else potts_grid(side, K, sd, T=T)
        out.append(p)
    return out


def poisson_arrivals(seed: int, rate: float, duration: float, n_templates: int, it_lo: int = 50, it_hi: int = 200):
    """Seeded Poisson arrival times in [0, duration) with a template index and an
    iteration count ~ U{it_lo..it_hi} per arrival."""
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += float(rng.exponential(1.0 / rate))
        if t >= duration:
            return out
        out.append((t, int(rng.integers(0, n_templates)), int(rng.integers(it_lo, it_hi + 1))))
