"""Independent dense references used to pin the oracle (test code only).

Nothing here is shared with the oracle or the CUDA path. Every factor is expanded into
a dense log-potential tensor over the product of its neighbours' state spaces (-inf on
configurations that are not listed, or that violate a logical factor), so these
routines evaluate the definitions by exhaustive enumeration:

* ``joint_scores``: the unnormalised log-probability of every joint configuration of a
  tiny graph (sum of evidence and factor log-potentials).
* ``exact_log_marginals``: log-marginals (T=1) or log max-marginals (T=0) by reducing the
  joint table; LBP must reproduce them on trees (Pearl 1988).
* ``dense_lbp``: flooding LBP with the messages kept unnormalised and damping applied to
  the raw messages; the normalised beliefs are invariant to per-edge constant shifts, so
  they must equal the oracle's (which normalises every message).
* ``logic_dense``: a logical factor's outgoing messages by enumerating all 2^(n+1)
  joint states of its parents and child.
"""
from __future__ import annotations

import itertools

import numpy as np

from paper_2202_04110_gb300.workloads import AND, OR, XOR


def lse(z, axis=None, T=1.0):
    z = np.asarray(z, np.float64)
    if T == 0.0:
        return np.max(z, axis=axis)
    m = np.max(z, axis=axis, keepdims=True)
    safe = np.where(np.isfinite(m), m, 0.0)
    with np.errstate(divide="ignore"):
        s = T * np.log(np.sum(np.exp((z - safe) / T), axis=axis, keepdims=True)) + safe
    s = np.where(np.isneginf(m), -np.inf, s)
    return np.squeeze(s, axis=axis) if axis is not None else s.reshape(())


def dense_factors(graph, log_pot):
    """List of (scope, tensor) in the flat edge order of the message layout."""
    out = []
    off = 0
    K = graph.num_states
    for g in graph.enum_groups:
        for f in range(g.n_fac):
            scope = [int(v) for v in g.vars[f]]
            t = np.full([int(K[v]) for v in scope], -np.inf)
            phi = log_pot[off:off + g.n_cfg] if g.shared else log_pot[off + f * g.n_cfg: off + (f + 1) * g.n_cfg]
            for c in range(g.n_cfg):
                t[tuple(g.cfg[c])] = np.logaddexp(t[tuple(g.cfg[c])], float(phi[c]))
            out.append((scope, t))
        off += g.n_potentials
    for g in graph.logic_groups:
        for f in range(g.n_fac):
            pars = [int(v) for v in g.parents[g.par_off[f]:g.par_off[f + 1]]]
            scope = pars + [int(g.child[f])]
            n = len(pars)
            t = np.full([2] * (n + 1), -np.inf)
            for p in itertools.product((0, 1), repeat=n):
                c = int(any(p)) if g.kind == OR else int(all(p)) if g.kind == AND else sum(p) % 2
                t[tuple(p) + (c,)] = 0.0
            out.append((scope, t))
    return out


def joint_scores(graph, log_pot, evidence):
    K = [int(k) for k in graph.num_states]
    V = len(K)
    vs = np.concatenate([[0], np.cumsum(K)])
    total = np.zeros(K)
    for v in range(V):
        shape = [1] * V
        shape[v] = K[v]
        total = total + np.asarray(evidence[vs[v]:vs[v + 1]], np.float64).reshape(shape)
    for scope, t in dense_factors(graph, np.asarray(log_pot, np.float64)):
        # broadcast t over the full joint: move its axes into place
        shape = [1] * V
        for ax, v in enumerate(scope):
            shape[v] = K[v]
        # scopes in tests never repeat a variable
        order = np.argsort(scope)
        tt = np.transpose(t, order).reshape(shape)
        total = total + tt
    return total


def exact_log_marginals(graph, log_pot, evidence, T):
    """Normalised log-marginals (T=1) or max-marginals shifted so that their LSE_1 is
    zero (T=0), variable-major [VS]."""
    J = joint_scores(graph, log_pot, evidence)
    V = J.ndim
    out = []
    for v in range(V):
        axes = tuple(a for a in range(V) if a != v)
        m = lse(J, axis=axes, T=T) if axes else J.copy()
        out.append(m - lse(m, T=1.0))
    return np.concatenate(out)


def brute_map(graph, log_pot, evidence):
    J = joint_scores(graph, log_pot, evidence)
    return np.array(np.unravel_index(np.argmax(J), J.shape)), float(np.max(J))


def _edges(graph, factors):
    """Flat edge list [(factor index, position, variable)] in the message layout order."""
    edges = []
    for fi, (scope, _) in enumerate(factors):
        for pos, v in enumerate(scope):
            edges.append((fi, pos, v))
    return edges


def factor_messages_dense(scope, t, v2f, T):
    """Outgoing messages of one dense factor from incoming messages v2f[pos] (raw)."""
    out = []
    a = len(scope)
    for i in range(a):
        s = t.copy()
        for j in range(a):
            if j == i:
                continue
            shape = [1] * a
            shape[j] = t.shape[j]
            s = s + v2f[j].reshape(shape)
        axes = tuple(j for j in range(a) if j != i)
        out.append(lse(s, axis=axes, T=T) if axes else s.copy())
    return out


def dense_lbp(graph, log_pot, evidence, T, damping, n_iters, msgs=None):
    """Flooding LBP with raw (never normalised) messages. Returns (normalised
    log-beliefs [VS], raw messages as a list per edge)."""
    K = [int(k) for k in graph.num_states]
    V = len(K)
    vs = np.concatenate([[0], np.cumsum(K)])
    ev = [np.asarray(evidence[vs[v]:vs[v + 1]], np.float64) for v in range(V)]
    factors = dense_factors(graph, np.asarray(log_pot, np.float64))
    edges = _edges(graph, factors)
    if msgs is None:
        m = [np.zeros(K[v]) for (_, _, v) in edges]
    else:
        m = [np.asarray(x, np.float64).copy() for x in msgs]
    by_var = [[] for _ in range(V)]
    for e, (_, _, v) in enumerate(edges):
        by_var[v].append(e)
    first_edge = []
    e = 0
    for scope, _ in factors:
        first_edge.append(e)
        e += len(scope)
    for _ in range(n_iters):
        v2f = []
        for e, (_, _, v) in enumerate(edges):
            s = ev[v].copy()
            for g in by_var[v]:
                if g != e:
                    s = s + m[g]
            v2f.append(s)
        new = [None] * len(edges)
        for fi, (scope, t) in enumerate(factors):
            e0 = first_edge[fi]
            outs = factor_messages_dense(scope, t, [v2f[e0 + j] for j in range(len(scope))], T)
            for j, o in enumerate(outs):
                new[e0 + j] = o if damping == 0.0 else damping * m[e0 + j] + (1 - damping) * o
        m = new
    beliefs = []
    for v in range(V):
        b = ev[v].copy()
        for g in by_var[v]:
            b = b + m[g]
        beliefs.append(b - lse(b))
    return np.concatenate(beliefs), m


def logic_dense(kind, v2f, T):
    """Outgoing max-normalised messages of one logical factor, v2f [(n+1), 2]."""
    v2f = np.asarray(v2f, np.float64)
    n = v2f.shape[0] - 1
    t = np.full([2] * (n + 1), -np.inf)
    for p in itertools.product((0, 1), repeat=n):
        c = int(any(p)) if kind == OR else int(all(p)) if kind == AND else sum(p) % 2
        t[tuple(p) + (c,)] = 0.0
    outs = factor_messages_dense(list(range(n + 1)), t, list(v2f), T)
    res = []
    for o in outs:
        res.append(o - np.max(o))
    return np.stack(res)


def log_potential_of(graph, log_pot, evidence, x):
    """Joint unnormalised log-probability of one full assignment x."""
    J = joint_scores(graph, log_pot, evidence)
    return float(J[tuple(int(v) for v in x)])
