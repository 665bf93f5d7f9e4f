"""FP64 CPU oracle for log-space loopy belief propagation (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may
import this package. It shares no code with the CUDA path: the arithmetic lives in
``lbp_oracle.c`` (plain C, double precision), this module only marshals numpy arrays.

Functions follow PGMax (arXiv 2202.04110): flooding LBP with damping (Sec. 3),
enumeration factors (Sec. 5.2), linear-time logical factors (Sec. 3), MAP decode
(Sec. 5.1). ``lbp_oracle.c`` states each step.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sysconfig

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

OR = 0
AND = 1
FLAG_CONTRADICTION = 1
FLAG_NAN = 2


def build(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (OpenMP over independent factors
    and variables; the arithmetic per message is sequential and deterministic)."""
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    cc = os.environ.get("CC", "gcc")
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = [cc, "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Graph(ctypes.Structure):
    _fields_ = [
        ("n_vars", ctypes.c_int32),
        ("num_states", ctypes.c_void_p),
        ("n_enum", ctypes.c_int32),
        ("e_arity", ctypes.c_void_p),
        ("e_ncfg", ctypes.c_void_p),
        ("e_nfac", ctypes.c_void_p),
        ("e_shared", ctypes.c_void_p),
        ("e_cfg", ctypes.c_void_p),
        ("e_vars", ctypes.c_void_p),
        ("n_logic", ctypes.c_int32),
        ("l_kind", ctypes.c_void_p),
        ("l_nfac", ctypes.c_void_p),
        ("l_paroff", ctypes.c_void_p),
        ("l_parents", ctypes.c_void_p),
        ("l_child", ctypes.c_void_p),
    ]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        lib.og_bp.restype = ctypes.c_int
        lib.og_bp.argtypes = [ctypes.POINTER(_Graph), ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                              ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
        lib.og_beliefs.restype = ctypes.c_int
        lib.og_beliefs.argtypes = [ctypes.POINTER(_Graph), ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                   ctypes.c_void_p]
        lib.og_logic_update.restype = ctypes.c_int
        lib.og_logic_update.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_double, ctypes.c_int, ctypes.c_void_p]
        lib.og_sizes.restype = ctypes.c_int
        lib.og_sizes.argtypes = [ctypes.POINTER(_Graph), ctypes.c_void_p]
        lib.og_grad.restype = ctypes.c_int
        lib.og_grad.argtypes = [ctypes.POINTER(_Graph), ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                ctypes.c_void_p]
        lib.og_num_threads.restype = ctypes.c_int
        lib.og_set_num_threads.restype = ctypes.c_int
        lib.og_set_num_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class _Marshalled:
    """Keeps the numpy buffers behind an ``og_graph`` alive."""

    def __init__(self, graph):
        keep = []

        def i32(a):
            a = np.ascontiguousarray(a, dtype=np.int32)
            keep.append(a)
            return a

        def ptrs(lst):
            arr = (ctypes.c_void_p * max(1, len(lst)))(*[_ptr(x) for x in lst])
            keep.append(arr)
            return ctypes.cast(arr, ctypes.c_void_p)

        eg, lg = graph.enum_groups, graph.logic_groups
        g = _Graph()
        g.n_vars = graph.n_vars
        g.num_states = _ptr(i32(graph.num_states))
        g.n_enum = len(eg)
        g.e_arity = _ptr(i32([e.arity for e in eg] or [0]))
        g.e_ncfg = _ptr(i32([e.n_cfg for e in eg] or [0]))
        g.e_nfac = _ptr(i32([e.n_fac for e in eg] or [0]))
        g.e_shared = _ptr(i32([int(e.shared) for e in eg] or [0]))
        g.e_cfg = ptrs([i32(e.cfg) for e in eg])
        g.e_vars = ptrs([i32(e.vars) for e in eg])
        g.n_logic = len(lg)
        g.l_kind = _ptr(i32([l.kind for l in lg] or [0]))
        g.l_nfac = _ptr(i32([l.n_fac for l in lg] or [0]))
        g.l_paroff = ptrs([i32(l.par_off) for l in lg])
        g.l_parents = ptrs([i32(l.parents if l.parents.size else np.zeros(1)) for l in lg])
        g.l_child = ptrs([i32(l.child if l.child.size else np.zeros(1)) for l in lg])
        self.g = g
        self.keep = keep


def sizes(graph) -> dict:
    """V, VS, E, ES and the number of log-potentials, computed by the oracle's own
    layout code."""
    lib = _load()
    m = _Marshalled(graph)
    out = np.zeros(6, np.int64)
    lib.og_sizes(ctypes.byref(m.g), _ptr(out))
    return dict(V=int(out[0]), VS=int(out[1]), E=int(out[2]), ES=int(out[3]), P=int(out[4]))


def run_bp(graph, log_pot, evidence, T: float, damping: float, n_iters: int,
           msgs: np.ndarray | None = None, logic_brute: bool = False, round_f32: bool = False):
    """Flooding LBP for ``n_iters`` iterations from ``msgs`` (zeros when None).
    ``round_f32`` rounds the messages to FP32 after every iteration (FP32 storage model).
    Returns (messages [ES] float64, flags)."""
    lib = _load()
    m = _Marshalled(graph)
    ES = sizes(graph)["ES"]
    out = np.zeros(max(ES, 1), np.float64) if msgs is None else np.array(msgs, np.float64)
    lp = np.ascontiguousarray(log_pot, np.float64)
    if lp.size == 0:
        lp = np.zeros(1)
    ev = np.ascontiguousarray(evidence, np.float64)
    fl = np.zeros(1, np.uint32)
    rc = lib.og_bp(ctypes.byref(m.g), _ptr(lp), _ptr(ev), float(T), float(damping),
                   int(n_iters), int(logic_brute), int(round_f32), _ptr(out), _ptr(fl))
    if rc != 0:
        raise ValueError("oracle: invalid T, damping or n_iters")
    return out[:ES], int(fl[0])


def beliefs(graph, evidence, msgs):
    """Returns (raw beliefs [VS], normalised log-beliefs [VS], decode [V], flags)."""
    lib = _load()
    m = _Marshalled(graph)
    VS, V = graph.n_var_states, graph.n_vars
    raw = np.zeros(VS, np.float64)
    nb = np.zeros(VS, np.float64)
    dec = np.zeros(V, np.int32)
    fl = np.zeros(1, np.uint32)
    ev = np.ascontiguousarray(evidence, np.float64)
    ms = np.ascontiguousarray(msgs, np.float64)
    if ms.size == 0:
        ms = np.zeros(1)
    lib.og_beliefs(ctypes.byref(m.g), _ptr(ev), _ptr(ms), _ptr(raw), _ptr(nb), _ptr(dec), _ptr(fl))
    return raw, nb, dec, int(fl[0])


def infer(problem, n_iters: int | None = None, T: float | None = None,
          logic_brute: bool = False):
    """Cold-start LBP on a ``workloads.Problem``. Returns (normalised log-beliefs,
    decode, messages, flags)."""
    it = problem.n_iters if n_iters is None else n_iters
    t = problem.T if T is None else T
    msgs, fl = run_bp(problem.graph, problem.log_pot, problem.evidence, t, problem.damping,
                      it, logic_brute=logic_brute)
    _, nb, dec, fl2 = beliefs(problem.graph, problem.evidence, msgs)
    return nb, dec, msgs, fl | fl2


def logic_update(kind: int, v2f: np.ndarray, T: float, brute: bool = False) -> np.ndarray:
    """One logical factor: ``v2f`` [(n+1), 2] incoming messages (parents, then child).
    Returns the outgoing max-normalised messages [(n+1), 2]."""
    lib = _load()
    v = np.ascontiguousarray(v2f, np.float64).reshape(-1, 2)
    n = v.shape[0] - 1
    out = np.zeros_like(v)
    lib.og_logic_update(int(kind), n, _ptr(v), float(T), int(brute), _ptr(out))
    return out


def grad(graph, log_pot, evidence, T: float, damping: float, n_iters: int, g_nb):
    """Gradient of L = sum(g_nb * normalised log-beliefs) after n_iters iterations from
    zero messages, w.r.t. (log-potentials, evidence). T > 0; logical factors of fan-in
    at most 20 (their adjoint enumerates the valid configurations)."""
    lib = _load()
    m = _Marshalled(graph)
    lp = np.ascontiguousarray(log_pot, np.float64)
    if lp.size == 0:
        lp = np.zeros(1)
    ev = np.ascontiguousarray(evidence, np.float64)
    gn = np.ascontiguousarray(g_nb, np.float64)
    dlp = np.zeros(max(graph.n_potentials, 1), np.float64)
    dev = np.zeros(graph.n_var_states, np.float64)
    rc = lib.og_grad(ctypes.byref(m.g), _ptr(lp), _ptr(ev), float(T), float(damping), int(n_iters),
                     _ptr(gn), _ptr(dlp), _ptr(dev))
    if rc == -2:
        raise ValueError("oracle grad: a logical factor has more than 20 parents")
    if rc != 0:
        raise ValueError("oracle grad: invalid T, damping or n_iters")
    return dlp[:graph.n_potentials], dev


def loss(graph, log_pot, evidence, T, damping, n_iters, g_nb) -> float:
    """L = sum(g_nb * normalised log-beliefs) after n_iters iterations from zero messages."""
    msgs, _ = run_bp(graph, log_pot, evidence, T, damping, n_iters)
    _, nb, _, _ = beliefs(graph, evidence, msgs)
    return float(np.dot(np.asarray(g_nb, np.float64), nb))


def num_threads() -> int:
    return int(_load().og_num_threads())


def set_num_threads(n: int) -> int:
    """OpenMP threads of the following calls (timing only; results do not depend on it).
    Returns the count in effect."""
    return int(_load().og_set_num_threads(int(n)))
