"""Thin ctypes binding over libpgm.so (include/pgm.h).

Argument marshalling only: every step of belief propagation runs in the library's CUDA
kernels. PyTorch supplies device memory and the current stream. There is no CPU
fallback: when the library is missing or CUDA is unavailable, calls raise.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpgm.so")

PGM_OK = 0
STATUS_NAMES = {-1: "PGM_EINVAL", -2: "PGM_ENOMEM", -3: "PGM_ECUDA", -4: "PGM_ENOTSUP",
                -5: "PGM_EBUSY", -6: "PGM_ETIMEDOUT"}
FLAG_CONTRADICTION = 1
FLAG_NAN = 2
FLAG_INDEX = 4

# Every symbol include/pgm.h declares.
EXPORTED = ["pgm_build", "pgm_build_batch", "pgm_batch_member", "pgm_check_desc", "pgm_free", "pgm_graph_info", "pgm_run_bp", "pgm_beliefs",
            "pgm_decode", "pgm_infer_host", "pgm_set_profiling", "pgm_pass_times", "pgm_launch_times",
            "pgm_device_flags", "pgm_checked_report", "pgm_audit_desc", "pgm_grid2_run_bp_noalloc", "pgm_grid2_noalloc_flags", "pgm_run_bp_multi", "pgm_pmp_sample", "pgm_run_bp_until", "pgm_run_bp_until_members", "pgm_run_bp_batch", "pgm_set_option", "pgm_get_option", "pgm_autotune",
            "pgm_launch_info", "pgm_grad", "pgm_serve_create", "pgm_serve_submit", "pgm_serve_submit_until", "pgm_serve_submit_borrowed", "pgm_serve_poll",
            "pgm_serve_wait", "pgm_serve_stats", "pgm_serve_destroy", "pgm_last_error"]
OPT_CUDA_GRAPH = 1
OPT_LOG_RATIO = 2
OPT_ENUM_BLOCK = 3
OPT_PAIR_FORM = 4
OPT_CHECKED = 5
OPT_SMALL_RUN = 6


class PgmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class EnumGroupC(ctypes.Structure):
    _fields_ = [("arity", ctypes.c_int32), ("n_cfg", ctypes.c_int32), ("cfg", ctypes.c_void_p),
                ("n_fac", ctypes.c_int32), ("vars", ctypes.c_void_p),
                ("shared_potentials", ctypes.c_int32)]


class LogicGroupC(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("n_fac", ctypes.c_int32), ("par_off", ctypes.c_void_p),
                ("parents", ctypes.c_void_p), ("child", ctypes.c_void_p)]


class GraphDescC(ctypes.Structure):
    _fields_ = [("n_vars", ctypes.c_int32), ("num_states", ctypes.c_void_p),
                ("n_enum_groups", ctypes.c_int32), ("enum_groups", ctypes.POINTER(EnumGroupC)),
                ("n_logic_groups", ctypes.c_int32), ("logic_groups", ctypes.POINTER(LogicGroupC))]


class InfoC(ctypes.Structure):
    _fields_ = [("n_vars", ctypes.c_int64), ("n_var_states", ctypes.c_int64),
                ("n_factors", ctypes.c_int64), ("n_edges", ctypes.c_int64),
                ("n_edge_states", ctypes.c_int64), ("n_potentials", ctypes.c_int64),
                ("max_states", ctypes.c_int32), ("max_degree", ctypes.c_int32),
                ("device_bytes", ctypes.c_int64), ("launches_per_iter", ctypes.c_int32),
                ("n_members", ctypes.c_int32)]


class ServerConfigC(ctypes.Structure):
    _fields_ = [("memory_budget_bytes", ctypes.c_int64), ("max_in_flight", ctypes.c_int32),
                ("max_pending", ctypes.c_int32)]


class ServerStatsC(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("submitted", "completed", "failed", "pending", "in_flight",
                                              "bytes_in_use", "peak_bytes", "updates_done")] + \
               [(n, ctypes.c_double) for n in ("span_s", "queue_s", "compile_s", "admit_s", "run_s")]


class MemberC(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("var_off", "n_vars", "vs_off", "n_var_states", "edge_off",
                                              "n_edges", "es_off", "n_edge_states", "pot_off",
                                              "n_potentials")]


_lib = None


def load_library(path: str | None = None):
    """Load libpgm.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"libpgm.so not built ({p}); run paper_2202_04110_gb300.build.build()")
    lib = ctypes.CDLL(p)
    vp, i32, f32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_float
    lib.pgm_build.restype = i32
    lib.pgm_build.argtypes = [ctypes.POINTER(GraphDescC), ctypes.POINTER(vp)]
    lib.pgm_build_batch.restype = i32
    lib.pgm_build_batch.argtypes = [ctypes.POINTER(ctypes.POINTER(GraphDescC)), i32, ctypes.POINTER(vp)]
    lib.pgm_batch_member.restype = i32
    lib.pgm_batch_member.argtypes = [vp, i32, ctypes.POINTER(MemberC)]
    lib.pgm_check_desc.restype = i32
    lib.pgm_check_desc.argtypes = [ctypes.POINTER(GraphDescC), ctypes.POINTER(InfoC)]
    lib.pgm_free.restype = None
    lib.pgm_free.argtypes = [vp]
    lib.pgm_graph_info.restype = i32
    lib.pgm_graph_info.argtypes = [vp, ctypes.POINTER(InfoC)]
    lib.pgm_run_bp.restype = i32
    lib.pgm_run_bp.argtypes = [vp, vp, vp, f32, f32, i32, vp, vp]
    lib.pgm_run_bp_multi.restype = i32
    lib.pgm_run_bp_multi.argtypes = [vp, i32, vp, i32, vp, f32, f32, i32, vp, vp]
    lib.pgm_run_bp_until.restype = i32
    lib.pgm_run_bp_until.argtypes = [vp, vp, vp, f32, f32, i32, f32, i32, vp, vp, vp, vp]
    lib.pgm_run_bp_until_members.restype = i32
    lib.pgm_run_bp_until_members.argtypes = [vp, vp, vp, f32, f32, i32, f32, i32, vp, vp, vp, vp]
    lib.pgm_run_bp_batch.restype = i32
    lib.pgm_run_bp_batch.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp]
    lib.pgm_pmp_sample.restype = i32
    lib.pgm_pmp_sample.argtypes = [vp, i32, vp, vp, vp, f32, i32, vp, vp, vp]
    lib.pgm_beliefs.restype = i32
    lib.pgm_beliefs.argtypes = [vp, vp, vp, vp, i32, vp]
    lib.pgm_decode.restype = i32
    lib.pgm_decode.argtypes = [vp, vp, vp, vp, vp]
    lib.pgm_infer_host.restype = i32
    lib.pgm_infer_host.argtypes = [vp, vp, vp, f32, f32, i32, vp, vp, vp]
    lib.pgm_set_profiling.restype = i32
    lib.pgm_set_profiling.argtypes = [vp, i32]
    lib.pgm_pass_times.restype = i32
    lib.pgm_pass_times.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                   ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    lib.pgm_checked_report.restype = i32
    lib.pgm_checked_report.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
    lib.pgm_audit_desc.restype = i32
    lib.pgm_audit_desc.argtypes = [ctypes.POINTER(GraphDescC), i32, ctypes.c_int64, ctypes.c_int64, ctypes.POINTER(i32),
                                   ctypes.POINTER(ctypes.c_int64)]
    lib.pgm_launch_times.restype = i32
    lib.pgm_launch_times.argtypes = [vp, i32, vp, vp, ctypes.POINTER(i32)]
    lib.pgm_device_flags.restype = i32
    lib.pgm_device_flags.argtypes = [vp, ctypes.POINTER(ctypes.c_uint32), i32, vp]
    lib.pgm_grid2_run_bp_noalloc.restype = i32
    lib.pgm_grid2_run_bp_noalloc.argtypes = [i32, i32, vp, vp, f32, f32, i32, vp, vp]
    lib.pgm_grid2_noalloc_flags.restype = i32
    lib.pgm_grid2_noalloc_flags.argtypes = [ctypes.POINTER(ctypes.c_uint32), i32, vp]
    lib.pgm_autotune.restype = i32
    lib.pgm_autotune.argtypes = [vp, vp, vp, f32, f32, vp]
    lib.pgm_launch_info.restype = i32
    lib.pgm_launch_info.argtypes = [vp, i32] + [ctypes.POINTER(i32)] * 4
    lib.pgm_grad.restype = i32
    lib.pgm_grad.argtypes = [vp, vp, vp, f32, f32, i32, i32, vp, vp, vp, vp]
    lib.pgm_serve_create.restype = i32
    lib.pgm_serve_create.argtypes = [ctypes.POINTER(ServerConfigC), ctypes.POINTER(vp)]
    lib.pgm_serve_submit.restype = i32
    lib.pgm_serve_submit.argtypes = [vp, ctypes.POINTER(GraphDescC), vp, vp, f32, f32, i32, ctypes.POINTER(ctypes.c_int64)]
    lib.pgm_serve_submit_until.restype = i32
    lib.pgm_serve_submit_until.argtypes = [vp, ctypes.POINTER(GraphDescC), vp, vp, f32, f32, i32, f32, i32,
                                           ctypes.POINTER(ctypes.c_int64)]
    lib.pgm_serve_submit_borrowed.restype = i32
    lib.pgm_serve_submit_borrowed.argtypes = [vp, ctypes.POINTER(GraphDescC), vp, vp, f32, f32, i32, f32, i32,
                                              ctypes.POINTER(ctypes.c_int64)]
    lib.pgm_serve_poll.restype = i32
    lib.pgm_serve_poll.argtypes = [vp, ctypes.c_int64, vp, vp, ctypes.POINTER(ctypes.c_double)]
    lib.pgm_serve_wait.restype = i32
    lib.pgm_serve_wait.argtypes = [vp, ctypes.c_int64, ctypes.c_int64, vp, vp, ctypes.POINTER(ctypes.c_double)]
    lib.pgm_serve_stats.restype = i32
    lib.pgm_serve_stats.argtypes = [vp, ctypes.POINTER(ServerStatsC)]
    lib.pgm_serve_destroy.restype = None
    lib.pgm_serve_destroy.argtypes = [vp]
    lib.pgm_set_option.restype = i32
    lib.pgm_set_option.argtypes = [vp, i32, ctypes.c_int64]
    lib.pgm_get_option.restype = i32
    lib.pgm_get_option.argtypes = [vp, i32, vp]
    lib.pgm_last_error.restype = ctypes.c_char_p
    lib.pgm_last_error.argtypes = []
    _lib = lib
    return lib


def check(status: int):
    if status != PGM_OK:
        msg = load_library().pgm_last_error().decode(errors="replace")
        raise PgmError(status, msg)


def marshal_desc(fg):
    """Build a pgm_graph_desc from a workloads.FactorGraph; returns (desc, keepalive)."""
    keep = []

    def arr(a):
        a = np.ascontiguousarray(a, dtype=np.int32)
        if a.size == 0:
            a = np.zeros(1, np.int32)
        keep.append(a)
        return a.ctypes.data

    eg = (EnumGroupC * max(1, len(fg.enum_groups)))()
    for i, g in enumerate(fg.enum_groups):
        eg[i] = EnumGroupC(g.arity, g.n_cfg, arr(g.cfg), g.n_fac, arr(g.vars), int(bool(g.shared)))
    lg = (LogicGroupC * max(1, len(fg.logic_groups)))()
    for i, g in enumerate(fg.logic_groups):
        lg[i] = LogicGroupC(int(g.kind), g.n_fac, arr(g.par_off), arr(g.parents), arr(g.child))
    keep += [eg, lg]
    d = GraphDescC(fg.n_vars, arr(fg.num_states), len(fg.enum_groups),
                   ctypes.cast(eg, ctypes.POINTER(EnumGroupC)), len(fg.logic_groups),
                   ctypes.cast(lg, ctypes.POINTER(LogicGroupC)))
    return d, keep


def check_desc(fg) -> dict:
    """Host-only validation and size report of a workloads.FactorGraph (no GPU)."""
    lib = load_library()
    desc, keep = marshal_desc(fg)
    info = InfoC()
    check(lib.pgm_check_desc(ctypes.byref(desc), ctypes.byref(info)))
    del keep
    return {k: getattr(info, k) for k, _ in InfoC._fields_}


def _stream_ptr(stream=None) -> int:
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _dptr(t, dtype=None, numel=None, name="tensor") -> int:
    import torch
    if t is None:
        return 0
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}")
    if numel is not None and t.numel() != numel:
        raise ValueError(f"{name} must have {numel} elements, has {t.numel()}")
    return int(t.data_ptr())


class Graph:
    """A compiled factor graph resident on the current CUDA device. `fg` is one
    workloads.FactorGraph (pgm_build) or a list of them (pgm_build_batch)."""

    def __init__(self, fg):
        lib = load_library()
        h = ctypes.c_void_p()
        if isinstance(fg, (list, tuple)):
            descs, keeps = zip(*[marshal_desc(x) for x in fg])
            arr = (ctypes.POINTER(GraphDescC) * len(descs))(*[ctypes.pointer(d) for d in descs])
            check(lib.pgm_build_batch(arr, len(descs), ctypes.byref(h)))
            del keeps, arr
        else:
            desc, keep = marshal_desc(fg)
            check(lib.pgm_build(ctypes.byref(desc), ctypes.byref(h)))
            del keep
        self._h = h
        info = InfoC()
        check(lib.pgm_graph_info(h, ctypes.byref(info)))
        self.info = {k: getattr(info, k) for k, _ in InfoC._fields_}

    def member(self, i: int) -> dict:
        """Offsets of member i of a batch (pgm_batch_member)."""
        m = MemberC()
        check(load_library().pgm_batch_member(self._h, int(i), ctypes.byref(m)))
        return {k: getattr(m, k) for k, _ in MemberC._fields_}

    @property
    def handle(self):
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().pgm_free(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # --- calls ---------------------------------------------------------------------
    def new_msgs(self):
        import torch
        return torch.zeros(max(self.info["n_edge_states"], 1), dtype=torch.float32, device="cuda")[: self.info["n_edge_states"]]

    def run_bp_multi(self, log_pot, evidence, T: float, damping: float, n_iters: int, msgs, stream=None):
        """In-place, for S samples at once (pgm_run_bp_multi): evidence [S, n_var_states],
        msgs [S, n_edge_states]; log_pot [n_potentials] (shared) or [S, n_potentials]."""
        import torch
        I = self.info
        S = int(evidence.shape[0]) if evidence.dim() == 2 else 1
        per_sample = log_pot is not None and log_pot.dim() == 2
        if I["n_potentials"]:
            lp = _dptr(log_pot, torch.float32, I["n_potentials"] * (S if per_sample else 1), "log_pot")
        else:
            lp = 0
        check(load_library().pgm_run_bp_multi(
            self._h, S, lp, int(per_sample), _dptr(evidence, torch.float32, S * I["n_var_states"], "evidence"),
            float(T), float(damping), int(n_iters), _dptr(msgs, torch.float32, S * I["n_edge_states"], "msgs"),
            _stream_ptr(stream)))
        return msgs

    def run_bp_until(self, log_pot, evidence, T: float, damping: float, max_iters: int, tol: float,
                     check_every: int, msgs, stream=None):
        """In-place early-exit run (pgm_run_bp_until). Returns (iterations run, last residual)."""
        import torch
        I = self.info
        done, res = ctypes.c_int32(), ctypes.c_float()
        lp = _dptr(log_pot, torch.float32, I["n_potentials"], "log_pot") if I["n_potentials"] else 0
        check(load_library().pgm_run_bp_until(
            self._h, lp, _dptr(evidence, torch.float32, I["n_var_states"], "evidence"), float(T), float(damping),
            int(max_iters), float(tol), int(check_every), _dptr(msgs, torch.float32, I["n_edge_states"], "msgs"),
            ctypes.byref(done), ctypes.byref(res), _stream_ptr(stream)))
        return done.value, res.value

    def run_bp_until_members(self, log_pot, evidence, T: float, damping: float, max_iters: int, tol: float,
                             check_every: int, msgs, stream=None):
        """In-place early exit per batch member (pgm_run_bp_until_members). Returns
        (iterations run [n_members], last residual [n_members]) as numpy arrays."""
        import torch
        I = self.info
        n = I["n_members"]
        done = np.zeros(n, np.int32)
        res = np.zeros(n, np.float32)
        lp = _dptr(log_pot, torch.float32, I["n_potentials"], "log_pot") if I["n_potentials"] else 0
        check(load_library().pgm_run_bp_until_members(
            self._h, lp, _dptr(evidence, torch.float32, I["n_var_states"], "evidence"), float(T), float(damping),
            int(max_iters), float(tol), int(check_every), _dptr(msgs, torch.float32, I["n_edge_states"], "msgs"),
            done.ctypes.data, res.ctypes.data, _stream_ptr(stream)))
        return done, res

    def run_bp_batch(self, log_pot, evidence, T, damping, n_iters, msgs, stream=None):
        """In-place batch run with per-member parameters (pgm_run_bp_batch): T, damping and
        n_iters are sequences of length n_members."""
        import torch
        I = self.info
        n = I["n_members"]
        Ta = np.ascontiguousarray(T, np.float32)
        da = np.ascontiguousarray(damping, np.float32)
        na = np.ascontiguousarray(n_iters, np.int32)
        if Ta.size != n or da.size != n or na.size != n:
            raise ValueError(f"T, damping and n_iters need {n} entries (one per member)")
        lp = _dptr(log_pot, torch.float32, I["n_potentials"], "log_pot") if I["n_potentials"] else 0
        check(load_library().pgm_run_bp_batch(
            self._h, lp, _dptr(evidence, torch.float32, I["n_var_states"], "evidence"), Ta.ctypes.data, da.ctypes.data,
            na.ctypes.data, _dptr(msgs, torch.float32, I["n_edge_states"], "msgs"), _stream_ptr(stream)))
        return msgs

    def pmp_sample(self, log_pot, evidence, noise, damping: float, n_iters: int, stream=None):
        """Perturb-and-max-product samples (pgm_pmp_sample): noise [S, n_var_states].
        Returns (samples [S, n_vars] int32, messages [S, n_edge_states])."""
        import torch
        I = self.info
        S = int(noise.shape[0])
        msgs = torch.empty(S, I["n_edge_states"], dtype=torch.float32, device=noise.device)
        out = torch.empty(S, I["n_vars"], dtype=torch.int32, device=noise.device)
        lp = _dptr(log_pot, torch.float32, I["n_potentials"], "log_pot") if I["n_potentials"] else 0
        check(load_library().pgm_pmp_sample(
            self._h, S, lp, _dptr(evidence, torch.float32, I["n_var_states"], "evidence"),
            _dptr(noise, torch.float32, S * I["n_var_states"], "noise"), float(damping), int(n_iters),
            _dptr(msgs, torch.float32, S * I["n_edge_states"], "msgs"), _dptr(out, torch.int32, S * I["n_vars"], "samples"),
            _stream_ptr(stream)))
        return out, msgs

    def run_bp(self, log_pot, evidence, T: float, damping: float, n_iters: int, msgs, stream=None):
        """In-place: msgs <- n_iters LBP iterations from msgs (pgm_run_bp)."""
        import torch
        I = self.info
        lp = _dptr(log_pot, torch.float32, I["n_potentials"], "log_pot") if I["n_potentials"] else 0
        check(load_library().pgm_run_bp(self._h, lp, _dptr(evidence, torch.float32, I["n_var_states"], "evidence"),
                                        float(T), float(damping), int(n_iters),
                                        _dptr(msgs, torch.float32, I["n_edge_states"], "msgs"),
                                        _stream_ptr(stream)))
        return msgs

    def beliefs(self, evidence, msgs, normalise: bool = True, out=None, stream=None):
        import torch
        I = self.info
        if out is None:
            out = torch.empty(I["n_var_states"], dtype=torch.float32, device="cuda")
        check(load_library().pgm_beliefs(self._h, _dptr(evidence, torch.float32, I["n_var_states"], "evidence"),
                                         _dptr(msgs, torch.float32, I["n_edge_states"], "msgs"),
                                         _dptr(out, torch.float32, I["n_var_states"], "out"),
                                         int(bool(normalise)), _stream_ptr(stream)))
        return out

    def decode(self, evidence, msgs, out=None, stream=None):
        import torch
        I = self.info
        if out is None:
            out = torch.empty(I["n_vars"], dtype=torch.int32, device="cuda")
        check(load_library().pgm_decode(self._h, _dptr(evidence, torch.float32, I["n_var_states"], "evidence"),
                                        _dptr(msgs, torch.float32, I["n_edge_states"], "msgs"),
                                        _dptr(out, torch.int32, I["n_vars"], "out"), _stream_ptr(stream)))
        return out

    def infer_host(self, log_pot: np.ndarray, evidence: np.ndarray, T: float, damping: float,
                   n_iters: int, beliefs: np.ndarray | None = None, decode: np.ndarray | None = None,
                   stream=None):
        """pgm_infer_host on host numpy buffers (pinned numpy views are fastest)."""
        I = self.info
        lp = np.ascontiguousarray(log_pot, np.float32)
        ev = np.ascontiguousarray(evidence, np.float32)
        if lp.size != I["n_potentials"] or ev.size != I["n_var_states"]:
            raise ValueError("log_pot / evidence sizes do not match the graph")
        if beliefs is None:
            beliefs = np.empty(I["n_var_states"], np.float32)
        if decode is None:
            decode = np.empty(I["n_vars"], np.int32)
        check(load_library().pgm_infer_host(self._h, lp.ctypes.data if lp.size else None, ev.ctypes.data,
                                            float(T), float(damping), int(n_iters), beliefs.ctypes.data,
                                            decode.ctypes.data, _stream_ptr(stream)))
        return beliefs, decode

    def autotune(self, log_pot, evidence, T: float, damping: float, stream=None):
        """pgm_autotune: pick the fastest launch shapes on these inputs."""
        import torch
        I = self.info
        lp = _dptr(log_pot, torch.float32, I["n_potentials"], "log_pot") if I["n_potentials"] else 0
        check(load_library().pgm_autotune(self._h, lp, _dptr(evidence, torch.float32, I["n_var_states"], "evidence"),
                                          float(T), float(damping), _stream_ptr(stream)))

    def launches(self) -> list:
        """[(kind, variant, threads, blocks)] of one iteration (pgm_launch_info)."""
        out = []
        for i in range(self.info["launches_per_iter"]):
            v = [ctypes.c_int32() for _ in range(4)]
            check(load_library().pgm_launch_info(self._h, i, *[ctypes.byref(x) for x in v]))
            out.append(tuple(x.value for x in v))
        return out

    def grad(self, log_pot, evidence, T: float, damping: float, n_iters: int, ckpt_every: int, d_beliefs,
             stream=None):
        """pgm_grad: (d_log_pot, d_evidence) of sum(d_beliefs * normalised log-beliefs)."""
        import torch
        I = self.info
        d_lp = torch.empty(max(I["n_potentials"], 1), dtype=torch.float32, device="cuda")[: I["n_potentials"]]
        d_ev = torch.empty(I["n_var_states"], dtype=torch.float32, device="cuda")
        lp = _dptr(log_pot, torch.float32, I["n_potentials"], "log_pot") if I["n_potentials"] else 0
        check(load_library().pgm_grad(self._h, lp, _dptr(evidence, torch.float32, I["n_var_states"], "evidence"),
                                      float(T), float(damping), int(n_iters), int(ckpt_every),
                                      _dptr(d_beliefs, torch.float32, I["n_var_states"], "d_beliefs"),
                                      _dptr(d_lp, torch.float32, I["n_potentials"], "d_log_pot") if I["n_potentials"] else 0,
                                      _dptr(d_ev, torch.float32, I["n_var_states"], "d_evidence"), _stream_ptr(stream)))
        return d_lp, d_ev

    def set_option(self, option: int, value: int):
        check(load_library().pgm_set_option(self._h, int(option), int(value)))

    def get_option(self, option: int) -> int:
        """Effective value of an option (pgm_get_option)."""
        v = ctypes.c_int64()
        check(load_library().pgm_get_option(self._h, int(option), ctypes.byref(v)))
        return int(v.value)

    def set_profiling(self, period: int):
        """Record per-pass CUDA events every `period` iterations (0 = off)."""
        check(load_library().pgm_set_profiling(self._h, int(period)))

    def pass_times(self):
        """(variable-pass ms, factor-pass ms, variable launches, factor launches) since the
        last call, from CUDA events recorded on the launching stream."""
        tv, tf = ctypes.c_double(), ctypes.c_double()
        nv, nf = ctypes.c_int64(), ctypes.c_int64()
        check(load_library().pgm_pass_times(self._h, ctypes.byref(tv), ctypes.byref(tf), ctypes.byref(nv), ctypes.byref(nf)))
        return tv.value, tf.value, nv.value, nf.value

    def launch_times(self, n: int = 32):
        """[(summed ms, sampled launches)] per launch position of the sampled iterations
        since the last call (pgm_launch_times), from CUDA events on the launching stream."""
        ms = np.zeros(max(n, 1), np.float64)
        cnt = np.zeros(max(n, 1), np.int64)
        npos = ctypes.c_int32(0)
        check(load_library().pgm_launch_times(self._h, int(n), ms.ctypes.data, cnt.ctypes.data, ctypes.byref(npos)))
        k = min(int(npos.value), n)
        return [(float(ms[i]), int(cnt[i])) for i in range(k)]

    def checked_report(self):
        """(array id, position, value) of the first checked-mode violation, array -1 if none."""
        a, pos, val = ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
        check(load_library().pgm_checked_report(self._h, ctypes.byref(a), ctypes.byref(pos), ctypes.byref(val)))
        return a.value, pos.value, val.value

    def flags(self, clear: bool = False, stream=None) -> int:
        f = ctypes.c_uint32(0)
        check(load_library().pgm_device_flags(self._h, ctypes.byref(f), int(bool(clear)), _stream_ptr(stream)))
        return int(f.value)


NOALLOC_SCRATCH_FLOATS = 4194304


def grid2_run_bp_noalloc(rows: int, cols: int, log_pot, evidence, T: float, damping: float,
                         n_iters: int, msgs, stream=None):
    """pgm_grid2_run_bp_noalloc: in-place LBP on a rows x cols binary grid with caller-owned
    CUDA tensors and no device allocation by the library (scratch in a static array)."""
    import torch
    F = rows * (cols - 1) + (rows - 1) * cols
    check(load_library().pgm_grid2_run_bp_noalloc(
        int(rows), int(cols), _dptr(log_pot, torch.float32, 4 * F, "log_pot") if F else 0,
        _dptr(evidence, torch.float32, 2 * rows * cols, "evidence"), float(T), float(damping),
        int(n_iters), _dptr(msgs, torch.float32, 4 * F, "msgs") if F else 0, _stream_ptr(stream)))
    return msgs


def audit_desc(fg, corrupt_array: int = -1, corrupt_pos: int = 0, corrupt_value: int = 0):
    """pgm_audit_desc: the checked-mode range checks run on the host copies of a
    description's index arrays (optionally after corrupting one entry). Returns (array,
    position) of the first violation, (-1, -1) if none. No GPU needed."""
    desc, keep = marshal_desc(fg)
    a, pos = ctypes.c_int32(), ctypes.c_int64()
    check(load_library().pgm_audit_desc(ctypes.byref(desc), int(corrupt_array), int(corrupt_pos), int(corrupt_value),
                                        ctypes.byref(a), ctypes.byref(pos)))
    del keep
    return a.value, pos.value


def grid2_noalloc_flags(clear: bool = False, stream=None) -> int:
    """pgm_grid2_noalloc_flags: the PGM_FLAG_* bits of the last allocation-free grid call
    on the current device (synchronises the stream)."""
    f = ctypes.c_uint32(0)
    check(load_library().pgm_grid2_noalloc_flags(ctypes.byref(f), int(bool(clear)), _stream_ptr(stream)))
    return int(f.value)


def infer(problem, n_iters: int | None = None, T: float | None = None, graph: Graph | None = None):
    """Cold-start LBP on a workloads.Problem on the GPU. Returns (graph, msgs,
    normalised log-beliefs, decode) as CUDA tensors."""
    import torch
    g = graph or Graph(problem.graph)
    lp = torch.as_tensor(problem.log_pot, dtype=torch.float32).cuda()
    ev = torch.as_tensor(problem.evidence, dtype=torch.float32).cuda()
    msgs = g.new_msgs()
    g.run_bp(lp, ev, problem.T if T is None else T, problem.damping,
             problem.n_iters if n_iters is None else n_iters, msgs)
    return g, msgs, g.beliefs(ev, msgs, True), g.decode(ev, msgs)


def _lbp_function():
    import torch

    class LBPFunction(torch.autograd.Function):
        """Normalised log-beliefs after n_iters LBP iterations from zero messages, as a
        differentiable function of (log_pot, evidence): forward through pgm_run_bp and
        pgm_beliefs, backward through pgm_grad (checkpoint every ckpt_every iterations)."""

        @staticmethod
        def forward(ctx, log_pot, evidence, graph, T, damping, n_iters, ckpt_every):
            lp = log_pot.detach().contiguous()
            ev = evidence.detach().contiguous()
            msgs = graph.new_msgs()
            graph.run_bp(lp, ev, T, damping, n_iters, msgs)
            nb = graph.beliefs(ev, msgs, True)
            ctx.save_for_backward(lp, ev)
            ctx.cfg = (graph, T, damping, n_iters, ckpt_every)
            return nb

        @staticmethod
        def backward(ctx, g):
            lp, ev = ctx.saved_tensors
            graph, T, damping, n_iters, ckpt_every = ctx.cfg
            d_lp, d_ev = graph.grad(lp, ev, T, damping, n_iters, ckpt_every, g.contiguous())
            return d_lp, d_ev, None, None, None, None, None

    return LBPFunction


_LBP = None


def lbp_beliefs(log_pot, evidence, graph: Graph, T: float, damping: float, n_iters: int, ckpt_every: int = 10):
    """Differentiable normalised log-beliefs (torch.autograd.Function over the C ABI)."""
    global _LBP
    if _LBP is None:
        _LBP = _lbp_function()
    return _LBP.apply(log_pot, evidence, graph, T, damping, n_iters, ckpt_every)


class Server:
    """The serving loop (pgm_serve_*): submit requests, poll or wait for results."""

    def __init__(self, memory_budget_bytes: int, max_in_flight: int, max_pending: int = 1 << 20):
        lib = load_library()
        cfg = ServerConfigC(int(memory_budget_bytes), int(max_in_flight), int(max_pending))
        h = ctypes.c_void_p()
        check(lib.pgm_serve_create(ctypes.byref(cfg), ctypes.byref(h)))
        self._h = h
        self._shapes = {}
        self._borrowed = {}  # request id -> what a borrowed submission points into

    def submit(self, fg, log_pot, evidence, T: float, damping: float, n_iters: int, desc=None,
               tol=None, check_every: int = 10, borrow: bool = False) -> int:
        """Queue a request. `desc` may be a (desc, keepalive) pair from marshal_desc(fg),
        reused across submissions of the same graph. With `tol`, the request stops early
        (pgm_serve_submit_until: n_iters is the limit, the residual is checked every
        `check_every` iterations). With `borrow`, nothing is copied
        (pgm_serve_submit_borrowed): the server keeps references to the description and
        arrays until the result is taken."""
        desc, keep = desc if desc is not None else marshal_desc(fg)
        lp = np.ascontiguousarray(log_pot, np.float32)
        ev = np.ascontiguousarray(evidence, np.float32)
        rid = ctypes.c_int64()
        lib = load_library()
        lpp = lp.ctypes.data if lp.size else None
        if borrow:
            check(lib.pgm_serve_submit_borrowed(self._h, ctypes.byref(desc), lpp, ev.ctypes.data, float(T),
                                                float(damping), int(n_iters), 0.0 if tol is None else float(tol),
                                                0 if tol is None else int(check_every), ctypes.byref(rid)))
            self._borrowed[rid.value] = (desc, keep, lp, ev)  # alive until the result is taken
        elif tol is None:
            check(lib.pgm_serve_submit(self._h, ctypes.byref(desc), lpp, ev.ctypes.data, float(T), float(damping),
                                       int(n_iters), ctypes.byref(rid)))
        else:
            check(lib.pgm_serve_submit_until(self._h, ctypes.byref(desc), lpp, ev.ctypes.data, float(T),
                                             float(damping), int(n_iters), float(tol), int(check_every),
                                             ctypes.byref(rid)))
        del keep
        self._shapes[rid.value] = (fg.n_var_states, fg.n_vars)
        return rid.value

    def _result(self, fn, rid, *args):
        VS, V = self._shapes[rid]
        bel = np.empty(VS, np.float32)
        dec = np.empty(V, np.int32)
        lat = ctypes.c_double()
        st = fn(self._h, ctypes.c_int64(rid), *args, bel.ctypes.data, dec.ctypes.data, ctypes.byref(lat))
        if st == -5:
            return None
        if st != -6:  # a timed-out request is still pending
            self._shapes.pop(rid, None)
            self._borrowed.pop(rid, None)
        check(st)
        return bel, dec, lat.value

    def poll(self, rid: int):
        """(beliefs, decode, latency_s) when done, else None."""
        return self._result(load_library().pgm_serve_poll, rid)

    def wait(self, rid: int, timeout_s: float):
        return self._result(load_library().pgm_serve_wait, rid, ctypes.c_int64(int(timeout_s * 1e6)))

    def stats(self) -> dict:
        st = ServerStatsC()
        check(load_library().pgm_serve_stats(self._h, ctypes.byref(st)))
        return {k: getattr(st, k) for k, _ in ServerStatsC._fields_}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            load_library().pgm_serve_destroy(self._h)
            self._h = ctypes.c_void_p()
        if hasattr(self, "_borrowed"):
            self._borrowed.clear()  # the server no longer reads them

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
