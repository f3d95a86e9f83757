"""GB300 DLMPC solver: Python binding of the C ABI in include/dlmpc.h.

The binding only marshals arguments: every step of the solver runs in the
CUDA library `libdlmpc.so` built in-tree by `paper_2103_14990_gb300.build`.
PyTorch supplies device memory and streams.  There is no CPU fallback: if the
library is missing, `load_library()` raises.
"""
from __future__ import annotations

import ctypes
import os
from typing import List, Optional, Sequence

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdlmpc.so")

DLMPC_OK = 0
DLMPC_MAX_ITER = 1
DLMPC_ERR_ARG = -1
DLMPC_ERR_INFEASIBLE_LOCALITY = -2
DLMPC_ERR_NONFINITE = -3
DLMPC_ERR_TIMEOUT = -4
DLMPC_ERR_CUDA = -5
DLMPC_ERR_NOMEM = -6
DLMPC_ERR_CAPACITY = -7
DLMPC_MAX_COUPLED = 4      # coupled rows per subsystem and slot kind
DLMPC_MAX_REGIONS = 1024   # explicit-solution regions per subsystem and slot kind

WARM_COLD = 0
WARM_PREVIOUS = 1
WARM_LEARNED = 2
WARM_CONVERGED = 3

OPT_FIXED_ITERS = 1
OPT_MAX_ITER = 2
OPT_TIMEOUT_MS = 3
OPT_EXPORT_PHI = 4
OPT_SWEEP_SHAPE = 5
OPT_TIMING = 7
OPT_RESIDENCY = 8
OPT_TRACE = 9
OPT_GRAPH = 10
OPT_LEARN_PLANT = 11
OPT_TEST_SKIP_ARRIVAL = 12
OPT_COMPACT = 13
OPT_BLOCK_PHI = 14
OPT_STALE_PROB = 15
OPT_STALE_SEED = 16

# Every entry point declared in include/dlmpc.h (checked by the tests).
EXPORTED = [
    "dlmpc_setup", "dlmpc_precompute", "dlmpc_update_plant", "dlmpc_step", "dlmpc_solve_batch", "dlmpc_step_host",
    "dlmpc_set_option", "dlmpc_get_info", "dlmpc_get_state", "dlmpc_set_state",
    "dlmpc_get_patch", "dlmpc_get_operator", "dlmpc_get_timing", "dlmpc_get_trace", "dlmpc_last_error",
    "dlmpc_destroy", "dlmpc_autotune",
    "dlmpc_mlp_create", "dlmpc_mlp_num_params", "dlmpc_mlp_set_params", "dlmpc_mlp_get_params",
    "dlmpc_mlp_forward", "dlmpc_mlp_gradients", "dlmpc_mlp_train_step", "dlmpc_mlp_last_error",
    "dlmpc_mlp_destroy", "dlmpc_learned_dims", "dlmpc_learned_features", "dlmpc_learned_targets",
    "dlmpc_attach_mlp", "dlmpc_run_variant",
    "dlmpc_factor_patch_noalloc",
    "dlmpc_export_operators", "dlmpc_import_operators",
]

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)


class Problem_C(ctypes.Structure):
    _fields_ = [("n_sub", ctypes.c_int32), ("nx", ctypes.c_int32), ("nu", ctypes.c_int32),
                ("T", ctypes.c_int32), ("d", ctypes.c_int32),
                ("adj_ptr", _ip), ("adj_idx", _ip),
                ("A_diag", _dp), ("A_off", _dp), ("B", _dp), ("q", _dp), ("r", _dp),
                ("x_lo", _dp), ("x_hi", _dp), ("u_lo", _dp), ("u_hi", _dp),
                ("rho", ctypes.c_double), ("eps_p", ctypes.c_double), ("eps_d", ctypes.c_double),
                ("max_iter", ctypes.c_int32), ("Q_blk", _dp), ("R_blk", _dp),
                ("n_cx", ctypes.c_int32), ("n_cu", ctypes.c_int32),
                ("Gx", _dp), ("gx", _dp), ("Gu", _dp), ("gu", _dp)]


class Stats_C(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("status", ctypes.c_int32),
                ("r_max", ctypes.c_float), ("s_max", ctypes.c_float)]


class TuneEntry_C(ctypes.Structure):
    _fields_ = [("group_threads", ctypes.c_int32), ("groups_per_cta", ctypes.c_int32), ("wave", ctypes.c_int32),
                ("residency", ctypes.c_int32), ("ms", ctypes.c_float)]


class Info_C(ctypes.Structure):
    _fields_ = [("n_inst", ctypes.c_int32), ("n_sub_total", ctypes.c_int32), ("nx", ctypes.c_int32),
                ("nu", ctypes.c_int32), ("n_items", ctypes.c_int32), ("max_dcol", ctypes.c_int32),
                ("max_nullity", ctypes.c_int32), ("state_floats", ctypes.c_int64),
                ("operator_bytes", ctypes.c_int64), ("offset_bytes", ctypes.c_int64),
                ("exchange_floats", ctypes.c_int64), ("grid_ctas", ctypes.c_int32),
                ("threads_per_cta", ctypes.c_int32), ("smem_bytes", ctypes.c_int32),
                ("group_threads", ctypes.c_int32), ("groups_per_cta", ctypes.c_int32), ("wave", ctypes.c_int32),
                ("resident_n_items", ctypes.c_int32), ("resident_state_items", ctypes.c_int32),
                ("iter_bytes", ctypes.c_int64), ("iter_bytes_min", ctypes.c_int64)]


_LIB = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libdlmpc.so (raises if it has not been built)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: run paper_2103_14990_gb300.build.build() first "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    vp, fp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_float)
    lib.dlmpc_setup.argtypes = [ctypes.POINTER(Problem_C), ctypes.c_int32, vp, ctypes.POINTER(vp)]
    lib.dlmpc_precompute.argtypes = [vp]
    lib.dlmpc_update_plant.argtypes = [vp, ctypes.c_int32, _ip, _dp, _dp, _dp]
    lib.dlmpc_export_operators.argtypes = [vp, vp, ctypes.c_int64]
    lib.dlmpc_export_operators.restype = ctypes.c_int64
    lib.dlmpc_import_operators.argtypes = [vp, ctypes.c_void_p, ctypes.c_int64]
    lib.dlmpc_step.argtypes = [vp, vp, vp, vp, ctypes.c_int32, ctypes.POINTER(Stats_C)]
    lib.dlmpc_step_host.argtypes = [vp, fp, fp, fp, ctypes.c_int32, ctypes.POINTER(Stats_C)]
    lib.dlmpc_solve_batch.argtypes = [vp, ctypes.POINTER(vp), ctypes.POINTER(vp), ctypes.POINTER(vp),
                                      ctypes.c_int32, ctypes.POINTER(Stats_C)]
    lib.dlmpc_set_option.argtypes = [vp, ctypes.c_int32, ctypes.c_double]
    lib.dlmpc_get_info.argtypes = [vp, ctypes.POINTER(Info_C)]
    lib.dlmpc_get_state.argtypes = [vp, vp, vp, vp]
    lib.dlmpc_set_state.argtypes = [vp, vp, vp]
    lib.dlmpc_get_patch.argtypes = [vp, ctypes.c_int32, _ip, ctypes.c_int32]
    lib.dlmpc_get_operator.argtypes = [vp, ctypes.c_int32, _dp, ctypes.c_int32, _dp, ctypes.c_int32]
    lib.dlmpc_get_timing.argtypes = [vp, ctypes.POINTER(ctypes.c_float)]
    lib.dlmpc_mlp_create.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, vp, ctypes.POINTER(vp)]
    lib.dlmpc_mlp_num_params.argtypes = [vp]
    lib.dlmpc_mlp_num_params.restype = ctypes.c_int64
    lib.dlmpc_mlp_set_params.argtypes = [vp, fp, ctypes.c_int64, fp, fp]
    lib.dlmpc_mlp_get_params.argtypes = [vp, fp, ctypes.c_int64]
    lib.dlmpc_mlp_forward.argtypes = [vp, vp, ctypes.c_int32, vp]
    lib.dlmpc_mlp_gradients.argtypes = [vp, vp, vp, ctypes.c_int32, fp, ctypes.POINTER(ctypes.c_double)]
    lib.dlmpc_mlp_train_step.argtypes = [vp, vp, vp, ctypes.c_int32, ctypes.c_float, ctypes.c_float,
                                         ctypes.POINTER(ctypes.c_double)]
    lib.dlmpc_mlp_last_error.argtypes = [vp]
    lib.dlmpc_mlp_last_error.restype = ctypes.c_char_p
    lib.dlmpc_mlp_destroy.argtypes = [vp]
    lib.dlmpc_mlp_destroy.restype = None
    lib.dlmpc_learned_dims.argtypes = [vp, ctypes.POINTER(ctypes.c_int32), ctypes.POINTER(ctypes.c_int32)]
    lib.dlmpc_learned_features.argtypes = [vp, vp, vp]
    lib.dlmpc_learned_targets.argtypes = [vp, vp]
    lib.dlmpc_attach_mlp.argtypes = [vp, vp]
    lib.dlmpc_run_variant.argtypes = [vp, ctypes.c_int32, vp, ctypes.c_int32, ctypes.c_int32,
                                      ctypes.POINTER(ctypes.c_double)]
    lib.dlmpc_autotune.argtypes = [vp, vp, ctypes.c_int32, ctypes.POINTER(TuneEntry_C), ctypes.c_int32]
    lib.dlmpc_get_trace.argtypes = [vp, ctypes.POINTER(ctypes.c_uint64), ctypes.c_int64]
    lib.dlmpc_last_error.argtypes = [vp]
    lib.dlmpc_last_error.restype = ctypes.c_char_p
    lib.dlmpc_destroy.argtypes = [vp]
    lib.dlmpc_destroy.restype = None
    lib.dlmpc_factor_patch_noalloc.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, vp, ctypes.c_int32, vp,
                                               ctypes.c_int32, vp, vp, vp, vp]
    _LIB = lib
    return lib


class DlmpcError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"dlmpc error {code}: {msg}")
        self.code = code


def _ptr(a: Optional[np.ndarray], ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


class Solver:
    """One context of n_inst >= 1 instances (see include/dlmpc.h).

    problems: list of `instances.Problem`.  stream: a torch.cuda.Stream or None
    (current stream)."""

    def __init__(self, problems, stream=None, precompute: bool = True):
        import torch
        if not isinstance(problems, (list, tuple)):
            problems = [problems]
        self.lib = load_library()
        self.problems = list(problems)
        self.torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._keep = []
        arr = (Problem_C * len(problems))()
        for k, p in enumerate(problems):
            arr[k] = self._marshal(p)
        self._ctx = ctypes.c_void_p()
        rc = self.lib.dlmpc_setup(arr, len(problems), ctypes.c_void_p(self.stream.cuda_stream),
                                  ctypes.byref(self._ctx))
        if rc != 0:
            raise DlmpcError(rc, self.lib.dlmpc_last_error(None).decode())
        self.nx, self.nu = problems[0].nx, problems[0].nu
        self.n_sub = sum(p.n_sub for p in problems)
        self.sub_off = np.cumsum([0] + [p.n_sub for p in problems])
        if precompute:
            self.precompute()

    def _marshal(self, p) -> Problem_C:
        def keep(a, dt):
            if a is None:
                return None
            a = np.ascontiguousarray(a, dtype=dt)
            self._keep.append(a)
            return a
        c = Problem_C()
        c.n_sub, c.nx, c.nu, c.T, c.d = p.n_sub, p.nx, p.nu, p.T, p.d
        c.adj_ptr = _ptr(keep(p.adj_ptr, np.int32), ctypes.c_int32)
        c.adj_idx = _ptr(keep(p.adj_idx if len(p.adj_idx) else np.zeros(1), np.int32), ctypes.c_int32)
        c.A_diag = _ptr(keep(p.A_diag, np.float64), ctypes.c_double)
        c.A_off = _ptr(keep(p.A_off if len(p.A_off) else np.zeros((1, p.nx, p.nx)), np.float64), ctypes.c_double)
        c.B = _ptr(keep(p.B, np.float64), ctypes.c_double)
        c.q = _ptr(keep(p.q, np.float64), ctypes.c_double)
        c.r = _ptr(keep(p.r, np.float64), ctypes.c_double)
        c.x_lo = _ptr(keep(p.x_lo, np.float64), ctypes.c_double)
        c.x_hi = _ptr(keep(p.x_hi, np.float64), ctypes.c_double)
        c.u_lo = _ptr(keep(p.u_lo, np.float64), ctypes.c_double)
        c.u_hi = _ptr(keep(p.u_hi, np.float64), ctypes.c_double)
        c.rho, c.eps_p, c.eps_d, c.max_iter = p.rho, p.eps_p, p.eps_d, p.max_iter
        c.Q_blk = _ptr(keep(getattr(p, "Q_blk", None), np.float64), ctypes.c_double)
        c.R_blk = _ptr(keep(getattr(p, "R_blk", None), np.float64), ctypes.c_double)
        Gx, Gu = getattr(p, "Gx", None), getattr(p, "Gu", None)
        c.n_cx = 0 if Gx is None else int(Gx.shape[1])
        c.n_cu = 0 if Gu is None else int(Gu.shape[1])
        c.Gx = _ptr(keep(Gx, np.float64), ctypes.c_double)
        c.gx = _ptr(keep(getattr(p, "gx", None) if Gx is not None else None, np.float64), ctypes.c_double)
        c.Gu = _ptr(keep(Gu, np.float64), ctypes.c_double)
        c.gu = _ptr(keep(getattr(p, "gu", None) if Gu is not None else None, np.float64), ctypes.c_double)
        return c

    def _check(self, rc: int) -> int:
        if rc < 0:
            raise DlmpcError(rc, self.lib.dlmpc_last_error(self._ctx).decode())
        return rc

    def precompute(self):
        self._check(self.lib.dlmpc_precompute(self._ctx))

    def update_plant(self, subsystems, A_diag, A_off, B) -> int:
        """New A_ii, A_ij (CSR rows of the changed subsystems, concatenated)
        and B_i for the listed global subsystems; re-factorises the patches
        that see them.  Returns the number of patches re-factorised."""
        sub = np.ascontiguousarray(subsystems, np.int32)
        ad = np.ascontiguousarray(A_diag, np.float64)
        ao = np.ascontiguousarray(A_off, np.float64) if A_off is not None and np.size(A_off) else None
        bb = np.ascontiguousarray(B, np.float64)
        return self._check(self.lib.dlmpc_update_plant(self._ctx, len(sub), _ptr(sub, ctypes.c_int32),
                                                       _ptr(ad, ctypes.c_double), _ptr(ao, ctypes.c_double),
                                                       _ptr(bb, ctypes.c_double)))

    def export_operators(self) -> bytes:
        """The precomputed operators as a blob (see dlmpc_import_operators)."""
        n = self._check(int(self.lib.dlmpc_export_operators(self._ctx, None, 0)))
        buf = ctypes.create_string_buffer(n)
        m = self._check(int(self.lib.dlmpc_export_operators(self._ctx, buf, n)))
        return buf.raw[:m]

    def import_operators(self, blob: bytes):
        """Replaces precompute() on a solver built with precompute=False."""
        self._check(self.lib.dlmpc_import_operators(self._ctx, blob, len(blob)))

    def set_option(self, key: int, value: float):
        self._check(self.lib.dlmpc_set_option(self._ctx, key, float(value)))

    def info(self) -> dict:
        i = Info_C()
        self._check(self.lib.dlmpc_get_info(self._ctx, ctypes.byref(i)))
        return {f: getattr(i, f) for f, _ in Info_C._fields_}

    def step(self, x, u, x_next=None, warm: int = WARM_COLD, stats: bool = True):
        """x, u, x_next: contiguous float32 CUDA tensors [n_sub, nx] / [n_sub, nu]."""
        st = (Stats_C * len(self.problems))() if stats else None
        rc = self._check(self.lib.dlmpc_step(self._ctx, ctypes.c_void_p(x.data_ptr()),
                                             ctypes.c_void_p(u.data_ptr()),
                                             ctypes.c_void_p(x_next.data_ptr()) if x_next is not None else None,
                                             warm, st))
        if not stats:
            return rc, None
        return rc, [dict(iters=s.iters, status=s.status, r_max=s.r_max, s_max=s.s_max) for s in st]

    def step_host(self, x: np.ndarray, warm: int = WARM_COLD, want_next: bool = True):
        """Host-buffer step: returns (rc, u, x_next, stats)."""
        xf = np.ascontiguousarray(x, dtype=np.float32).reshape(-1)
        u = np.zeros(self.n_sub * self.nu, np.float32)
        xn = np.zeros(self.n_sub * self.nx, np.float32) if want_next else None
        st = (Stats_C * len(self.problems))()
        fp = ctypes.POINTER(ctypes.c_float)
        rc = self._check(self.lib.dlmpc_step_host(self._ctx, _ptr(xf, ctypes.c_float), _ptr(u, ctypes.c_float),
                                                  _ptr(xn, ctypes.c_float) if xn is not None else None, warm, st))
        return rc, u, xn, [dict(iters=s.iters, status=s.status, r_max=s.r_max, s_max=s.s_max) for s in st]

    def step_host_ptr(self, x_addr: int, u_addr: int, xn_addr: Optional[int], warm: int = WARM_COLD):
        """Host-buffer step on raw host addresses (e.g. pinned torch tensors)."""
        st = (Stats_C * len(self.problems))()
        fp = ctypes.POINTER(ctypes.c_float)
        rc = self._check(self.lib.dlmpc_step_host(self._ctx, ctypes.cast(x_addr, fp), ctypes.cast(u_addr, fp),
                                                  ctypes.cast(xn_addr, fp) if xn_addr else None, warm, st))
        return rc, [dict(iters=s.iters, status=s.status, r_max=s.r_max, s_max=s.s_max) for s in st]

    def solve_batch(self, xs: Sequence, us: Sequence, xns: Optional[Sequence] = None, warm: int = WARM_COLD):
        n = len(self.problems)
        vp = ctypes.c_void_p
        X = (vp * n)(*[vp(t.data_ptr()) for t in xs])
        U = (vp * n)(*[vp(t.data_ptr()) for t in us])
        XN = (vp * n)(*[vp(t.data_ptr()) for t in xns]) if xns is not None else None
        st = (Stats_C * n)()
        rc = self._check(self.lib.dlmpc_solve_batch(self._ctx, X, U, XN, warm, st))
        return rc, [dict(iters=s.iters, status=s.status, r_max=s.r_max, s_max=s.s_max) for s in st]

    def timing(self):
        """(sweep kernel ms, whole step ms) of the last step (needs OPT_TIMING)."""
        ms = (ctypes.c_float * 2)()
        self._check(self.lib.dlmpc_get_timing(self._ctx, ms))
        return float(ms[0]), float(ms[1])

    def autotune(self, x, iters: int = 20):
        """Times every feasible sweep launch shape on `x` (CUDA tensor) and keeps
        the fastest; returns the measured table (fastest first).  `iters` near
        the steps' own iteration count weighs each plan's one-time prologue as
        the steps will."""
        cap = 512
        arr = (TuneEntry_C * cap)()
        n = self._check(self.lib.dlmpc_autotune(self._ctx, ctypes.c_void_p(x.data_ptr()), iters, arr, cap))
        out = [{f: getattr(arr[i], f) for f, _ in TuneEntry_C._fields_} for i in range(min(n, cap))]
        return sorted(out, key=lambda e: e["ms"])

    def learned_dims(self):
        a, o = ctypes.c_int32(), ctypes.c_int32()
        self._check(self.lib.dlmpc_learned_dims(self._ctx, ctypes.byref(a), ctypes.byref(o)))
        return a.value, o.value

    def learned_features(self, x):
        d_in, _ = self.learned_dims()
        out = self.torch.empty(self.n_sub, d_in, dtype=self.torch.float32, device="cuda")
        self._check(self.lib.dlmpc_learned_features(self._ctx, ctypes.c_void_p(x.data_ptr()),
                                                    ctypes.c_void_p(out.data_ptr())))
        return out

    def learned_targets(self):
        """Phi rows then Lambda rows of every subsystem from the last step
        (needs OPT_EXPORT_PHI during that step)."""
        _, d_out = self.learned_dims()
        out = self.torch.empty(self.n_sub, d_out, dtype=self.torch.float32, device="cuda")
        self._check(self.lib.dlmpc_learned_targets(self._ctx, ctypes.c_void_p(out.data_ptr())))
        return out

    def attach_mlp(self, mlp):
        self._mlp = mlp
        self._check(self.lib.dlmpc_attach_mlp(self._ctx, mlp._h if mlp is not None else None))

    def run_variant(self, variant: int, x, iters: int, warm: int = WARM_COLD) -> float:
        """Paper mapping ablation (0 naive, 1 combined, 2 persistent sweep); host ms."""
        ms = ctypes.c_double()
        self._check(self.lib.dlmpc_run_variant(self._ctx, variant, ctypes.c_void_p(x.data_ptr()), iters, warm,
                                               ctypes.byref(ms)))
        return ms.value

    def trace(self) -> np.ndarray:
        """[ctas, 8 iterations, 8 points] globaltimer stamps (ns) of the last step."""
        cap = 1 << 20
        buf = np.zeros(cap, np.uint64)
        n = self._check(self.lib.dlmpc_get_trace(self._ctx, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)), cap))
        return buf[:n * 64].reshape(n, 8, 8)

    def get_state(self, phi: bool = False):
        torch = self.torch
        nf = self.info()["state_floats"]
        out = [torch.empty(nf, dtype=torch.float32, device="cuda") for _ in range(3)]
        self._check(self.lib.dlmpc_get_state(self._ctx, ctypes.c_void_p(out[0].data_ptr()) if phi else None,
                                             ctypes.c_void_p(out[1].data_ptr()),
                                             ctypes.c_void_p(out[2].data_ptr())))
        return (out[0] if phi else None), out[1], out[2]

    def set_state(self, psi, lam):
        self._check(self.lib.dlmpc_set_state(self._ctx, ctypes.c_void_p(psi.data_ptr()),
                                             ctypes.c_void_p(lam.data_ptr())))

    def patch(self, j: int) -> np.ndarray:
        n = self._check(self.lib.dlmpc_get_patch(self._ctx, j, None, 0))
        out = np.zeros(n, np.int32)
        self._check(self.lib.dlmpc_get_patch(self._ctx, j, _ptr(out, ctypes.c_int32), n))
        return out

    def operator(self, j: int):
        """(N [D_col, k], q [nx, D_col]) of column patch j, full variable order."""
        n_mem = len(self.patch(j))
        inst = int(np.searchsorted(self.sub_off, j, side="right") - 1)
        p = self.problems[inst]
        dcol = p.r_sub * n_mem
        N = np.zeros(dcol * dcol)
        q = np.zeros(self.nx * dcol)
        k = self._check(self.lib.dlmpc_get_operator(self._ctx, j, _ptr(N, ctypes.c_double), dcol * dcol,
                                                    _ptr(q, ctypes.c_double), self.nx * dcol))
        return N[:dcol * k].reshape(dcol, k), q.reshape(self.nx, dcol)

    def close(self):
        if getattr(self, "_ctx", None) is not None and self._ctx.value:
            self.lib.dlmpc_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MLP:
    """The warm-start network of the C ABI (x -> GELU -> GELU -> linear), BF16
    tensor-core GEMMs, FP32 masters, AdamW.  Parameters are initialised here
    (seeded, uniform +-1/sqrt(fan_in), zero biases) and uploaded."""

    def __init__(self, d_in: int, hidden: int, d_out: int, stream=None, seed: int = 0):
        import torch
        self.lib = load_library()
        self.torch = torch
        self.d_in, self.hidden, self.d_out = d_in, hidden, d_out
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self._h = ctypes.c_void_p()
        rc = self.lib.dlmpc_mlp_create(d_in, hidden, d_out, ctypes.c_void_p(self.stream.cuda_stream),
                                       ctypes.byref(self._h))
        if rc != 0:
            raise DlmpcError(rc, "dlmpc_mlp_create failed")
        self.n_params = int(self.lib.dlmpc_mlp_num_params(self._h))
        rng = np.random.default_rng(seed)
        parts = []
        for fan_in, fan_out in [(d_in, hidden), (hidden, hidden), (hidden, d_out)]:
            lim = 1.0 / np.sqrt(fan_in)
            parts.append(rng.uniform(-lim, lim, fan_in * fan_out))
            parts.append(np.zeros(fan_out))
        self.set_params(np.concatenate(parts).astype(np.float32))

    def _check(self, rc):
        if rc < 0:
            raise DlmpcError(rc, self.lib.dlmpc_mlp_last_error(self._h).decode())
        return rc

    def unpack(self, p):
        """dict W1, b1, W2, b2, W3, b3 (views) of a flat parameter vector."""
        I, H, O = self.d_in, self.hidden, self.d_out
        out, o = {}, 0
        for name, shape in [("W1", (I, H)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (H, O)), ("b3", (O,))]:
            n = int(np.prod(shape))
            out[name] = p[o:o + n].reshape(shape)
            o += n
        return out

    def set_params(self, params, scale=None, shift=None):
        p = np.ascontiguousarray(params, np.float32)
        fp = ctypes.POINTER(ctypes.c_float)
        sc = np.ascontiguousarray(scale, np.float32) if scale is not None else None
        sh = np.ascontiguousarray(shift, np.float32) if shift is not None else None
        self._check(self.lib.dlmpc_mlp_set_params(self._h, _ptr(p, ctypes.c_float), p.size,
                                                  _ptr(sc, ctypes.c_float), _ptr(sh, ctypes.c_float)))

    def get_params(self):
        p = np.zeros(self.n_params, np.float32)
        self._check(self.lib.dlmpc_mlp_get_params(self._h, _ptr(p, ctypes.c_float), p.size))
        return p

    def forward(self, x):
        y = self.torch.empty(x.shape[0], self.d_out, dtype=self.torch.float32, device="cuda")
        self._check(self.lib.dlmpc_mlp_forward(self._h, ctypes.c_void_p(x.data_ptr()), x.shape[0],
                                               ctypes.c_void_p(y.data_ptr())))
        return y

    def gradients(self, x, t):
        g = np.zeros(self.n_params, np.float32)
        loss = ctypes.c_double()
        self._check(self.lib.dlmpc_mlp_gradients(self._h, ctypes.c_void_p(x.data_ptr()),
                                                 ctypes.c_void_p(t.data_ptr()), x.shape[0],
                                                 _ptr(g, ctypes.c_float), ctypes.byref(loss)))
        return g, loss.value

    def train_step(self, x, t, lr: float, weight_decay: float = 0.0, want_loss: bool = False):
        loss = ctypes.c_double()
        self._check(self.lib.dlmpc_mlp_train_step(self._h, ctypes.c_void_p(x.data_ptr()),
                                                  ctypes.c_void_p(t.data_ptr()), x.shape[0], lr, weight_decay,
                                                  ctypes.byref(loss) if want_loss else None))
        return loss.value if want_loss else None

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self.lib.dlmpc_mlp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
