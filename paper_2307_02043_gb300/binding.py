"""ctypes binding of libmqnpm (argument marshalling only).

Every numerical step runs in the CUDA library; this module converts torch
tensors to device pointers, passes the current torch stream and raises on any
non-zero status.  There is no CPU or PyTorch fallback: if the library cannot be
loaded, importing the handle class fails.
"""
from __future__ import annotations

import ctypes
import math
import os
from typing import Optional, Sequence

import numpy as np
import torch

from . import build as _build

OK = 0
STATUS = {
    0: "OK", 1: "INVALID_ARG", 2: "BUDGET", 3: "CUDA", 4: "NOT_CONVERGED", 5: "NONFINITE",
    6: "TIMEOUT", 7: "UNSUPPORTED", 8: "STATE",
}
MODEL = {"born": 0, "ls": 1}
TV = {"iso": 0, "aniso": 1}
KERNEL = {"sampled": 0, "truncated": 1}
MAX_S = 16
SUPPORTED_N = (8, 12, 16, 24, 32, 48, 64, 96, 128, 160, 192)   # every edge of a grid takes one of these


class MQNPMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("%s (%d): %s" % (STATUS.get(code, "?"), code, msg))
        self.code = code


class NotConverged(MQNPMError):
    pass


class Config(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("h", ctypes.c_double), ("kb", ctypes.c_double), ("model", ctypes.c_int),
        ("L", ctypes.c_int), ("kdir", ctypes.POINTER(ctypes.c_double)),
        ("S", ctypes.c_int), ("subset_of", ctypes.POINTER(ctypes.c_int)),
        ("alpha", ctypes.POINTER(ctypes.c_double)), ("step", ctypes.c_double), ("strategy", ctypes.c_int),
        ("strategy_draws", ctypes.POINTER(ctypes.c_int)), ("n_draws", ctypes.c_int),
        ("tv", ctypes.c_int), ("lam", ctypes.c_double), ("box_lo", ctypes.c_double), ("box_hi", ctypes.c_double),
        ("gamma", ctypes.c_double), ("tau_max", ctypes.c_double), ("delta1", ctypes.c_double),
        ("delta2", ctypes.c_double), ("krylov_tol", ctypes.c_double), ("krylov_maxit", ctypes.c_int),
        ("dual_iters", ctypes.c_int), ("newton_tol", ctypes.c_double), ("newton_maxit", ctypes.c_int),
        ("max_batch", ctypes.c_int), ("hbm_budget_bytes", ctypes.c_size_t), ("device", ctypes.c_int),
        ("stream", ctypes.c_void_p), ("warm_start", ctypes.c_int), ("direct_launches", ctypes.c_int),
        ("green_hat", ctypes.POINTER(ctypes.c_float)), ("tile", ctypes.c_int),
        ("det_distance", ctypes.c_double), ("det_na", ctypes.c_double), ("guard_bytes", ctypes.c_size_t),
        ("barrier_wait_cycles", ctypes.c_longlong), ("green_kernel", ctypes.c_int),
        ("adjoint_start", ctypes.c_int), ("forward_start", ctypes.c_int),
    ]


class StepInfo(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("subset", ctypes.c_int), ("loss", ctypes.c_double),
                ("tau_star", ctypes.c_double), ("rank", ctypes.c_int), ("sr1_branch", ctypes.c_int),
                ("krylov_iters_max", ctypes.c_int), ("newton_iters_max", ctypes.c_int),
                ("krylov_iters_total", ctypes.c_int), ("n_illum", ctypes.c_int),
                ("ms_gradient", ctypes.c_double), ("ms_metric", ctypes.c_double), ("ms_prox", ctypes.c_double)]


_LIB = None

# Every entry point of include/mqnpm.h with its ctypes signature.
SIGNATURES = {
    "mqnpm_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_void_p)]),
    "mqnpm_destroy": (None, [ctypes.c_void_p]),
    "mqnpm_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "mqnpm_set_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "mqnpm_set_wait_limit": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_longlong]),
    "mqnpm_workspace_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "mqnpm_set_measurements": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "mqnpm_green_apply": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int]),
    "mqnpm_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                     ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "mqnpm_grad_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                        ctypes.c_double, ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                        ctypes.POINTER(ctypes.c_int)]),
    "mqnpm_loss_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                        ctypes.c_double, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]),
    "mqnpm_grad_fields": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int,
                                         ctypes.c_double, ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "mqnpm_wprox": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double, ctypes.c_void_p, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_void_p, ctypes.c_void_p]),
    "mqnpm_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(StepInfo)]),
    "mqnpm_step_subset": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                         ctypes.POINTER(ctypes.c_int)]),
    "mqnpm_step_with_gradient": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_double,
                                                ctypes.POINTER(StepInfo)]),
    "mqnpm_lipschitz": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.c_int, ctypes.c_double,
                                       ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "mqnpm_save_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_size_t)]),
    "mqnpm_load_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "mqnpm_launch_count": (ctypes.c_longlong, [ctypes.c_void_p]),
    "mqnpm_check_guards": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int)]),
    "mqnpm_debug_poke_guard": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "mqnpm_diagnostics": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_double)]),
    "mqnpm_tile_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                       ctypes.POINTER(ctypes.c_double)]),
    "mqnpm_prox_trace": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_longlong), ctypes.c_int,
                                        ctypes.POINTER(ctypes.c_int)]),
    "mqnpm_profile_begin": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "mqnpm_profile_end": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_int)]),
    "mqnpm_green_apply_noalloc": (ctypes.c_int, [ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                                 ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "mqnpm_noalloc_scratch_bytes": (ctypes.c_size_t, []),
    "mqnpm_group_create": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int, ctypes.c_int, ctypes.c_size_t,
                                          ctypes.POINTER(ctypes.c_void_p)]),
    "mqnpm_group_destroy": (None, [ctypes.c_void_p]),
    "mqnpm_group_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p), ctypes.POINTER(StepInfo)]),
    "mqnpm_group_set_stream": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "mqnpm_group_workspace_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "mqnpm_group_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
}


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libmqnpm.so (building it first if needed); raises if it cannot be loaded."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError("libmqnpm.so is not built (run __graft_entry__.build())")
        _build.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _check_cuda(t: torch.Tensor, dtype, numel: int, name: str, device: int):
    if not isinstance(t, torch.Tensor):
        raise TypeError("%s must be a torch tensor" % name)
    if not t.is_cuda or t.device.index != device:
        raise ValueError("%s must live on cuda:%d" % (name, device))
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if t.numel() != numel:
        raise ValueError("%s must have %d elements, got %d" % (name, numel, t.numel()))


def green_apply_noalloc(n: int, h: float, kb: float, v: torch.Tensor, out: torch.Tensor,
                        adjoint: bool = False) -> torch.Tensor:
    """G v (or G^H v) of one n^3 volume into `out` with the library's static
    device scratch: the C call allocates nothing (n <= 32)."""
    lib = load()
    dev = v.device.index if v.is_cuda else -1
    _check_cuda(v, torch.complex64, n ** 3, "v", dev)
    _check_cuda(out, torch.complex64, n ** 3, "out", dev)
    with torch.cuda.device(dev):
        s = torch.cuda.current_stream(dev).cuda_stream
        rc = lib.mqnpm_green_apply_noalloc(int(n), float(h), float(kb), _ptr(v), _ptr(out), int(adjoint),
                                           ctypes.c_void_p(s))
    if rc != OK:
        raise MQNPMError(rc, "green_apply_noalloc failed")
    return out


class MQNPM:
    """One reconstruction problem on one GPU (a handle of libmqnpm).  n is the
    grid edge of a cubic grid or the (nz, ny, nx) edges of a box."""

    def __init__(self, n, kdir, subset_of, alpha, *, model: str = "ls", h: float = 1.0,
                 kb: float = math.pi / 2, tv: str = "iso", lam: float = 1e-3, box=(0.0, 1.0),
                 step: float = 1.0, strategy: int = 1, draws: Optional[Sequence[int]] = None,
                 gamma: float = 0.8, tau_max: float = 0.0, krylov_tol: float = 1e-6, krylov_maxit: int = 500,
                 dual_iters: int = 20, newton_tol: float = 1e-6, newton_maxit: int = 50, max_batch: int = 8,
                 hbm_budget_bytes: int = 0, device: int = 0, warm_start: bool = False,
                 direct_launches: bool = False, green_hat: Optional[np.ndarray] = None, tile: int = -1,
                 det_distance: float = 0.0, det_na: float = 0.0, guard_bytes: int = 0,
                 barrier_wait_cycles: int = 0, green_kernel: str = "sampled", adjoint_start: str = "b",
                 forward_start: str = "refine"):
        self.lib = load()
        if np.ndim(n) == 0:
            self.shape = (int(n),) * 3
            self.n = int(n)
        else:
            self.shape = tuple(int(v) for v in n)
            if len(self.shape) != 3:
                raise ValueError("n must be an edge or (nz, ny, nx)")
            self.n = self.shape
        nz, ny, nx = self.shape
        self.N = nx * ny * nz
        self.M = nx * ny
        self.device = int(device)
        kd = np.ascontiguousarray(np.asarray(kdir, dtype=np.float64).reshape(-1, 3))
        so = np.ascontiguousarray(np.asarray(subset_of, dtype=np.int32))
        al = np.ascontiguousarray(np.asarray(alpha, dtype=np.float64))
        dr = np.ascontiguousarray(np.asarray(draws if draws is not None else [], dtype=np.int32))
        self.L = kd.shape[0]
        self.S = al.shape[0]
        self._keep = (kd, so, al, dr)
        cfg = Config()
        cfg.nz, cfg.ny, cfg.nx = self.shape
        cfg.h = h
        cfg.kb = kb
        cfg.model = MODEL[model]
        cfg.L = self.L
        cfg.kdir = kd.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        cfg.S = self.S
        cfg.subset_of = so.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        cfg.alpha = al.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        cfg.step = step
        cfg.strategy = strategy
        cfg.strategy_draws = dr.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
        cfg.n_draws = dr.shape[0]
        cfg.tv = TV[tv]
        cfg.lam = lam
        cfg.box_lo, cfg.box_hi = float(box[0]), float(box[1])
        cfg.gamma = gamma
        cfg.tau_max = tau_max
        cfg.delta1 = 1e-8
        cfg.delta2 = 1e-12
        cfg.krylov_tol = krylov_tol
        cfg.krylov_maxit = krylov_maxit
        cfg.dual_iters = dual_iters
        cfg.newton_tol = newton_tol
        cfg.newton_maxit = newton_maxit
        cfg.max_batch = max_batch
        cfg.hbm_budget_bytes = hbm_budget_bytes
        cfg.warm_start = int(bool(warm_start))
        cfg.direct_launches = int(bool(direct_launches))
        cfg.tile = int(tile)
        cfg.det_distance = float(det_distance)
        cfg.det_na = float(det_na)
        cfg.guard_bytes = int(guard_bytes)
        cfg.barrier_wait_cycles = int(barrier_wait_cycles)
        cfg.green_kernel = KERNEL[green_kernel]
        cfg.adjoint_start = {"b": 0, "zero": 1}[adjoint_start]
        cfg.forward_start = {"refine": 0, "stored": 1}[forward_start]
        if green_hat is not None:
            gh = np.ascontiguousarray(np.asarray(green_hat, dtype=np.complex64))
            if gh.size != (nx + 1) * (ny + 1) * (nz + 1):
                raise ValueError("green_hat must hold (nz+1)(ny+1)(nx+1) complex values")
            self._keep = self._keep + (gh,)
            cfg.green_hat = gh.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
        cfg.device = self.device
        with torch.cuda.device(self.device):
            cfg.stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        self.max_batch = max_batch
        handle = ctypes.c_void_p()
        rc = self.lib.mqnpm_create(ctypes.byref(cfg), ctypes.byref(handle))
        if rc != OK:
            raise MQNPMError(rc, "mqnpm_create failed")
        self._h = handle

    # -- plumbing ----------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None):
            self.lib.mqnpm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _stream(self):
        s = torch.cuda.current_stream(self.device).cuda_stream
        self.lib.mqnpm_set_stream(self._h, ctypes.c_void_p(s))

    def _raise(self, rc: int, allow_not_converged: bool = False):
        if rc == OK or (allow_not_converged and rc == 4):
            return
        msg = self.lib.mqnpm_last_error(self._h).decode()
        if rc == 4:
            raise NotConverged(rc, msg)
        raise MQNPMError(rc, msg)

    @property
    def workspace_bytes(self) -> int:
        return int(self.lib.mqnpm_workspace_bytes(self._h))

    @property
    def launch_count(self) -> int:
        """Kernels launched by this handle since creation."""
        return int(self.lib.mqnpm_launch_count(self._h))

    def diagnostics(self, x_prev: torch.Tensor, s_prime: int, x_cur: Optional[torch.Tensor] = None,
                    allow_not_converged: bool = False) -> dict:
        """Section 6 convergence diagnostics at iteration k: the bias error e_k^2,
        ||x_k - x_{k-1}||^2 and the full data term at x_{k-1}."""
        _check_cuda(x_prev, torch.float32, self.N, "x_prev", self.device)
        if x_cur is not None:
            _check_cuda(x_cur, torch.float32, self.N, "x_cur", self.device)
        out = (ctypes.c_double * 3)()
        self._stream()
        rc = self.lib.mqnpm_diagnostics(self._h, _ptr(x_prev), _ptr(x_cur) if x_cur is not None else None,
                                        int(s_prime), out)
        self._raise(rc, allow_not_converged)
        return {"bias_error": out[0], "step_sq": out[1], "data_term": out[2]}

    def set_wait_limit(self, cycles: int):
        """Grid-barrier wait limit of the proximal mapping (SM cycles; 0 = default)."""
        self._raise(self.lib.mqnpm_set_wait_limit(self._h, int(cycles)))

    def check_guards(self) -> int:
        """Guard bands (guard_bytes > 0) no longer holding their fill pattern."""
        bad = ctypes.c_int()
        self._stream()
        self._raise(self.lib.mqnpm_check_guards(self._h, ctypes.byref(bad)))
        return bad.value

    def tile_info(self) -> dict:
        """Launch shapes of the Green's passes and the autotuner's timings (ms per apply)."""
        tile = ctypes.c_int()
        shape = (ctypes.c_int * 6)()
        ms = (ctypes.c_double * 32)()
        self._raise(self.lib.mqnpm_tile_info(self._h, ctypes.byref(tile), shape, ms))
        return {"tile": tile.value, "x": {"lines_per_cta": shape[0], "threads_per_line": shape[1]},
                "y": {"columns_per_cta": shape[2], "threads_per_column": shape[3]},
                "z": {"columns_per_cta": shape[4], "threads_per_column": shape[5],
                      "exchange_buffers": 2 if tile.value & 8 else 1},
                "fused_xy": bool(tile.value & 16),
                "tuned_ms": [round(m, 4) if m >= 0 else None for m in ms]}

    # -- calls -------------------------------------------------------------
    def set_measurements(self, y: torch.Tensor):
        _check_cuda(y, torch.complex64, self.L * self.M, "y", self.device)
        self._stream()
        self._raise(self.lib.mqnpm_set_measurements(self._h, _ptr(y)))

    def green_apply(self, v: torch.Tensor, adjoint: bool = False) -> torch.Tensor:
        nb = v.numel() // self.N
        _check_cuda(v, torch.complex64, nb * self.N, "v", self.device)
        out = torch.empty_like(v)
        self._stream()
        self._raise(self.lib.mqnpm_green_apply(self._h, _ptr(v), _ptr(out), nb, int(adjoint)))
        return out

    def forward(self, x: torch.Tensor, illum: Sequence[int], allow_not_converged=False):
        _check_cuda(x, torch.float32, self.N, "x", self.device)
        il = (ctypes.c_int * len(illum))(*[int(i) for i in illum])
        its = (ctypes.c_int * len(illum))()
        y = torch.empty((len(illum), self.M), dtype=torch.complex64, device=x.device)
        self._stream()
        rc = self.lib.mqnpm_forward(self._h, _ptr(x), il, len(illum), _ptr(y), its)
        self._raise(rc, allow_not_converged)
        return y, list(its)

    def grad_batch(self, x: torch.Tensor, illum: Sequence[int], scale: float, out: Optional[torch.Tensor] = None,
                   allow_not_converged=False):
        _check_cuda(x, torch.float32, self.N, "x", self.device)
        if out is None:
            out = torch.empty_like(x)
        _check_cuda(out, torch.float32, self.N, "grad_out", self.device)
        nb = len(illum)
        il = (ctypes.c_int * nb)(*[int(i) for i in illum])
        its = (ctypes.c_int * (2 * nb))()
        loss = ctypes.c_double()
        self._stream()
        rc = self.lib.mqnpm_grad_batch(self._h, _ptr(x), il, nb, float(scale), _ptr(out), ctypes.byref(loss), its)
        self._raise(rc, allow_not_converged)
        return out, loss.value, [(its[2 * b], its[2 * b + 1]) for b in range(nb)]

    def loss_batch(self, x: torch.Tensor, illum: Sequence[int], scale: float, allow_not_converged=False):
        """scale * sum f_l(x) without the gradient; keeps the fields of a single
        chunk for grad_fields."""
        _check_cuda(x, torch.float32, self.N, "x", self.device)
        nb = len(illum)
        il = (ctypes.c_int * nb)(*[int(i) for i in illum])
        its = (ctypes.c_int * nb)()
        loss = ctypes.c_double()
        self._stream()
        rc = self.lib.mqnpm_loss_batch(self._h, _ptr(x), il, nb, float(scale), ctypes.byref(loss), its)
        self._raise(rc, allow_not_converged)
        return loss.value, list(its)

    def grad_fields(self, x: torch.Tensor, illum: Sequence[int], scale: float, reuse: bool = True,
                    out: Optional[torch.Tensor] = None, allow_not_converged=False):
        """scale * sum grad f_l(x), reusing the fields of the last loss_batch
        when allowed; returns (gradient, reused)."""
        _check_cuda(x, torch.float32, self.N, "x", self.device)
        if out is None:
            out = torch.empty_like(x)
        _check_cuda(out, torch.float32, self.N, "grad_out", self.device)
        nb = len(illum)
        il = (ctypes.c_int * nb)(*[int(i) for i in illum])
        reused = ctypes.c_int()
        self._stream()
        rc = self.lib.mqnpm_grad_fields(self._h, _ptr(x), il, nb, float(scale), _ptr(out), int(bool(reuse)),
                                        ctypes.byref(reused))
        self._raise(rc, allow_not_converged)
        return out, bool(reused.value)

    def wprox(self, v: torch.Tensor, tau: float, U: Optional[torch.Tensor], c: float,
              P_warm: Optional[torch.Tensor] = None, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        _check_cuda(v, torch.float32, self.N, "v", self.device)
        S_eff = 0
        if U is not None and U.numel() > 0:
            S_eff = U.numel() // self.N
            _check_cuda(U, torch.float32, S_eff * self.N, "U", self.device)
        else:
            U = None
        if P_warm is not None:
            _check_cuda(P_warm, torch.float32, 3 * self.N, "P_warm", self.device)
        if out is None:
            out = torch.empty_like(v)
        self._stream()
        rc = self.lib.mqnpm_wprox(self._h, _ptr(v), float(tau), _ptr(U), S_eff, float(c), _ptr(P_warm), _ptr(out))
        self._raise(rc)
        return out

    def step(self, x: torch.Tensor, allow_not_converged=False) -> dict:
        _check_cuda(x, torch.float32, self.N, "x", self.device)
        info = StepInfo()
        self._stream()
        rc = self.lib.mqnpm_step(self._h, _ptr(x), ctypes.byref(info))
        self._raise(rc, allow_not_converged)
        return {f: getattr(info, f) for f, _ in StepInfo._fields_}

    def step_subset(self):
        """(subset, illuminations) that the next iteration uses."""
        sub = ctypes.c_int()
        cnt = ctypes.c_int()
        il = (ctypes.c_int * self.L)()
        self._raise(self.lib.mqnpm_step_subset(self._h, ctypes.byref(sub), il, ctypes.byref(cnt)))
        return sub.value, [il[i] for i in range(cnt.value)]

    def step_with_gradient(self, x: torch.Tensor, g: torch.Tensor, loss: float) -> dict:
        """The next iteration with the caller's subset gradient g = grad F_s(x) and loss F_s(x)."""
        _check_cuda(x, torch.float32, self.N, "x", self.device)
        _check_cuda(g, torch.float32, self.N, "g", self.device)
        info = StepInfo()
        self._stream()
        self._raise(self.lib.mqnpm_step_with_gradient(self._h, _ptr(x), _ptr(g), float(loss), ctypes.byref(info)))
        return {f: getattr(info, f) for f, _ in StepInfo._fields_}

    def lipschitz(self, illum: Sequence[int], scale: float, start: torch.Tensor, iters: int = 20) -> float:
        _check_cuda(start, torch.float32, self.N, "start", self.device)
        il = (ctypes.c_int * len(illum))(*[int(i) for i in illum])
        out = ctypes.c_double()
        self._stream()
        self._raise(self.lib.mqnpm_lipschitz(self._h, il, len(illum), float(scale), _ptr(start), int(iters),
                                             ctypes.byref(out)))
        return out.value

    def save_state(self) -> bytes:
        size = ctypes.c_size_t()
        self._raise(self.lib.mqnpm_save_state(self._h, None, ctypes.byref(size)))
        buf = ctypes.create_string_buffer(size.value)
        self._stream()
        self._raise(self.lib.mqnpm_save_state(self._h, buf, ctypes.byref(size)))
        return buf.raw

    def load_state(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        self._stream()
        self._raise(self.lib.mqnpm_load_state(self._h, buf, len(blob)))

    def prox_trace(self) -> dict:
        """Time (us) spent per phase tag in the last weighted proximal mapping."""
        cap = 1024
        buf = (ctypes.c_longlong * (2 * cap))()
        cnt = ctypes.c_int()
        self._stream()
        self._raise(self.lib.mqnpm_prox_trace(self._h, buf, cap, ctypes.byref(cnt)))
        names = {1: "gram", 2: "x_plain", 3: "div_UTd", 4: "newton_eval", 5: "x_fixup", 6: "dual_update", 99: "tail"}
        out = {"barriers": cnt.value - 1, "total_us": 0.0}
        counts = {}
        prev = buf[1]
        for e in range(1, cnt.value + 1):
            tag, t = buf[2 * e], buf[2 * e + 1]
            key = names.get(int(tag), str(tag))
            out[key] = out.get(key, 0.0) + (t - prev) / 1e3
            out["total_us"] += (t - prev) / 1e3
            counts[key] = counts.get(key, 0) + 1
            prev = t
        acc = ["dual_update_block0", "pre_dual_block0", "newton_pass_block0", "newton_decide_block0",
               "div_pass_block0", "barrier_wait_block0"]
        for k, nm in enumerate(acc):
            out[nm] = buf[2000 + k] / 1e3
        out = {k: (round(v, 1) if isinstance(v, float) else v) for k, v in out.items()}
        out["counts"] = counts
        return out

    def profile_begin(self, max_calls: int = 4096):
        self._raise(self.lib.mqnpm_profile_begin(self._h, int(max_calls)))

    def profile_end(self) -> dict:
        """Per-pass device time (ms) of the Green's applies since profile_begin."""
        ms = (ctypes.c_double * 5)()
        slots = ctypes.c_longlong()
        calls = ctypes.c_int()
        self._stream()
        self._raise(self.lib.mqnpm_profile_end(self._h, ms, ctypes.byref(slots), ctypes.byref(calls)))
        return {"pass_ms": list(ms), "slot_launches": slots.value, "calls": calls.value}


class Group:
    """Several reconstructions of one grid whose subset gradients run in shared
    launches (a libmqnpm group of member handles)."""

    def __init__(self, members: Sequence[MQNPM], max_slots: int, hbm_budget_bytes: int = 0):
        self.lib = load()
        self.members = list(members)
        if not self.members:
            raise ValueError("a group needs at least one member")
        arr = (ctypes.c_void_p * len(self.members))(*[m._h.value for m in self.members])
        g = ctypes.c_void_p()
        rc = self.lib.mqnpm_group_create(arr, len(self.members), int(max_slots), int(hbm_budget_bytes),
                                         ctypes.byref(g))
        if rc != OK:
            raise MQNPMError(rc, "mqnpm_group_create failed")
        self._g = g
        self.device = self.members[0].device

    def close(self):
        if getattr(self, "_g", None):
            self.lib.mqnpm_group_destroy(self._g)
            self._g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def workspace_bytes(self) -> int:
        return int(self.lib.mqnpm_group_workspace_bytes(self._g))

    def step(self, xs: Sequence[torch.Tensor], allow_not_converged=False) -> list:
        if len(xs) != len(self.members):
            raise ValueError("one iterate per member")
        for m, x in zip(self.members, xs):
            _check_cuda(x, torch.float32, m.N, "x", self.device)
        ptrs = (ctypes.c_void_p * len(xs))(*[x.data_ptr() for x in xs])
        infos = (StepInfo * len(xs))()
        s = torch.cuda.current_stream(self.device).cuda_stream
        self.lib.mqnpm_group_set_stream(self._g, ctypes.c_void_p(s))
        rc = self.lib.mqnpm_group_step(self._g, ptrs, infos)
        if rc != OK and not (allow_not_converged and rc == 4):
            msg = self.lib.mqnpm_group_last_error(self._g).decode()
            raise (NotConverged if rc == 4 else MQNPMError)(rc, msg)
        return [{f: getattr(i, f) for f, _ in StepInfo._fields_} for i in infos]
