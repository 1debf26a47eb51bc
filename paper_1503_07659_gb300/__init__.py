"""semax: the element-local spectral-element Laplacian operator (Ax) on one
GB300, behind the C ABI of include/semax.h.

PyTorch supplies device memory and streams; the operator runs in the
library's own CUDA kernels.  Functions take CUDA tensors in the layouts of the
header (u, w [E,n,n,n]; G [E,6,n,n,n]; D [n,n]) and queue work on the current
torch stream unless `stream` is given.
"""
from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import (SemaxError, semax_group, check, SEMAX_OK, SEMAX_ETIMEOUT, SEMAX_F32, SEMAX_F64, SEMAX_PLAN_F64X, SEMAX_PLAN_F64TC, SEMAX_PLAN_F64TC_PREPARED,
                   SEMAX_PCG_F64X, SEMAX_PCG_F64TC, SEMAX_PCG_MIXED)

__all__ = ["GatherScatter", "PCG", "sem_ax_diag", "sem_ax", "sem_ax_helmholtz", "sem_ax_helmholtz_f64tc", "sem_ax_f64x", "sem_ax_f64tc", "sem_ax_f64tc_prepared", "f64tc_prepare", "set_wait_polls", "fma_probe", "sem_ax_f32", "sem_ax_bf16x3", "sem_ax_f16x3", "sem_ax_bf16x3_geo", "sem_ax_batched", "Plan", "reduce",
           "sem_ax_from_host", "SemaxError", "library_path"]


def library_path() -> str:
    return _lib.LIB_PATH


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _dims(u: torch.Tensor, D: torch.Tensor) -> tuple[int, int]:
    n = D.shape[0]
    E = u.shape[0]
    return E, n - 1


def _ptr(t):
    return None if t is None else t.data_ptr()


def _out(w, u):
    return torch.empty_like(u) if w is None else w


def sem_ax(u: torch.Tensor, G: torch.Tensor, D: torch.Tensor, w: torch.Tensor | None = None,
           stream=None) -> torch.Tensor:
    """FP64 Ax: w = sum_ab D_a^T diag(G_ab) D_b u per element."""
    E, N = _dims(u, D)
    w = _out(w, u)
    check(_lib.lib().sem_ax(E, N, _ptr(u), _ptr(G), _ptr(D), _ptr(w), _stream(stream)), "sem_ax")
    return w


def sem_ax_helmholtz(u: torch.Tensor, G: torch.Tensor, B: torch.Tensor, D: torch.Tensor, h1: float,
                     h2: float, w: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """FP64 w = h1 A u + h2 B u (B the diagonal mass matrix, [E,n,n,n])."""
    E, N = _dims(u, D)
    w = _out(w, u)
    check(_lib.lib().sem_ax_helmholtz(E, N, _ptr(u), _ptr(G), _ptr(B), _ptr(D), float(h1), float(h2), _ptr(w),
                                      _stream(stream)), "sem_ax_helmholtz")
    return w


def sem_ax_helmholtz_f64tc(u: torch.Tensor, G: torch.Tensor, B: torch.Tensor, D: torch.Tensor, h1: float,
                           h2: float, w: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """w = h1 A u + h2 B u with A u FP64-accurate on tensor cores (N = 7; FP64 otherwise)."""
    E, N = _dims(u, D)
    w = _out(w, u)
    check(_lib.lib().sem_ax_helmholtz_f64tc(E, N, _ptr(u), _ptr(G), _ptr(B), _ptr(D), float(h1), float(h2), _ptr(w),
                                            _stream(stream)), "sem_ax_helmholtz_f64tc")
    return w


def sem_ax_f64x(u: torch.Tensor, G: torch.Tensor, D: torch.Tensor, w: torch.Tensor | None = None,
                stream=None) -> torch.Tensor:
    """FP64 in/out, FP64-accurate; contractions in double-float on the FP32 pipe."""
    E, N = _dims(u, D)
    w = _out(w, u)
    check(_lib.lib().sem_ax_f64x(E, N, _ptr(u), _ptr(G), _ptr(D), _ptr(w), _stream(stream)), "sem_ax_f64x")
    return w


def sem_ax_f64tc(u: torch.Tensor, G: torch.Tensor, D: torch.Tensor, w: torch.Tensor | None = None,
                 stream=None, status: torch.Tensor | None = None) -> torch.Tensor:
    """FP64 in/out, FP64-accurate; contractions on FP16 tensor cores by exact digit slicing (N = 7, 15).
    status: optional int32 device tensor that the kernel sets to SEMAX_ETIMEOUT (-6) if a staging wait
    gives up (sem_ax_f64tc_status)."""
    E, N = _dims(u, D)
    w = _out(w, u)
    if status is None:
        check(_lib.lib().sem_ax_f64tc(E, N, _ptr(u), _ptr(G), _ptr(D), _ptr(w), _stream(stream)), "sem_ax_f64tc")
    else:
        check(_lib.lib().sem_ax_f64tc_status(E, N, _ptr(u), _ptr(G), _ptr(D), _ptr(w), _ptr(status),
                                             _stream(stream)), "sem_ax_f64tc_status")
    return w


def fma_probe(prec: str = "f64", blocks: int | None = None, iters: int = 4096, stream=None) -> tuple[torch.Tensor, float]:
    """Launch the FMA-pipe probe (semax_fma_probe) on the current device; returns (sink, flops).
    The caller times the launch with events on `stream`."""
    dt = torch.float64 if prec == "f64" else torch.float32
    if blocks is None:
        blocks = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count * 8
    sink = torch.empty(blocks * 256, dtype=dt, device="cuda")
    flops = ctypes.c_double(0.0)
    check(_lib.lib().semax_fma_probe(SEMAX_F64 if prec == "f64" else SEMAX_F32, int(blocks), int(iters), _ptr(sink),
                                     ctypes.byref(flops), _stream(stream)), "semax_fma_probe")
    return sink, flops.value


def set_wait_polls(polls: int) -> None:
    """Poll limit of the tensor-core kernels' first staging wait for later launches (< 0: default)."""
    check(_lib.lib().semax_set_wait_polls(int(polls)), "semax_set_wait_polls")


def f64tc_prepare(G: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """The prepared geometric factor of sem_ax_f64tc_prepared (order 7): a
    uint8 device tensor of E * 24592 bytes (E * 196624 at order 15)."""
    if G.dim() != 5 or G.shape[1] != 6:
        raise ValueError("f64tc_prepare: G must be [E, 6, n, n, n]")
    E, N = G.shape[0], G.shape[2] - 1
    size = ctypes.c_size_t(0)
    check(_lib.lib().sem_ax_f64tc_prepare_size(E, N, ctypes.byref(size)), "sem_ax_f64tc_prepare_size")
    if out is None:
        out = torch.empty(size.value, dtype=torch.uint8, device=G.device)
    elif out.numel() * out.element_size() < size.value:
        raise ValueError("f64tc_prepare: out too small")
    check(_lib.lib().sem_ax_f64tc_prepare(E, N, _ptr(G), _ptr(out), _stream(stream)), "sem_ax_f64tc_prepare")
    return out


def sem_ax_f64tc_prepared(u: torch.Tensor, Gp: torch.Tensor, D: torch.Tensor, w: torch.Tensor | None = None,
                          stream=None, status: torch.Tensor | None = None) -> torch.Tensor:
    """sem_ax_f64tc with the geometric factor from f64tc_prepare, bit for bit (status as in sem_ax_f64tc)."""
    E, N = _dims(u, D)
    w = _out(w, u)
    if status is None:
        check(_lib.lib().sem_ax_f64tc_prepared(E, N, _ptr(u), _ptr(Gp), _ptr(D), _ptr(w), _stream(stream)),
              "sem_ax_f64tc_prepared")
    else:
        check(_lib.lib().sem_ax_f64tc_prepared_status(E, N, _ptr(u), _ptr(Gp), _ptr(D), _ptr(w), _ptr(status),
                                                      _stream(stream)), "sem_ax_f64tc_prepared_status")
    return w


def sem_ax_f32(u, G, D, w=None, G_scale=None, stream=None) -> torch.Tensor:
    """FP32 storage and compute; optional per-element G scale [E]."""
    E, N = _dims(u, D)
    w = _out(w, u)
    check(_lib.lib().sem_ax_f32(E, N, _ptr(u), _ptr(G), _ptr(D), _ptr(w), _ptr(G_scale),
                                _stream(stream)), "sem_ax_f32")
    return w


def sem_ax_bf16x3(u, G, D, w=None, G_scale=None, terms: int = 3, stream=None) -> torch.Tensor:
    """FP32 storage; contractions on tensor cores with BF16 operand splits."""
    E, N = _dims(u, D)
    w = _out(w, u)
    check(_lib.lib().sem_ax_bf16x3(E, N, _ptr(u), _ptr(G), _ptr(D), _ptr(w), _ptr(G_scale),
                                   int(terms), _stream(stream)), "sem_ax_bf16x3")
    return w


def sem_ax_f16x3(u, G, D, w=None, G_scale=None, stream=None) -> torch.Tensor:
    """FP32 storage; contractions on tensor cores with FP16 operand splits (3 products) after
    power-of-two scaling of each operand group."""
    E, N = _dims(u, D)
    w = _out(w, u)
    check(_lib.lib().sem_ax_f16x3(E, N, _ptr(u), _ptr(G), _ptr(D), _ptr(w), _ptr(G_scale), _stream(stream)),
          "sem_ax_f16x3")
    return w


def sem_ax_bf16x3_geo(u, X, xi_wq, D, w=None, terms: int = 3, stream=None) -> torch.Tensor:
    """BF16-split tensor-core form with G recomputed from the vertices X [E,8,3]."""
    E, N = _dims(u, D)
    w = _out(w, u)
    check(_lib.lib().sem_ax_bf16x3_geo(E, N, _ptr(u), _ptr(X), _ptr(xi_wq), _ptr(D), _ptr(w), int(terms),
                                       _stream(stream)), "sem_ax_bf16x3_geo")
    return w


def _groups(meshes) -> ctypes.Array:
    """meshes: iterable of (N, u, G, D, w) with FP64 CUDA tensors."""
    items = list(meshes)
    arr = (semax_group * max(1, len(items)))()
    for q, (N, u, G, D, w) in enumerate(items):
        arr[q] = semax_group(int(N), int(u.shape[0]), _ptr(u), _ptr(G), _ptr(D), _ptr(w))
    return arr, len(items)


def sem_ax_batched(groups, workspace: torch.Tensor | None = None, stream=None) -> None:
    """All groups (N, u, G, D, w) in one persistent launch (w written in place)."""
    arr, ng = _groups(groups)
    size = ctypes.c_size_t(0)
    check(_lib.lib().sem_ax_batched_workspace_size(arr, ng, ctypes.byref(size)), "sem_ax_batched_workspace_size")
    if workspace is None:
        workspace = torch.empty(size.value, dtype=torch.uint8, device="cuda")
    check(_lib.lib().sem_ax_batched(arr, ng, _ptr(workspace), workspace.numel(), _stream(stream)),
          "sem_ax_batched")


class Plan:
    """Graph-captured persistent batched launch (see sem_ax_plan_create)."""

    def __init__(self, groups, tune: bool = False, cache_path: str | None = None, f64x: bool = False,
                 f64tc: bool = False, f64tc_prepared: bool = False):
        self._arr, ng = _groups(groups)
        self._handle = ctypes.c_void_p()
        flags = ((SEMAX_PLAN_F64X if f64x else 0) | (SEMAX_PLAN_F64TC if f64tc else 0) |
                 (SEMAX_PLAN_F64TC_PREPARED if f64tc_prepared else 0))
        check(_lib.lib().sem_ax_plan_create(ctypes.byref(self._handle), self._arr, ng, int(bool(tune)),
                                            cache_path.encode() if cache_path else None, flags),
              "sem_ax_plan_create")

    def __call__(self, stream=None) -> None:
        check(_lib.lib().sem_ax_plan_exec(self._handle, _stream(stream)), "sem_ax_plan_exec")

    def status(self, stream=None) -> int:
        """SEMAX_OK, or SEMAX_ETIMEOUT if a tensor-core launch of the plan had a staging wait give up since
        the last call (blocks until the stream's queued work is done; clears the word)."""
        st = _lib.lib().sem_ax_plan_status(self._handle, _stream(stream))
        if st not in (SEMAX_OK, SEMAX_ETIMEOUT):
            check(st, "sem_ax_plan_status")
        return st

    def config(self, N: int) -> tuple[int, int]:
        epb, mp = ctypes.c_int(0), ctypes.c_int(0)
        check(_lib.lib().sem_ax_plan_config(self._handle, int(N), ctypes.byref(epb), ctypes.byref(mp)),
              "sem_ax_plan_config")
        return epb.value, mp.value

    def close(self) -> None:
        if self._handle:
            check(_lib.lib().sem_ax_plan_destroy(self._handle), "sem_ax_plan_destroy")
            self._handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def reduce(a: torch.Tensor, b: torch.Tensor, out: torch.Tensor | None = None,
           workspace: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """[max|a-b|, max|b|, a.b] in FP64 on the GPU (a, b FP64 or FP32)."""
    if a.numel() != b.numel():
        raise ValueError("reduce: size mismatch")
    prec = {torch.float64: SEMAX_F64, torch.float32: SEMAX_F32}
    count = a.numel()
    size = ctypes.c_size_t(0)
    check(_lib.lib().semax_reduce_workspace_size(count, ctypes.byref(size)), "semax_reduce_workspace_size")
    if workspace is None:
        workspace = torch.empty(size.value, dtype=torch.uint8, device=a.device)
    if out is None:
        out = torch.empty(3, dtype=torch.float64, device=a.device)
    check(_lib.lib().semax_reduce(count, _ptr(a), prec[a.dtype], _ptr(b), prec[b.dtype], _ptr(out),
                                  _ptr(workspace), workspace.numel(), _stream(stream)), "semax_reduce")
    return out


def sem_ax_from_host(u_host: torch.Tensor, G_host: torch.Tensor, D_host: torch.Tensor,
                     w_host: torch.Tensor, bufs: dict | None = None, stream=None) -> dict:
    """End-to-end FP64 Ax from (pinned) host tensors: copy u, G, D to the
    device, run sem_ax, copy w back into w_host.  `bufs` caches the device
    buffers between calls; it is returned.  The caller synchronises."""
    if bufs is None:
        bufs = {"u": torch.empty(u_host.shape, dtype=u_host.dtype, device="cuda"),
                "G": torch.empty(G_host.shape, dtype=G_host.dtype, device="cuda"),
                "D": torch.empty(D_host.shape, dtype=D_host.dtype, device="cuda"),
                "w": torch.empty(u_host.shape, dtype=u_host.dtype, device="cuda")}
    s = torch.cuda.current_stream() if stream is None else stream
    with torch.cuda.stream(s):
        bufs["u"].copy_(u_host, non_blocking=True)
        bufs["G"].copy_(G_host, non_blocking=True)
        bufs["D"].copy_(D_host, non_blocking=True)
        sem_ax(bufs["u"], bufs["G"], bufs["D"], bufs["w"], stream=s)
        w_host.copy_(bufs["w"], non_blocking=True)
    return bufs


class GatherScatter:
    """Direct stiffness summation over shared nodes (semax_gs_*)."""

    def __init__(self, local_to_global, nglobal: int, dirichlet=None):
        import numpy as np
        l2g = np.ascontiguousarray(local_to_global, dtype=np.int64)
        self._dir = None if dirichlet is None else np.ascontiguousarray(dirichlet, dtype=np.uint8)
        self._handle = ctypes.c_void_p()
        check(_lib.lib().semax_gs_create(ctypes.byref(self._handle), l2g.size, l2g.ctypes.data, int(nglobal),
                                         None if self._dir is None else self._dir.ctypes.data),
              "semax_gs_create")
        self.nlocal = l2g.size

    def __call__(self, v: torch.Tensor, mask: bool = True, stream=None) -> torch.Tensor:
        check(_lib.lib().semax_gs_apply(self._handle, _ptr(v), int(bool(mask)), _stream(stream)), "semax_gs_apply")
        return v

    def close(self) -> None:
        if self._handle:
            check(_lib.lib().semax_gs_destroy(self._handle), "semax_gs_destroy")
            self._handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sem_ax_diag(G: torch.Tensor, D: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    n = D.shape[0]
    E = G.shape[0]
    if out is None:
        out = torch.empty((E, n, n, n), dtype=torch.float64, device=G.device)
    check(_lib.lib().sem_ax_diag(E, n - 1, _ptr(G), _ptr(D), _ptr(out), _stream(stream)), "sem_ax_diag")
    return out


class PCG:
    """Jacobi-PCG on Q A_L Q^T (sem_pcg_*); G, D and the gather-scatter stay bound."""

    def __init__(self, G: torch.Tensor, D: torch.Tensor, gs: GatherScatter, f64x: bool = False,
                 f64tc: bool = False, mixed: bool = False):
        self._keep = (G, D, gs)
        self._handle = ctypes.c_void_p()
        flags = ((SEMAX_PCG_F64X if f64x else 0) | (SEMAX_PCG_F64TC if f64tc else 0)
                 | (SEMAX_PCG_MIXED if mixed else 0))
        check(_lib.lib().sem_pcg_create(ctypes.byref(self._handle), G.shape[0], D.shape[0] - 1, _ptr(G), _ptr(D),
                                        gs._handle, flags), "sem_pcg_create")

    def solve(self, b: torch.Tensor, x: torch.Tensor, max_iter: int = 1000, rtol: float = 1e-10,
              stream=None) -> tuple[int, float]:
        it, rel = ctypes.c_int(0), ctypes.c_double(0.0)
        check(_lib.lib().sem_pcg_solve(self._handle, _ptr(b), _ptr(x), int(max_iter), float(rtol), ctypes.byref(it),
                                       ctypes.byref(rel), _stream(stream)), "sem_pcg_solve")
        return it.value, rel.value

    def close(self) -> None:
        if self._handle:
            check(_lib.lib().sem_pcg_destroy(self._handle), "sem_pcg_destroy")
            self._handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
