"""B300-native Taylor-Green-vortex hot path (arXiv 2505.20911).

The fused explicit finite-difference residual of the 3-D compressible
Navier-Stokes equations and the low-storage RK3 update it feeds, as CUDA
kernels for sm_103a behind a C ABI (include/tgv.h).  This module is the thin
Python binding: it marshals torch tensors (device memory) and CUDA streams
into the C calls, with the same names.  PyTorch provides memory and streams
only; every step of the path runs in libtgv.so.
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass, replace

import torch

from . import _abi
from ._abi import (TGV_BF16, TGV_DIAG_COUNT, TGV_ENC_OFFSET, TGV_ENC_PLAIN, TGV_F16,  # noqa: F401
                   TGV_F32, TGV_F64, TGV_FLAG_ALLOW_UNSTABLE_DT, TGV_SPLIT_BLAISDELL,
                   TGV_SPLIT_DIVERGENCE, TGVError, check, lib)

DIAG_NAMES = ("K", "K_rho", "enstrophy", "eps_S", "rho", "rho_u", "rho_v", "rho_w",
              "rho_E", "nonfinite")

TORCH_DTYPE = {TGV_F64: torch.float64, TGV_F32: torch.float32, TGV_BF16: torch.bfloat16,
               TGV_F16: torch.float16}

# Named precision modes: (q_storage, qt_storage, compute, accumulate).
MODES = {
    "fp64": (TGV_F64, TGV_F64, TGV_F64, TGV_F64),          # double
    "spdp": (TGV_F64, TGV_F64, TGV_F32, TGV_F64),          # single-double: Q FP64, R FP32
    "fp32s_fp64c": (TGV_F32, TGV_F32, TGV_F64, TGV_F64),   # FP32 storage / FP64 compute
    "fp32": (TGV_F32, TGV_F32, TGV_F32, TGV_F32),          # single
    "bf16_fp32": (TGV_BF16, TGV_BF16, TGV_F32, TGV_F32),   # bf16 storage / FP32 compute
    "fp16_fp32": (TGV_F16, TGV_F16, TGV_F32, TGV_F32),     # half-single
    "fp16": (TGV_F16, TGV_F16, TGV_F16, TGV_F32),          # pure half
    "hpsp": (TGV_F32, TGV_F16, TGV_F32, TGV_F32),          # Q FP32, Qt FP16
}


@dataclass(frozen=True)
class Config:
    """Python mirror of tgv_config (include/tgv.h)."""

    n: int
    mode: str = "fp64"
    mach: float = 0.1
    re: float = 1600.0
    pr: float = 0.71
    gamma: float = 1.4
    mu: float = 1.0
    split: str = "blaisdell"
    encoding: str = "plain"
    tile: int = 0
    zchunk: int = 0
    allow_unstable_dt: bool = False
    check_finite: bool = False
    cell_centered: bool = False
    symmetric: bool = False      # the symmetric box (TGSym); set length = pi
    length: float = 2.0 * math.pi

    def with_(self, **kw) -> "Config":
        return replace(self, **kw)

    @property
    def q_dtype(self) -> torch.dtype:
        return TORCH_DTYPE[MODES[self.mode][0]]

    @property
    def qt_dtype(self) -> torch.dtype:
        return TORCH_DTYPE[MODES[self.mode][1]]

    @property
    def compute_dtype(self) -> torch.dtype:
        return TORCH_DTYPE[MODES[self.mode][2]]

    def c(self) -> _abi.tgv_config:
        qs, qts, comp, acc = MODES[self.mode]
        return _abi.tgv_config(
            n=self.n,
            split_form={"blaisdell": TGV_SPLIT_BLAISDELL, "divergence": TGV_SPLIT_DIVERGENCE,
                        "kgp": _abi.TGV_SPLIT_KGP, "keep": _abi.TGV_SPLIT_KEEP,
                        "feiereisen": _abi.TGV_SPLIT_FEIEREISEN}[self.split],
            q_storage=qs, qt_storage=qts, compute=comp, accumulate=acc,
            encoding={"plain": TGV_ENC_PLAIN, "offset": TGV_ENC_OFFSET}[self.encoding],
            tile=self.tile, zchunk=self.zchunk,
            flags=(TGV_FLAG_ALLOW_UNSTABLE_DT if self.allow_unstable_dt else 0)
            | (_abi.TGV_FLAG_CHECK_FINITE if self.check_finite else 0)
            | (_abi.TGV_FLAG_CELL_CENTERED if self.cell_centered else 0)
            | (_abi.TGV_FLAG_SYMMETRIC if self.symmetric else 0),
            length=self.length, gamma=self.gamma, mach=self.mach, re=self.re, pr=self.pr,
            mu=self.mu)


def _ptr(t) -> int | None:
    """Device pointer of an optional CUDA tensor (contiguous, on the current
    device); sizes are checked by _dev where the caller knows them."""
    if t is None:
        return None
    return _dev(t, "tensor")


def _nbytes(t) -> int:
    return t.numel() * t.element_size()


def _dev(t, name: str, dtype=None, nbytes: int | None = None) -> int:
    """Validate a device buffer before it reaches the library: a contiguous
    CUDA tensor on the current device, of `dtype` (if given) and at least
    `nbytes` bytes (if given).  Raises ValueError; nothing is launched."""
    if not getattr(t, "is_cuda", False):
        raise ValueError(f"{name}: expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name}: expected a contiguous tensor")
    cur = torch.cuda.current_device()
    if t.device.index != cur:
        raise ValueError(f"{name} is on cuda:{t.device.index}, the current device is cuda:{cur}")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name}: expected {dtype}, got {t.dtype}")
    if nbytes is not None and _nbytes(t) < nbytes:
        raise ValueError(f"{name}: {_nbytes(t)} bytes, the library needs {nbytes}")
    return t.data_ptr()


def _host(t, name: str, dtype=None, nbytes: int | None = None) -> int:
    """Validate a host buffer (contiguous CPU tensor of `dtype`, >= nbytes)."""
    if not isinstance(t, torch.Tensor) or t.is_cuda or not t.is_contiguous():
        raise ValueError(f"{name}: host buffers must be contiguous CPU tensors")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name}: expected {dtype}, got {t.dtype}")
    if nbytes is not None and _nbytes(t) < nbytes:
        raise ValueError(f"{name}: {_nbytes(t)} bytes, the library needs {nbytes}")
    return t.data_ptr()


def _field_bytes(cfg: "Config", dtype: torch.dtype, fields: int = 5) -> int:
    return fields * cfg.n ** 3 * torch.tensor([], dtype=dtype).element_size()


def _nrec(nsteps: int, diag_every: int) -> int:
    return nsteps // diag_every + 1 if diag_every > 0 else 0


def _stream(stream) -> int | None:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


# ------------------------------------------------------------------ host-only
def tgv_check_config(cfg: Config) -> int:
    return lib().tgv_check_config(C.byref(cfg.c()))


def tgv_state_bytes(cfg: Config) -> int:
    return lib().tgv_state_bytes(C.byref(cfg.c()))


def tgv_qt_bytes(cfg: Config) -> int:
    return lib().tgv_qt_bytes(C.byref(cfg.c()))


def tgv_dt_max(cfg: Config) -> float:
    return lib().tgv_dt_max(C.byref(cfg.c()))


def tgv_workspace_bytes(cfg: Config) -> int:
    return lib().tgv_workspace_bytes(C.byref(cfg.c()))


def tgv_tile_shapes() -> list[tuple[int, int]]:
    out = []
    for t in range(1, lib().tgv_tile_count() + 1):
        tx, ty = C.c_int32(), C.c_int32()
        check(lib().tgv_tile_shape(t, C.byref(tx), C.byref(ty)), "tgv_tile_shape")
        out.append((tx.value, ty.value))
    return out


# ------------------------------------------------------------ allocation help
def empty_state(cfg: Config, device="cuda") -> torch.Tensor:
    """A (5, N, N, N) tensor of the Q storage type."""
    return torch.empty((5, cfg.n, cfg.n, cfg.n), dtype=cfg.q_dtype, device=device)


def empty_qt(cfg: Config, device="cuda") -> torch.Tensor:
    return torch.empty((5, cfg.n, cfg.n, cfg.n), dtype=cfg.qt_dtype, device=device)


def empty_workspace(cfg: Config, device="cuda") -> torch.Tensor:
    return torch.empty(max(tgv_workspace_bytes(cfg), 8), dtype=torch.uint8, device=device)


# ------------------------------------------------------------------ C entries
def _q(cfg: Config, t, name: str) -> int:
    return _dev(t, name, cfg.q_dtype, tgv_state_bytes(cfg))


def _qt(cfg: Config, t, name: str) -> int:
    return _dev(t, name, cfg.qt_dtype, tgv_qt_bytes(cfg))


def _ws(t, name: str = "workspace"):
    """(pointer, bytes) of an optional device workspace; the library checks the size."""
    if t is None:
        return None, 0
    return _dev(t, name), _nbytes(t)


def tgv_init(cfg: Config, q: torch.Tensor, stream=None) -> None:
    pq = _q(cfg, q, "q")
    check(lib().tgv_init(C.byref(cfg.c()), pq, _stream(stream)), "tgv_init")


def rhs_eval(cfg: Config, q: torch.Tensor, r: torch.Tensor, stream=None) -> None:
    pq = _q(cfg, q, "q")
    pr = _dev(r, "r", cfg.compute_dtype, _field_bytes(cfg, cfg.compute_dtype))
    check(lib().rhs_eval(C.byref(cfg.c()), pq, pr, _stream(stream)), "rhs_eval")


def rk_substep(cfg: Config, q_in, q_out, qt, i: int, dt: float, stream=None) -> None:
    args = (_q(cfg, q_in, "q_in"), _q(cfg, q_out, "q_out"), _qt(cfg, qt, "qt"))
    check(lib().rk_substep(C.byref(cfg.c()), *args, int(i), float(dt), _stream(stream)),
          "rk_substep")


def rk_step(cfg: Config, q_a, q_b, qt, dt: float, nsteps: int, diag_every: int = 0,
            diag=None, workspace=None, stream=None) -> int:
    """Advance nsteps; returns the parity (0: result in q_a, 1: in q_b)."""
    par = C.c_int32(-1)
    pa, pb, pt = _q(cfg, q_a, "q_a"), _q(cfg, q_b, "q_b"), _qt(cfg, qt, "qt")
    nrec = _nrec(int(nsteps), int(diag_every))
    pd = _dev(diag, "diag", torch.float64, nrec * TGV_DIAG_COUNT * 8) if nrec else _ptr(diag)
    pw, ws_bytes = _ws(workspace)
    check(lib().rk_step(C.byref(cfg.c()), pa, pb, pt, float(dt), int(nsteps), int(diag_every),
                        pd, pw, ws_bytes, C.byref(par), _stream(stream)), "rk_step")
    return par.value


def diagnostics_reduce(cfg: Config, q, out, workspace, stream=None) -> None:
    pq = _q(cfg, q, "q")
    po = _dev(out, "out", torch.float64, TGV_DIAG_COUNT * 8)
    pw, ws_bytes = _ws(workspace)
    check(lib().diagnostics_reduce(C.byref(cfg.c()), pq, po, pw, ws_bytes, _stream(stream)),
          "diagnostics_reduce")


def diagnostics_reduce_noalloc(cfg: Config, q, out, stream=None) -> None:
    """diagnostics_reduce with the partial sums in the library's own fixed
    device array instead of a caller workspace (for callers that cannot
    allocate device memory); calls that overlap on the GPU race."""
    pq = _q(cfg, q, "q")
    po = _dev(out, "out", torch.float64, TGV_DIAG_COUNT * 8)
    check(lib().diagnostics_reduce_noalloc(C.byref(cfg.c()), pq, po, _stream(stream)),
          "diagnostics_reduce_noalloc")


def tgv_run_host_workspace_bytes(cfg: Config, nsteps: int, diag_every: int) -> int:
    return lib().tgv_run_host_workspace_bytes(C.byref(cfg.c()), int(nsteps), int(diag_every))


def tgv_run_host(cfg: Config, q_host_in, q_host_out, dt: float, nsteps: int,
                 diag_every: int = 0, diag_host=None, dev_workspace=None, stream=None) -> None:
    """End-to-end call with host (CPU, ideally pinned) tensors."""
    qb = tgv_state_bytes(cfg)
    pin = _host(q_host_in, "q_host_in", cfg.q_dtype, qb)
    pout = _host(q_host_out, "q_host_out", cfg.q_dtype, qb)
    nrec = _nrec(int(nsteps), int(diag_every))
    pd = (_host(diag_host, "diag_host", torch.float64, nrec * TGV_DIAG_COUNT * 8)
          if diag_host is not None else None)
    pw, ws_bytes = _ws(dev_workspace, "dev_workspace")
    check(lib().tgv_run_host(C.byref(cfg.c()), pin, pout, float(dt), int(nsteps),
                             int(diag_every), pd, pw, ws_bytes, _stream(stream)), "tgv_run_host")


def tgv_run_host_stream_workspace_bytes(cfg: Config, nsteps: int, diag_every: int) -> int:
    return lib().tgv_run_host_stream_workspace_bytes(C.byref(cfg.c()), int(nsteps),
                                                     int(diag_every))


def tgv_run_host_stream(cfg: Config, qs_host_in, qs_host_out, dt: float, nsteps: int,
                        diag_every: int = 0, diag_host=None, dev_workspace=None,
                        compute_stream=None, copy_stream=None) -> None:
    """Several independent states from host (CPU, ideally pinned) tensors, the
    copies overlapped with the steps on a second stream (tgv_run_host_stream)."""
    qs_host_in, qs_host_out = list(qs_host_in), list(qs_host_out)
    if len(qs_host_in) != len(qs_host_out):
        raise ValueError("as many output buffers as input buffers")
    if copy_stream is None:
        raise ValueError("copy_stream is required (a stream other than the compute stream)")
    qb = tgv_state_bytes(cfg)
    count = len(qs_host_in)
    p_in = [_host(q, f"q_host_in[{i}]", cfg.q_dtype, qb) for i, q in enumerate(qs_host_in)]
    p_out = [_host(q, f"q_host_out[{i}]", cfg.q_dtype, qb) for i, q in enumerate(qs_host_out)]
    nrec = _nrec(int(nsteps), int(diag_every))
    pd = (_host(diag_host, "diag_host", torch.float64, count * nrec * TGV_DIAG_COUNT * 8)
          if diag_host is not None else None)
    pw, ws_bytes = _ws(dev_workspace, "dev_workspace")
    arr_in = (C.c_void_p * max(count, 1))(*p_in)
    arr_out = (C.c_void_p * max(count, 1))(*p_out)
    check(lib().tgv_run_host_stream(C.byref(cfg.c()), count, arr_in, arr_out, float(dt),
                                    int(nsteps), int(diag_every), pd, pw, ws_bytes,
                                    _stream(compute_stream), _stream(copy_stream)),
          "tgv_run_host_stream")


# ------------------------------------------------------------------ z-slabs
def _slab(z0: int, nz: int) -> _abi.tgv_slab:
    return _abi.tgv_slab(z0=int(z0), nz=int(nz))


def tgv_slab_state_bytes(cfg: Config, z0: int, nz: int) -> int:
    return lib().tgv_slab_state_bytes(C.byref(cfg.c()), C.byref(_slab(z0, nz)))


def tgv_slab_qt_bytes(cfg: Config, z0: int, nz: int) -> int:
    return lib().tgv_slab_qt_bytes(C.byref(cfg.c()), C.byref(_slab(z0, nz)))


def empty_slab_state(cfg: Config, nz: int, device="cuda") -> torch.Tensor:
    """A (5, nz + 4, N, N) slab state of the Q storage type (2 ghost planes
    below and above the owned planes)."""
    return torch.empty((5, nz + 4, cfg.n, cfg.n), dtype=cfg.q_dtype, device=device)


def empty_slab_qt(cfg: Config, nz: int, device="cuda") -> torch.Tensor:
    return torch.empty((5, nz, cfg.n, cfg.n), dtype=cfg.qt_dtype, device=device)


def tgv_slab_init(cfg: Config, z0: int, nz: int, q, stream=None) -> None:
    pq = _dev(q, "q", cfg.q_dtype, tgv_slab_state_bytes(cfg, z0, nz))
    check(lib().tgv_slab_init(C.byref(cfg.c()), C.byref(_slab(z0, nz)), pq, _stream(stream)),
          "tgv_slab_init")


def tgv_slab_substep(cfg: Config, z0: int, nz: int, q_in, q_out, qt, i: int, dt: float,
                     diag=None, workspace=None, stream=None) -> None:
    qb = tgv_slab_state_bytes(cfg, z0, nz)
    pi, po = _dev(q_in, "q_in", cfg.q_dtype, qb), _dev(q_out, "q_out", cfg.q_dtype, qb)
    pt = _dev(qt, "qt", cfg.qt_dtype, tgv_slab_qt_bytes(cfg, z0, nz))
    pd = _dev(diag, "diag", torch.float64, TGV_DIAG_COUNT * 8) if diag is not None else None
    pw, ws_bytes = _ws(workspace)
    check(lib().tgv_slab_substep(C.byref(cfg.c()), C.byref(_slab(z0, nz)), pi, po, pt, int(i),
                                 float(dt), pd, pw, ws_bytes, _stream(stream)),
          "tgv_slab_substep")


def tgv_slab_exchange_local(cfg: Config, slabs, qs, stream=None) -> None:
    """Ghost exchange among slabs (list of (z0, nz), tiling [0, N) in order)
    whose states qs all live on the current device."""
    if len(slabs) != len(qs) or not slabs:
        raise ValueError("one state per slab")
    ptrs = [_dev(q, f"q[{r}]", cfg.q_dtype, tgv_slab_state_bytes(cfg, *sl))
            for r, (sl, q) in enumerate(zip(slabs, qs))]
    arr = (_abi.tgv_slab * len(slabs))(*[_slab(*sl) for sl in slabs])
    check(lib().tgv_slab_exchange_local(C.byref(cfg.c()), len(slabs), arr,
                                        (C.c_void_p * len(qs))(*ptrs), _stream(stream)),
          "tgv_slab_exchange_local")


# -------------------------------------------------------------- measurement
PROBE_KINDS = {"ffma": 0, "ffma2": 1, "hfma2": 2}


def probe_fma_tflops(kind: str, iters: int = 4096, blocks_per_sm: int = 8, reps: int = 5) -> float:
    """Throughput of the FMA pipe in one arithmetic form (scalar FP32, paired
    FP32, packed FP16), TFLOP/s: the best of `reps` timed launches of the
    library's probe kernel (tgv_probe_fma) on the current device."""
    dev = torch.cuda.current_device()
    blocks = blocks_per_sm * torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.empty(blocks * 256, dtype=torch.float32, device="cuda")
    flops = C.c_double(0.0)
    stream = torch.cuda.current_stream()
    best = None
    for r in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        check(lib().tgv_probe_fma(PROBE_KINDS[kind], int(iters), blocks, _dev(sink, "sink"),
                                  sink.numel(), C.byref(flops), _stream(stream)), "tgv_probe_fma")
        e1.record(stream)
        e1.synchronize()
        if r:  # the first launch is a warm-up
            t = flops.value / (e0.elapsed_time(e1) * 1e-3) / 1e12
            best = t if best is None else max(best, t)
    return best


def diagnostics(cfg: Config, q: torch.Tensor, workspace=None) -> dict:
    """Convenience: diagnostics_reduce into a fresh tensor, returned as a dict."""
    ws = workspace if workspace is not None else empty_workspace(cfg, q.device)
    out = torch.empty(TGV_DIAG_COUNT, dtype=torch.float64, device=q.device)
    diagnostics_reduce(cfg, q, out, ws)
    return dict(zip(DIAG_NAMES, out.cpu().tolist()))


# ------------------------------------------------------------------- adjoint
def tgv_adjoint_workspace_bytes(cfg: Config) -> int:
    return lib().tgv_adjoint_workspace_bytes(C.byref(cfg.c()))


def rhs_vjp(cfg: Config, q, lam, q_bar, workspace=None, stream=None) -> None:
    """q_bar = (dR/dQ)^T lam at state q (FP64 cotangents)."""
    f64 = _field_bytes(cfg, torch.float64)
    pq = _q(cfg, q, "q")
    pl, pb = _dev(lam, "lam", torch.float64, f64), _dev(q_bar, "q_bar", torch.float64, f64)
    ws = workspace if workspace is not None else torch.empty(
        tgv_adjoint_workspace_bytes(cfg), dtype=torch.uint8, device=q.device)
    pw, ws_bytes = _ws(ws)
    check(lib().rhs_vjp(C.byref(cfg.c()), pq, pl, pb, pw, ws_bytes, _stream(stream)), "rhs_vjp")


def rk_step_adjoint(cfg: Config, stage_inputs, q_bar, dt: float, workspace=None,
                    stream=None) -> None:
    """One RK3 step backwards; stage_inputs is a (3, 5, N, N, N) tensor."""
    ps = _dev(stage_inputs, "stage_inputs", cfg.q_dtype, 3 * tgv_state_bytes(cfg))
    pb = _dev(q_bar, "q_bar", torch.float64, _field_bytes(cfg, torch.float64))
    ws = workspace if workspace is not None else torch.empty(
        tgv_adjoint_workspace_bytes(cfg), dtype=torch.uint8, device=q_bar.device)
    pw, ws_bytes = _ws(ws)
    check(lib().rk_step_adjoint(C.byref(cfg.c()), ps, pb, float(dt), pw, ws_bytes,
                                _stream(stream)), "rk_step_adjoint")


def tgv_grad_workspace_bytes(cfg: Config, nsteps: int, ckpt_every: int) -> int:
    return lib().tgv_grad_workspace_bytes(C.byref(cfg.c()), int(nsteps), int(ckpt_every))


def tgv_grad_final_ke(cfg: Config, q0, dt: float, nsteps: int, ckpt_every: int, grad_mom,
                      j_out, workspace=None, stream=None) -> None:
    pq = _q(cfg, q0, "q0")
    pg = _dev(grad_mom, "grad_mom", torch.float64, _field_bytes(cfg, torch.float64, 3))
    pj = _dev(j_out, "j_out", torch.float64, 8)
    ws = workspace if workspace is not None else torch.empty(
        tgv_grad_workspace_bytes(cfg, nsteps, ckpt_every), dtype=torch.uint8, device=q0.device)
    pw, ws_bytes = _ws(ws)
    check(lib().tgv_grad_final_ke(C.byref(cfg.c()), pq, float(dt), int(nsteps),
                                  int(ckpt_every), pg, pj, pw, ws_bytes, _stream(stream)),
          "tgv_grad_final_ke")


class TGVFinalKE(torch.autograd.Function):
    """J = K(Q_nsteps) as a function of the initial momentum (rho u, rho v,
    rho w) with the initial density and total energy held fixed; backward uses
    the discrete adjoint (tgv_grad_final_ke), with uniform checkpointing."""

    @staticmethod
    def forward(ctx, rho_u, rho_v, rho_w, rho, rho_E, cfg: Config, dt: float, nsteps: int,
                ckpt_every: int):
        q0 = torch.stack([rho, rho_u, rho_v, rho_w, rho_E]).to(cfg.q_dtype).contiguous()
        grad = torch.empty((3,) + tuple(rho.shape), dtype=torch.float64, device=q0.device)
        j = torch.empty(1, dtype=torch.float64, device=q0.device)
        tgv_grad_final_ke(cfg, q0, dt, nsteps, ckpt_every, grad, j)
        ctx.save_for_backward(grad)
        return j[0].clone()

    @staticmethod
    def backward(ctx, g):
        (grad,) = ctx.saved_tensors
        gg = g.to(torch.float64) * grad
        return gg[0], gg[1], gg[2], None, None, None, None, None, None


# ------------------------------------------------------------------ ensemble
class Ensemble:
    """Owner of a tgv_ensemble handle: `count` TGV instances of uneven size,
    all in one precision mode, advanced together (one persistent launch per RK
    stage, replayed from a CUDA graph of steps_per_graph steps).  Buffers are torch tensors the
    caller keeps alive; q_a[i] holds instance i's state after every run()."""

    def __init__(self, cfgs, q_a, q_b, qt, dts, steps_per_graph: int = 10, stream=None):
        n = len(cfgs)
        arr = (_abi.tgv_config * n)(*[c.c() for c in cfgs])
        if not (len(q_a) == len(q_b) == len(qt) == len(dts) == n):
            raise ValueError("one q_a, q_b, qt and dt per instance")
        pa = [_q(c, t, f"q_a[{i}]") for i, (c, t) in enumerate(zip(cfgs, q_a))]
        pb = [_q(c, t, f"q_b[{i}]") for i, (c, t) in enumerate(zip(cfgs, q_b))]
        pt = [_qt(c, t, f"qt[{i}]") for i, (c, t) in enumerate(zip(cfgs, qt))]
        ptrs = lambda ps: (C.c_void_p * n)(*ps)
        self._keep = (list(q_a), list(q_b), list(qt))
        handle = C.c_void_p()
        check(lib().tgv_ensemble_create(arr, n, ptrs(pa), ptrs(pb), ptrs(pt),
                                        (C.c_double * n)(*[float(d) for d in dts]),
                                        int(steps_per_graph), _stream(stream), C.byref(handle)),
              "tgv_ensemble_create")
        self.handle = handle
        self.steps_per_graph = int(steps_per_graph)

    def run(self, replays: int = 1, stream=None) -> None:
        check(lib().tgv_ensemble_run(self.handle, int(replays), _stream(stream)),
              "tgv_ensemble_run")

    def info(self) -> dict:
        vals = [C.c_int32() for _ in range(5)]
        check(lib().tgv_ensemble_info(self.handle, *[C.byref(v) for v in vals]),
              "tgv_ensemble_info")
        keys = ("tile", "zchunk_target", "grid", "items", "steps_per_graph")
        return dict(zip(keys, (v.value for v in vals)))

    def close(self) -> None:
        if self.handle:
            check(lib().tgv_ensemble_destroy(self.handle), "tgv_ensemble_destroy")
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def ensemble_instances(draws=None, device="cuda", mode: str = "fp32", encoding: str = "plain"):
    """The 48-instance ensemble workload: (cfgs, dts) from tgv_inputs'
    seeded draws, dt_i = min(0.004, 0.8 dt_max,i); FP32 by default, any
    precision mode on request."""
    import tgv_inputs
    draws = draws if draws is not None else tgv_inputs.ensemble_draws()
    cfgs, dts = [], []
    for n, re, m in draws:
        c = Config(n=n, mode=mode, re=re, mach=m, encoding=encoding)
        cfgs.append(c)
        dts.append(min(0.004, 0.8 * tgv_dt_max(c)))
    return cfgs, dts
