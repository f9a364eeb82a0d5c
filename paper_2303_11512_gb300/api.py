"""Python binding of the MG-MLMC++ library: the C-ABI calls under the same
names, taking torch CUDA tensors (complex128 for FP64/MIXED vectors,
complex64 for FP32) and returning plain Python/numpy results.

Vectors are [nrhs, n] tensors (row-major, so the C layout [rhs][site][dof]),
gauge fields [L, L, 2] complex128 tensors on the GPU.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import (ACCUMULATED, BF16, FP16, FP32, FP64, MIXED, NOISE_RADEMACHER, NOISE_Z4, OPTIMAL, REDUCED, TF32,
                   TRACE_GAMMA5, TRACE_PLAIN, UNIFORM, EstParams, EstResult, HutchParams, HutchResult, MgParams,
                   SolveParams, SolveStats, check)

__all__ = ["Context", "Hierarchy", "Sketch", "schwinger_apply", "mgmlmc_rademacher", "mg_setup",
           "fgmres_batched", "mlmc_level_sample", "mg_restrict_to_level", "hutchpp_sketch_qr",
           "hutchpp_project", "trace_estimate", "hutchinson_estimate", "mgmlmc_noise", "mlmc_update_active",
           "FP64", "FP32", "FP16", "MIXED", "ACCUMULATED", "REDUCED", "OPTIMAL", "UNIFORM", "NOISE_RADEMACHER", "NOISE_Z4",
           "TRACE_PLAIN", "TRACE_GAMMA5"]


def _ptr(t: torch.Tensor, dtype=None) -> int:
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError("expected dtype %s, got %s" % (dtype, t.dtype))
    return t.data_ptr()


# The C entry points receive bare device pointers and sizes and cannot see a tensor's shape or device, so every
# wrapper checks both before the call: a vector tensor of the wrong size would become an out-of-bounds device
# access, and one on another GPU a launch on the wrong device's memory.
def _rows(name: str, t: torch.Tensor, n: int) -> int:
    """Rows of the vector tensor t: [nrhs, n], or [n] as one row."""
    if t.dim() == 1 and t.shape[0] == n:
        return 1
    if t.dim() != 2 or t.shape[1] != n:
        raise ValueError("%s must be [nrhs, %d], got %s" % (name, n, tuple(t.shape)))
    return int(t.shape[0])


def check_vectors(device, *spec) -> int:
    """spec: (name, tensor, n) triples, each tensor [nrhs, n] with one common nrhs and, unless device is None, on
    `device`.  Returns nrhs; raises ValueError on a mismatch."""
    nrhs = None
    for name, t, n in spec:
        r = _rows(name, t, n)
        if nrhs is None:
            nrhs = r
        elif r != nrhs:
            raise ValueError("%s has %d rows, %d expected" % (name, r, nrhs))
        if device is not None and t.device != device:
            raise ValueError("%s is on %s, the launches go to %s" % (name, t.device, device))
    return nrhs


def check_field(device, U: torch.Tensor, L: int):
    """Gauge links U must be [L, L, 2] (on `device` unless it is None); raises ValueError."""
    if tuple(U.shape) != (L, L, 2):
        raise ValueError("U must be [%d, %d, 2], got %s" % (L, L, tuple(U.shape)))
    if device is not None and U.device != device:
        raise ValueError("U is on %s, the launches go to %s" % (U.device, device))


def check_level(level: int, top: int):
    if not 0 <= level < top:
        raise ValueError("level %d outside 0 .. %d" % (level, top - 1))


def _dev(ctx) -> torch.device:
    """The device the context's launches go to: that of its stream."""
    return ctx.stream.device


def _vec_dtype(prec: int):
    return torch.complex64 if prec in (FP32, TF32, BF16, FP16) else torch.complex128


class Context:
    """Library context bound to a CUDA stream (default: torch's current stream)."""

    def __init__(self, stream: torch.cuda.Stream | None = None):
        lib = _lib.load()
        s = stream if stream is not None else torch.cuda.current_stream()
        self.stream = s
        h = C.c_void_p()
        check(lib.mgmlmc_ctx_create(C.c_void_p(s.cuda_stream), C.byref(h)))
        self.ptr = h

    @property
    def launches(self) -> int:
        return int(_lib.load().mgmlmc_launch_count(self.ptr))

    def timing(self, on: bool = True, filter: str | None = None):
        """Bracket launches of kernels whose name contains `filter` with CUDA events."""
        check(_lib.load().mgmlmc_timing_enable(self.ptr, int(on), filter.encode() if filter else None))

    def timing_report(self) -> dict:
        """{kernel: dict(launches, ms, bytes, flops)} for the launches recorded since the last report."""
        buf = C.create_string_buffer(1 << 16)
        check(_lib.load().mgmlmc_timing_report(self.ptr, buf, len(buf)), self.ptr)
        out = {}
        for line in buf.value.decode().splitlines():
            name, n, ms, by, fl = line.split("\t")
            out[name] = dict(launches=int(n), ms=float(ms), bytes=float(by), flops=float(fl))
        return out

    def close(self):
        if self.ptr:
            _lib.load().mgmlmc_ctx_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def schwinger_apply(ctx: Context, U: torch.Tensor, L: int, m0: float, x: torch.Tensor, y: torch.Tensor,
                    prec: int = FP64):
    """y = D x (fine Schwinger operator); x, y [nrhs, 2 L^2]."""
    dt = _vec_dtype(prec)
    check_field(_dev(ctx), U, L)
    nrhs = check_vectors(_dev(ctx), ("x", x, 2 * L * L), ("y", y, 2 * L * L))
    check(_lib.load().schwinger_apply(ctx.ptr, _ptr(U, torch.complex128), L, m0, _ptr(x, dt), _ptr(y, dt),
                                      nrhs, prec), ctx.ptr)


def mgmlmc_rademacher(ctx: Context, seed: int, level: int, phase: int, sample0: int, n: int, nrhs: int,
                      out: torch.Tensor | None = None) -> torch.Tensor:
    if out is None:
        out = torch.empty((nrhs, n), dtype=torch.complex128, device=_dev(ctx))
    elif check_vectors(_dev(ctx), ("out", out, n)) != nrhs:
        raise ValueError("out must be [%d, %d], got %s" % (nrhs, n, tuple(out.shape)))
    check(_lib.load().mgmlmc_rademacher(ctx.ptr, seed, level, phase, sample0, n, nrhs,
                                        _ptr(out, torch.complex128)), ctx.ptr)
    return out


def mgmlmc_noise(ctx: Context, kind: int, seed: int, level: int, phase: int, sample0: int, n: int, nrhs: int,
                 out: torch.Tensor | None = None) -> torch.Tensor:
    """Rademacher (kind NOISE_RADEMACHER) or Z4 (NOISE_Z4) vectors of the counter-based streams."""
    if out is None:
        out = torch.empty((nrhs, n), dtype=torch.complex128, device=_dev(ctx))
    elif check_vectors(_dev(ctx), ("out", out, n)) != nrhs:
        raise ValueError("out must be [%d, %d], got %s" % (nrhs, n, tuple(out.shape)))
    check(_lib.load().mgmlmc_noise(ctx.ptr, kind, seed, level, phase, sample0, n, nrhs,
                                   _ptr(out, torch.complex128)), ctx.ptr)
    return out


def mg_params(**kw) -> MgParams:
    p = MgParams()
    _lib.load().mg_params_default(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def solve_params(**kw) -> SolveParams:
    p = SolveParams()
    _lib.load().solve_params_default(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


class Hierarchy:
    def __init__(self, ctx: Context, handle: C.c_void_p, L: int, m0: float):
        self.ctx, self.ptr, self.L, self.m0 = ctx, handle, L, m0
        lib = _lib.load()
        self.levels = lib.mg_num_levels(handle)
        self.side, self.dof, self.n = [], [], []
        for l in range(self.levels):
            s, d, n = C.c_int(), C.c_int(), C.c_int64()
            check(lib.mg_level_info(handle, l, C.byref(s), C.byref(d), C.byref(n)))
            self.side.append(s.value)
            self.dof.append(d.value)
            self.n.append(n.value)

    def coarsest_trace(self) -> complex:
        t = (C.c_double * 2)()
        check(_lib.load().mg_coarsest_trace(self.ptr, t))
        return complex(t[0], t[1])

    def apply(self, level: int, x: torch.Tensor, y: torch.Tensor, prec: int = FP64):
        dt = _vec_dtype(prec)
        check_level(level, self.levels)
        nrhs = check_vectors(_dev(self.ctx), ("x", x, self.n[level]), ("y", y, self.n[level]))
        check(_lib.load().mg_apply(self.ctx.ptr, self.ptr, level, _ptr(x, dt), _ptr(y, dt), nrhs, prec),
              self.ctx.ptr)

    def restrict(self, level: int, xf: torch.Tensor, xc: torch.Tensor, prec: int = FP64):
        dt = _vec_dtype(prec)
        check_level(level, self.levels - 1)
        nrhs = check_vectors(_dev(self.ctx), ("xf", xf, self.n[level]), ("xc", xc, self.n[level + 1]))
        check(_lib.load().mg_restrict(self.ctx.ptr, self.ptr, level, _ptr(xf, dt), _ptr(xc, dt), nrhs, prec),
              self.ctx.ptr)

    def prolong(self, level: int, xc: torch.Tensor, xf: torch.Tensor, prec: int = FP64):
        dt = _vec_dtype(prec)
        check_level(level, self.levels - 1)
        nrhs = check_vectors(_dev(self.ctx), ("xc", xc, self.n[level + 1]), ("xf", xf, self.n[level]))
        check(_lib.load().mg_prolong(self.ctx.ptr, self.ptr, level, _ptr(xc, dt), _ptr(xf, dt), nrhs, prec),
              self.ctx.ptr)

    def smooth(self, level: int, f: torch.Tensor, x: torch.Tensor, prec: int = FP64, sweeps: int = 1):
        """SAP sweeps for D_l x = f, x updated in place (prec FP64, FP32, or TF32 / BF16 on the tensor cores)."""
        dt = _vec_dtype(prec)
        check_level(level, self.levels)
        nrhs = check_vectors(_dev(self.ctx), ("f", f, self.n[level]), ("x", x, self.n[level]))
        check(_lib.load().mg_smooth(self.ctx.ptr, self.ptr, level, _ptr(f, dt), _ptr(x, dt), nrhs, prec, sweeps),
              self.ctx.ptr)

    def tc_status(self) -> int:
        return _lib.load().mg_tc_status(self.ctx.ptr, self.ptr)

    def autotune(self, nrhs_list=(8, 16, 32, 64, 128, 256), force: bool = False):
        """Time the launch variants of this hierarchy's tunable kernels and record the fastest (mg_autotune)."""
        arr = (C.c_int * len(nrhs_list))(*nrhs_list)
        check(_lib.load().mg_autotune(self.ctx.ptr, self.ptr, arr, len(nrhs_list), int(force)), self.ctx.ptr)

    def vcycle(self, level: int, b: torch.Tensor, x: torch.Tensor, prec: int = FP64):
        dt = _vec_dtype(prec)
        check_level(level, self.levels)
        nrhs = check_vectors(_dev(self.ctx), ("b", b, self.n[level]), ("x", x, self.n[level]))
        check(_lib.load().mg_vcycle(self.ctx.ptr, self.ptr, level, _ptr(b, dt), _ptr(x, dt), nrhs, prec),
              self.ctx.ptr)

    def get_prolongator(self, level: int, agg: int, ntv: int) -> np.ndarray:
        Lc = self.side[level + 1]
        bsz = agg * agg * self.dof[level] // 2
        out = np.empty((Lc * Lc, 2, bsz, ntv), dtype=np.complex128)
        check(_lib.load().mg_get_prolongator(self.ctx.ptr, self.ptr, level, out.ctypes.data), self.ctx.ptr)
        return out

    def get_stencil(self, level: int) -> np.ndarray:
        s, d = self.side[level], self.dof[level]
        out = np.empty((s * s, 5, d, d), dtype=np.complex128)
        check(_lib.load().mg_get_stencil(self.ctx.ptr, self.ptr, level, out.ctypes.data), self.ctx.ptr)
        return out

    def close(self):
        if self.ptr:
            _lib.load().mg_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


TUNE_KINDS = {0: "fine stencil (FP32)", 1: "tensor-core stencil", 2: "tensor-core SAP block update"}


def alu_peak(ctx: Context, fp64: bool) -> float:
    """Measured CUDA-core FMA throughput (TFLOP/s) of the current device, FP64 or FP32."""
    v = C.c_double()
    check(_lib.load().mgmlmc_alu_peak(ctx.ptr, 1 if fp64 else 0, C.byref(v)), ctx.ptr)
    return v.value


def tune_table() -> list:
    """The process-wide launch-variant table: [dict(device, kind, side, bucket, format, variant, us)]."""
    buf = C.create_string_buffer(1 << 16)
    check(_lib.load().mgmlmc_tune_report(buf, len(buf)))
    out = []
    for line in buf.value.decode().splitlines():
        dev, kind, side, bucket, fmt, var, us = line.split("\t")
        out.append(dict(device=int(dev), kind=int(kind), side=int(side), bucket=int(bucket), format=int(fmt),
                        variant=int(var), us=float(us)))
    return out


def tune_set(entries):
    """Load entries (as tune_table returns them) into the table of the current device."""
    for e in entries:
        check(_lib.load().mgmlmc_tune_set(e["kind"], e["side"], e["bucket"], e["format"], e["variant"]))


def tune_clear():
    """Drop the table's entries of the current device (later launches take the default variants)."""
    check(_lib.load().mgmlmc_tune_clear())


def mg_setup(ctx: Context, U: torch.Tensor, L: int, m0: float, **params) -> Hierarchy:
    check_field(_dev(ctx), U, L)
    p = mg_params(**params)
    h = C.c_void_p()
    check(_lib.load().mg_setup(ctx.ptr, _ptr(U, torch.complex128), L, m0, C.byref(p), C.byref(h)), ctx.ptr)
    return Hierarchy(ctx, h, L, m0)


def _stats(st: SolveStats) -> dict:
    return dict(iters=st.iters, outer=st.outer, max_relres=st.max_relres, converged=bool(st.converged),
                total_iters=st.total_iters)


def fgmres_batched(ctx: Context, h: Hierarchy, level: int, b: torch.Tensor, x: torch.Tensor,
                   raise_on_nonconvergence: bool = True, **solve) -> dict:
    check_level(level, h.levels)
    nrhs = check_vectors(_dev(ctx), ("b", b, h.n[level]), ("x", x, h.n[level]))
    sp = solve_params(**solve)
    dt = _vec_dtype(sp.prec)
    st = SolveStats()
    its = np.zeros(nrhs, dtype=np.int32)
    rc = _lib.load().fgmres_batched(ctx.ptr, h.ptr, level, _ptr(b, dt), _ptr(x, dt), nrhs, C.byref(sp),
                                    C.byref(st), its.ctypes.data)
    if rc != _lib.ERR_NOT_CONVERGED or raise_on_nonconvergence:
        check(rc, ctx.ptr)
    d = _stats(st)
    d["its"] = its
    return d


def mlmc_level_sample(ctx: Context, h: Hierarchy, level: int, zeta: torch.Tensor, y: torch.Tensor,
                      form: int = REDUCED, **solve) -> dict:
    """Level difference `level` applied to zeta: level-size vectors (REDUCED) or fine-size vectors
    (ACCUMULATED, y = Phat A Rhat zeta)."""
    check_level(level, h.levels - 1)
    n = h.n[0] if form == ACCUMULATED else h.n[level]
    nrhs = check_vectors(_dev(ctx), ("zeta", zeta, n), ("y", y, n))
    sp = solve_params(**solve)
    st = SolveStats()
    check(_lib.load().mlmc_level_sample(ctx.ptr, h.ptr, level, form, _ptr(zeta, torch.complex128),
                                        _ptr(y, torch.complex128), nrhs, C.byref(sp), C.byref(st)),
          ctx.ptr)
    return _stats(st)


def mg_restrict_to_level(ctx: Context, h: Hierarchy, level: int, zeta_fine: torch.Tensor,
                         out: torch.Tensor | None = None) -> torch.Tensor:
    check_level(level, h.levels)
    nrhs = check_vectors(_dev(ctx), ("zeta_fine", zeta_fine, h.n[0]))
    if out is None:
        out = torch.empty((nrhs, h.n[level]), dtype=torch.complex128, device=_dev(ctx))
    check_vectors(_dev(ctx), ("zeta_fine", zeta_fine, h.n[0]), ("out", out, h.n[level]))
    check(_lib.load().mg_restrict_to_level(ctx.ptr, h.ptr, level, _ptr(zeta_fine, torch.complex128),
                                           _ptr(out, torch.complex128), nrhs), ctx.ptr)
    return out


class Sketch:
    def __init__(self, ctx: Context, handle: C.c_void_p):
        self.ctx, self.ptr = ctx, handle
        d, n = C.c_int(), C.c_int64()
        check(_lib.load().hutchpp_sketch_get_q(ctx.ptr, handle, None, C.byref(d), C.byref(n)), ctx.ptr)
        self.d, self.n = d.value, n.value

    def Q(self) -> torch.Tensor:
        q = torch.empty((self.d, self.n), dtype=torch.complex128, device=_dev(self.ctx))
        check(_lib.load().hutchpp_sketch_get_q(self.ctx.ptr, self.ptr, _ptr(q), None, None), self.ctx.ptr)
        torch.cuda.synchronize()
        return q

    def close(self):
        if self.ptr:
            _lib.load().hutchpp_sketch_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hutchpp_sketch_qr(ctx: Context, h: Hierarchy, level: int, d: int, k: int, seed: int,
                      form: int = ACCUMULATED, **solve):
    sp = solve_params(**solve)
    s = C.c_void_p()
    t = (C.c_double * 2)()
    check(_lib.load().hutchpp_sketch_qr(ctx.ptr, h.ptr, level, d, k, seed, form, C.byref(sp), C.byref(s), t),
          ctx.ptr)
    return Sketch(ctx, s), complex(t[0], t[1])


def mg_dense_inverse(ctx: Context, A: torch.Tensor, prec: int = FP64, barrier_polls: int = 0):
    """In-place inverse of the square device matrix A (complex128 for FP64, complex64 for FP32)."""
    if A.dim() != 2 or A.shape[0] != A.shape[1]:
        raise ValueError("A must be square")
    check_vectors(_dev(ctx), ("A", A, A.shape[1]))
    check(_lib.load().mg_dense_inverse(ctx.ptr, _ptr(A, _vec_dtype(prec)), A.shape[0], prec, barrier_polls),
          ctx.ptr)


def hutchpp_cholqr2(ctx: Context, Y: torch.Tensor):
    """In-place CholeskyQR2 of the basis Y [d, n] (rows are the vectors), complex128."""
    if Y.dim() != 2:
        raise ValueError("Y must be [d, n]")
    check_vectors(_dev(ctx), ("Y", Y, Y.shape[1]))
    check(_lib.load().hutchpp_cholqr2(ctx.ptr, _ptr(Y, torch.complex128), Y.shape[0], Y.shape[1]), ctx.ptr)


def hutchpp_project(ctx: Context, sketch: Sketch | None, zeta: torch.Tensor, y: torch.Tensor) -> np.ndarray:
    if zeta.dim() != 2:
        raise ValueError("zeta must be [nrhs, n], got %s" % (tuple(zeta.shape),))
    n = int(zeta.shape[1])
    if sketch is not None and sketch.d > 0 and sketch.n != n:
        raise ValueError("the sketch's basis has vectors of %d entries, zeta of %d" % (sketch.n, n))
    nrhs = check_vectors(_dev(ctx), ("zeta", zeta, n), ("y", y, n))
    out = np.empty(nrhs, dtype=np.complex128)
    check(_lib.load().hutchpp_project(ctx.ptr, sketch.ptr if sketch else None, _ptr(zeta, torch.complex128),
                                      _ptr(y, torch.complex128), n, nrhs,
                                      out.ctypes.data_as(C.POINTER(C.c_double))), ctx.ptr)
    return out


class Net:
    """Learned gauge-covariant correction M ~ D^{-1} (see include/mgmlmc.h, nn_*)."""

    def __init__(self, ctx: Context, U: torch.Tensor, L: int, layers: int = 4, channels: int = 16, seed: int = 0,
                 tensor_cores: bool | None = None):
        """tensor_cores: True = BF16 tcgen05 layers, False = FP32 CUDA-core layers, None = the library's
        default (tensor cores where L is a multiple of 16)."""
        check_field(_dev(ctx), U, L)
        self.ctx, self.L = ctx, L
        h = C.c_void_p()
        check(_lib.load().nn_create(ctx.ptr, _ptr(U, torch.complex128), L, layers, channels, seed, C.byref(h)),
              ctx.ptr)
        self.ptr = h
        self.nparams = int(_lib.load().nn_num_params(h))
        if tensor_cores is not None:
            self.set_format(1 if tensor_cores else 0)

    def set_format(self, fmt: int):
        check(_lib.load().nn_set_format(self.ctx.ptr, self.ptr, fmt), self.ctx.ptr)

    @property
    def format(self) -> int:
        return int(_lib.load().nn_get_format(self.ptr))

    def set_field(self, U: torch.Tensor, L: int):
        """Rebind to another gauge field (weights and Adam state kept)."""
        check_field(_dev(self.ctx), U, L)
        check(_lib.load().nn_set_field(self.ctx.ptr, self.ptr, _ptr(U, torch.complex128), L), self.ctx.ptr)
        self.L = L

    def set_params(self, p: np.ndarray):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.nparams
        check(_lib.load().nn_set_params(self.ctx.ptr, self.ptr, p.ctypes.data), self.ctx.ptr)

    def get_params(self) -> np.ndarray:
        p = np.empty(self.nparams, dtype=np.float32)
        check(_lib.load().nn_get_params(self.ctx.ptr, self.ptr, p.ctypes.data), self.ctx.ptr)
        return p

    def forward(self, r: torch.Tensor, y: torch.Tensor | None = None) -> torch.Tensor:
        y = torch.empty_like(r) if y is None else y
        n = 2 * self.L * self.L
        nrhs = check_vectors(_dev(self.ctx), ("r", r, n), ("y", y, n))
        check(_lib.load().nn_forward(self.ctx.ptr, self.ptr, _ptr(r, torch.complex64), _ptr(y, torch.complex64),
                                     nrhs), self.ctx.ptr)
        return y

    def loss_grad(self, r: torch.Tensor, e: torch.Tensor):
        n = 2 * self.L * self.L
        nrhs = check_vectors(_dev(self.ctx), ("r", r, n), ("e", e, n))
        loss = C.c_double()
        g = np.empty(self.nparams, dtype=np.float32)
        check(_lib.load().nn_loss_grad(self.ctx.ptr, self.ptr, _ptr(r, torch.complex64), _ptr(e, torch.complex64),
                                       nrhs, C.byref(loss), g.ctypes.data), self.ctx.ptr)
        return loss.value, g

    def train_step(self, r: torch.Tensor, e: torch.Tensor, lr: float = 1e-3) -> float:
        n = 2 * self.L * self.L
        nrhs = check_vectors(_dev(self.ctx), ("r", r, n), ("e", e, n))
        loss = C.c_double()
        check(_lib.load().nn_train_step(self.ctx.ptr, self.ptr, _ptr(r, torch.complex64), _ptr(e, torch.complex64),
                                        nrhs, lr, C.byref(loss)), self.ctx.ptr)
        return loss.value

    def attach(self, h: "Hierarchy"):
        check(_lib.load().mg_attach_nn(self.ctx.ptr, h.ptr, self.ptr), self.ctx.ptr)

    def close(self):
        if self.ptr:
            _lib.load().nn_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def nn_harvest_pairs(ctx: Context, h: "Hierarchy", count: int, seed: int = 3, sample0: int = 0,
                     tol: float = 1e-6):
    """Training pairs (R, E) [count, n_0] complex64 from the hierarchy's own V-cycle and FP32 solves
    (R = (zeta - D V zeta)/|.|, E = (D^{-1} zeta - V zeta)/|.|; see nn_harvest_pairs in the header)."""
    n = h.n[0]
    R = torch.empty((count, n), dtype=torch.complex64, device=_dev(ctx))
    E = torch.empty_like(R)
    check(_lib.load().nn_harvest_pairs(ctx.ptr, h.ptr, seed, sample0, count, tol, _ptr(R, torch.complex64),
                                       _ptr(E, torch.complex64)), ctx.ptr)
    return R, E


def pack_params(W, b) -> np.ndarray:
    """Flat float32 parameter vector from per-layer complex W[9][c_out][c_in] and real biases."""
    out = []
    for l, w in enumerate(W):
        w = np.asarray(w, complex)
        out.append(np.stack([w.real, w.imag], axis=-1).ravel())
        if l < len(W) - 1:
            out.append(np.asarray(b[l], float).ravel())
    return np.concatenate(out).astype(np.float32)


def unpack_params(p: np.ndarray, layers: int, channels: int):
    dims = [2] + [channels] * (layers - 1) + [2]
    W, b, o = [], [], 0
    for l in range(layers):
        ci, co = dims[l], dims[l + 1]
        cnt = 9 * co * ci
        w = p[o:o + 2 * cnt].reshape(9, co, ci, 2)
        W.append(w[..., 0] + 1j * w[..., 1])
        o += 2 * cnt
        if l < layers - 1:
            b.append(p[o:o + co].copy())
            o += co
    return W, b


def check_noalloc_args(Q, zeta, y, tau_out, device=None):
    """Shape and device checks of hutchpp_project_noalloc's tensors (the C entry point receives bare pointers
    and cannot check them): zeta and y [nrhs, n] alike, Q [d, n], tau_out with at least nrhs entries, every
    tensor on `device` (the device the launches go to; not checked when None).  Raises ValueError."""
    if zeta.dim() != 2:
        raise ValueError("zeta must be [nrhs, n]")
    nrhs, n = zeta.shape
    if tuple(y.shape) != (nrhs, n):
        raise ValueError("y must have the shape of zeta, %s, got %s" % (tuple(zeta.shape), tuple(y.shape)))
    if Q is not None and (Q.dim() != 2 or Q.shape[1] != n):
        raise ValueError("Q must be [d, %d], got %s" % (n, tuple(Q.shape)))
    if tau_out.numel() < nrhs:
        raise ValueError("tau_out holds %d entries, %d needed" % (tau_out.numel(), nrhs))
    if device is not None:
        for name, t in (("Q", Q), ("zeta", zeta), ("y", y), ("tau_out", tau_out)):
            if t is not None and t.device != device:
                raise ValueError("%s is on %s, the launches go to %s" % (name, t.device, device))
    return nrhs, n, (0 if Q is None else Q.shape[0])


def hutchpp_project_noalloc(Q: torch.Tensor | None, zeta: torch.Tensor, y: torch.Tensor,
                            tau_out: torch.Tensor, stream: torch.cuda.Stream | None = None):
    """Projected samples into the device tensor `tau_out` ([nrhs] complex128) without any
    device allocation inside the library (for callers that cannot allocate; see the header).
    The launches go to the current device on `stream` (default: its current stream); every tensor
    must live on that device."""
    s = stream if stream is not None else torch.cuda.current_stream()
    dev = torch.device("cuda", torch.cuda.current_device())
    if s.device != dev:
        raise ValueError("stream is on %s, the current device is %s" % (s.device, dev))
    nrhs, n, d = check_noalloc_args(Q, zeta, y, tau_out, dev)
    check(_lib.load().hutchpp_project_noalloc(C.c_void_p(s.cuda_stream), _ptr(Q, torch.complex128) if d else None,
                                              d, _ptr(zeta, torch.complex128), _ptr(y, torch.complex128), n, nrhs,
                                              _ptr(tau_out, torch.complex128)))


def trace_estimate(ctx: Context, h: Hierarchy, eps: float = 1e-3, d=32, k: int = 2, nrhs_max: int = 256,
                   nrhs_first: int = 32, policy: int = OPTIMAL, form: int = ACCUMULATED, seed: int = 0,
                   cost=None, cost_mode: int = 0, min_samples: int = 2, max_samples: int = 1 << 20,
                   keep_samples: int = 0, noise: int = NOISE_RADEMACHER, weight: int = TRACE_PLAIN,
                   **solve) -> dict:
    p = EstParams()
    lib = _lib.load()
    lib.est_params_default(C.byref(p))
    nd = h.levels - 1
    dl = [d] * nd if np.isscalar(d) else list(d)
    for l in range(nd):
        p.d[l] = int(dl[l])
        p.cost[l] = float(1.0 if cost is None else cost[l])
    p.eps, p.k, p.nrhs_max, p.nrhs_first = eps, k, nrhs_max, nrhs_first
    p.policy, p.form, p.seed, p.cost_mode = policy, form, seed, cost_mode
    p.min_samples, p.max_samples = min_samples, max_samples
    p.noise, p.weight = noise, weight
    p.solve = solve_params(**solve)
    bufs = []
    if keep_samples:
        for l in range(nd):
            b = np.zeros(2 * keep_samples, dtype=np.float64)
            bufs.append(b)
            p.sample_out[l] = b.ctypes.data_as(C.POINTER(C.c_double))
        p.sample_cap = keep_samples
    r = EstResult()
    check(lib.trace_estimate(ctx.ptr, h.ptr, C.byref(p), C.byref(r)), ctx.ptr)
    out = dict(tau=complex(r.tau[0], r.tau[1]), sigma=r.sigma, tau_L=complex(r.tau_L[0], r.tau_L[1]),
               N=[r.N[l] for l in range(nd)], computed=[r.computed[l] for l in range(nd)],
               mean=[complex(r.mean[l][0], r.mean[l][1]) for l in range(nd)],
               V=[r.V[l] for l in range(nd)], C=[r.C[l] for l in range(nd)],
               tau_lr=[complex(r.tau_lr[l][0], r.tau_lr[l][1]) for l in range(nd)],
               solves=r.solves, inner_iters=r.inner_iters, steps=r.steps, flops=r.flops)
    if keep_samples:
        out["samples"] = [bufs[l].view(np.complex128)[: min(keep_samples, out["computed"][l])] for l in range(nd)]
    return out


def deflation_basis(ctx: Context, h: Hierarchy, k: int, sweeps: int, seed: int = 0, **solve):
    """Deflation basis of the exactly deflated Hutchinson comparator: (Sketch with V [k, n_0], tau_defl,
    residual of the subspace)."""
    sp = solve_params(**solve)
    s = C.c_void_p()
    t = (C.c_double * 2)()
    res = C.c_double()
    check(_lib.load().deflation_basis(ctx.ptr, h.ptr, k, sweeps, seed, C.byref(sp), C.byref(s), t, C.byref(res)),
          ctx.ptr)
    return Sketch(ctx, s), complex(t[0], t[1]), res.value


def hutchinson_estimate(ctx: Context, h: Hierarchy, eps: float = 1e-2, seed: int = 0, nrhs_first: int = 32,
                        nrhs_max: int = 256, noise: int = NOISE_RADEMACHER, weight: int = TRACE_PLAIN,
                        min_samples: int = 2, max_samples: int = 1 << 20, keep_samples: int = 0,
                        deflate: "Sketch | None" = None, **solve) -> dict:
    """Plain Hutchinson (Algorithm 1) on the fine operator of h; with `deflate` (a deflation_basis) the exactly
    deflated estimator."""
    p = HutchParams()
    lib = _lib.load()
    lib.hutch_params_default(C.byref(p))
    p.eps, p.seed, p.nrhs_first, p.nrhs_max = eps, seed, nrhs_first, nrhs_max
    p.noise, p.weight, p.min_samples, p.max_samples = noise, weight, min_samples, max_samples
    p.solve = solve_params(**solve)
    p.deflate = deflate.ptr if deflate is not None else None
    buf = None
    if keep_samples:
        buf = np.zeros(2 * keep_samples, dtype=np.float64)
        p.sample_out = buf.ctypes.data_as(C.POINTER(C.c_double))
        p.sample_cap = keep_samples
    r = HutchResult()
    check(lib.hutchinson_estimate(ctx.ptr, h.ptr, C.byref(p), C.byref(r)), ctx.ptr)
    out = dict(tau=complex(r.tau[0], r.tau[1]), sigma=r.sigma, N=r.N, computed=r.computed, solves=r.solves,
               inner_iters=r.inner_iters, tau_defl=complex(r.tau_defl[0], r.tau_defl[1]))
    if keep_samples:
        out["samples"] = buf.view(np.complex128)[: min(keep_samples, r.computed)]
    return out


def mlmc_update_active(active, V, N, C_, eps: float, tau_abs: float, policy: int = OPTIMAL,
                       min_samples: int = 2):
    """Host-only stop test of Algorithm 2 (no GPU needed)."""
    nd = len(active)
    a = (C.c_int * nd)(*[int(x) for x in active])
    v = (C.c_double * nd)(*V)
    n = (C.c_int64 * nd)(*N)
    c = (C.c_double * nd)(*C_)
    check(_lib.load().mlmc_update_active(nd, a, v, n, c, eps, tau_abs, policy, min_samples))
    return [bool(x) for x in a]
