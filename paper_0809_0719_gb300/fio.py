"""Thin Python binding of the C ABI in include/fio.h (argument marshalling only).

Every step of the butterfly runs in the CUDA library libfio.so; this module only
checks tensor shapes, dtypes and devices, passes raw pointers and the current
CUDA stream, and turns status codes into exceptions.  There is no CPU path: if
the library cannot be built or loaded, every call raises.

Operator (Candes, Demanet & Ying 2008, eq. dfio): u(x) = sum_k e^{2 pi i Phi(x,k)} f(k)
on N x N grids.  Tensors are (nrhs, N, N) complex (complex128 for precision
"f64", complex64 for "f32"); f[r, k1 + N/2, k2 + N/2] is the source at k,
u[r, i1, i2] the potential at x = (i1/N, i2/N).
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

FIO_OK, FIO_EINVAL, FIO_ENOMEM, FIO_ECUDA, FIO_ETIMEOUT, FIO_EDEVICE = 0, -1, -2, -3, -4, -5
F64, F32 = 0, 1
PHASES = {"linear": 0, "ellipse": 1, "circle": 2, "separable": 3}
PRECISIONS = {"f64": F64, "f32": F32}

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_HERE, "libfio.so")
_lock = threading.Lock()
_lib = None


class FIOError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("fio status %d: %s" % (code, msg))
        self.code = code


class KernelTime(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 24), ("launches", ctypes.c_longlong), ("ms", ctypes.c_double)]


class PlanInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in ("N", "L", "q", "s", "e", "l0", "lm", "l1", "phase_id", "precision",
                                            "nrhs_max", "nstages")] + [
        ("pairs_per_level", ctypes.c_longlong), ("state_bytes", ctypes.c_longlong),
        ("table_bytes", ctypes.c_longlong), ("max_box_sources", ctypes.c_int), ("switch_impl", ctypes.c_int),
        ("trans_rs", ctypes.c_int), ("switch_rhs_tile", ctypes.c_int), ("trans_rs_x", ctypes.c_int)]


class PlanInfo3(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in ("N", "L", "q", "s", "e", "l0", "lm", "l1", "phase_id", "nrhs_max")] + [
        ("pairs_per_level", ctypes.c_longlong), ("state_bytes", ctypes.c_longlong),
        ("table_bytes", ctypes.c_longlong), ("max_box_sources", ctypes.c_int)]


class BatchInfo(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int) for n in ("nplans", "ngroups", "launches_fwd", "launches_adj", "parallel_groups",
                                            "tuned")] + [("total_elems", ctypes.c_longlong), ("tune_ms", ctypes.c_double)]


def lib() -> ctypes.CDLL:
    """Load libfio.so, building it first (nvcc, sm_103a) if it is missing or stale."""
    global _lib
    with _lock:
        if _lib is None:
            from . import build as _build

            path = _build.build()
            L = ctypes.CDLL(path)
            vp, ip = ctypes.c_void_p, ctypes.c_int
            L.fio_plan.argtypes = [ctypes.POINTER(vp), ip, ip, ip, ctypes.POINTER(ctypes.c_double), ip, ip, ip, ip, ip]
            L.fio_destroy.argtypes = [vp]
            L.fio_apply.argtypes = [vp, vp, vp, ip, vp]
            L.fio_apply_adjoint.argtypes = [vp, vp, vp, ip, vp]
            L.fio_apply_host.argtypes = [vp, vp, vp, ip, ip, vp]
            L.fio_debug_stage.argtypes = [vp, vp, ip, vp, vp]
            L.fio_plan_info.argtypes = [vp, ctypes.POINTER(PlanInfo)]
            L.fio_kernel_launches.argtypes = [vp, ip, ip]
            L.fio_profile.argtypes = [vp, ip]
            L.fio_profile_read.argtypes = [vp, ctypes.POINTER(KernelTime), ip, ctypes.POINTER(ip)]
            L.fio_peak_probe.argtypes = [ip, ctypes.POINTER(ctypes.c_double)]
            L.fio_plan_set_switch.argtypes = [vp, ip]
            L.fio_plan_set_wait_limit.argtypes = [vp, ctypes.c_ulonglong]
            L.fio_plan_set_tuning.argtypes = [vp, ip, ip, ip, ip]
            L.fio_direct.argtypes = [vp, vp, ip, vp, ip, vp, vp]
            L.fio_apply_amplitude.argtypes = [vp, vp, vp, vp, ip, vp, ip, ip, vp]
            L.fio_apply_wave.argtypes = [vp, vp, vp, vp, ip, ctypes.c_double, ctypes.c_double, ip, vp]
            L.fio_apply_wave_series.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ip, vp, vp, ip, vp]
            L.fio_plan_auto.argtypes = [ctypes.POINTER(vp), ip, ip, ctypes.POINTER(ctypes.c_double), ip, ip, ip, ip,
                                        ip, ctypes.c_double, ip, ctypes.c_ulonglong, ctypes.POINTER(ip),
                                        ctypes.POINTER(ctypes.c_double)]
            L.fio_check.argtypes = [vp, vp]
            L.fio_batch_create.argtypes = [ctypes.POINTER(vp), ip, ctypes.POINTER(vp), ctypes.POINTER(ip), ip]
            L.fio_batch_destroy.argtypes = [vp]
            L.fio_batch_offsets.argtypes = [vp, ctypes.POINTER(ctypes.c_longlong)]
            L.fio_batch_apply.argtypes = [vp, vp, vp, ip, vp]
            L.fio_batch_info.argtypes = [vp, ctypes.POINTER(BatchInfo)]
            L.fio_batch_profile.argtypes = [vp, vp, vp, ip, vp, ctypes.POINTER(KernelTime), ip, ctypes.POINTER(ip)]
            L.fio_apply_batch.argtypes = [ctypes.POINTER(vp), ip, ctypes.POINTER(vp), ctypes.POINTER(vp),
                                          ctypes.POINTER(ip), vp]
            L.fio_apply_batch_adjoint.argtypes = L.fio_apply_batch.argtypes
            L.fio_workspace_bytes.argtypes = [vp, ip]
            L.fio_workspace_bytes.restype = ctypes.c_size_t
            L.fio3_plan.argtypes = [ctypes.POINTER(vp), ip, ip, ip, ctypes.POINTER(ctypes.c_double), ip, ip, ip, ip]
            L.fio3_destroy.argtypes = [vp]
            L.fio3_apply.argtypes = [vp, vp, vp, ip, vp]
            L.fio3_apply_adjoint.argtypes = [vp, vp, vp, ip, vp]
            L.fio3_plan_info.argtypes = [vp, ctypes.POINTER(PlanInfo3)]
            L.fio_last_error.restype = ctypes.c_char_p
            _lib = L
        return _lib


def _check(rc: int) -> None:
    if rc != FIO_OK:
        raise FIOError(rc, lib().fio_last_error().decode())


def _stream_ptr(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream)


class Plan:
    """A butterfly plan: fio_plan(N, q, phase, params, precision, nrhs_max, s, e)."""

    def __init__(self, N: int, q: int, phase="ellipse", params=(2.0, 1.0, 16.0, 1.0), precision="f32",
                 nrhs_max: int = 1, s: int = -1, e: int = -1):
        self._h = None
        L = lib()
        pid = PHASES[phase] if isinstance(phase, str) else int(phase)
        prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        prm = [] if pid == 0 else list(params)
        arr = (ctypes.c_double * max(1, len(prm)))(*prm)
        h = ctypes.c_void_p()
        _check(L.fio_plan(ctypes.byref(h), N, q, pid, arr, len(prm), prec, nrhs_max, s, e))
        self._h = h
        self.info = PlanInfo()
        _check(L.fio_plan_info(h, ctypes.byref(self.info)))
        self.N, self.q = N, q
        self.dtype = torch.complex128 if prec == F64 else torch.complex64

    def close(self) -> None:
        if self._h is not None and _lib is not None:
            _lib.fio_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev_tensor(self, x: torch.Tensor, name: str) -> torch.Tensor:
        if not isinstance(x, torch.Tensor) or not x.is_cuda:
            raise TypeError("%s must be a CUDA tensor" % name)
        if x.dtype != self.dtype:
            raise TypeError("%s must be %s for this plan, got %s" % (name, self.dtype, x.dtype))
        if x.dim() == 2:
            x = x.unsqueeze(0)
        if x.shape[-2:] != (self.N, self.N):
            raise ValueError("%s must have shape (nrhs, %d, %d), got %s" % (name, self.N, self.N, tuple(x.shape)))
        return x.contiguous()

    def apply(self, f: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """u = B f (fio_apply) on the current (or given) CUDA stream."""
        f = self._dev_tensor(f, "f")
        u = torch.empty_like(f) if out is None else out
        _check(lib().fio_apply(self._h, f.data_ptr(), u.data_ptr(), f.shape[0], _stream_ptr(stream)))
        return u

    def adjoint(self, g: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """fbar = B^H g (fio_apply_adjoint)."""
        g = self._dev_tensor(g, "g")
        fb = torch.empty_like(g) if out is None else out
        _check(lib().fio_apply_adjoint(self._h, g.data_ptr(), fb.data_ptr(), g.shape[0], _stream_ptr(stream)))
        return fb

    def apply_host(self, x: torch.Tensor, out: torch.Tensor, adjoint: bool = False, stream=None) -> torch.Tensor:
        """fio_apply_host: host (ideally pinned) input and output; copies happen inside the call."""
        if x.is_cuda or out.is_cuda or x.dtype != self.dtype or out.dtype != self.dtype:
            raise TypeError("apply_host takes CPU tensors of dtype %s" % self.dtype)
        if not (x.is_contiguous() and out.is_contiguous()):
            raise ValueError("apply_host needs contiguous tensors")
        n = x.shape[0] if x.dim() == 3 else 1
        _check(lib().fio_apply_host(self._h, x.data_ptr(), out.data_ptr(), n, int(adjoint), _stream_ptr(stream)))
        return out

    def debug_stage(self, f: torch.Tensor, stage: int, stream=None) -> torch.Tensor:
        """State after `stage` as complex128 (a1, a2, b1, b2, t1, t2) (fio_debug_stage, RHS 0 of f)."""
        f = self._dev_tensor(f, "f")[:1].contiguous()
        out = torch.empty(self.info.pairs_per_level * self.q * self.q, dtype=torch.complex128, device=f.device)
        _check(lib().fio_debug_stage(self._h, f.data_ptr(), stage, out.data_ptr(), _stream_ptr(stream)))
        return out

    def apply_amplitude(self, x: torch.Tensor, g: torch.Tensor, h: torch.Tensor, adjoint: bool = False,
                        out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """fio_apply_amplitude: the FIO with amplitude a(x,k) = sum_t g[t](x) h[t](k) (eq. allfio),
        or its conjugate transpose.  x, out: (nrhs, N, N); g, h: (nt, N, N)."""
        x = self._dev_tensor(x, "input")
        g = self._dev_tensor(g, "g")
        h = self._dev_tensor(h, "h")
        if g.shape[0] != h.shape[0]:
            raise ValueError("g and h must have the same number of terms")
        out = torch.empty_like(x) if out is None else self._dev_tensor(out, "out")
        _check(lib().fio_apply_amplitude(self._h, x.data_ptr(), g.data_ptr(), h.data_ptr(), g.shape[0], out.data_ptr(),
                                         x.shape[0], int(adjoint), _stream_ptr(stream)))
        return out

    def direct(self, f: torch.Tensor, xi: torch.Tensor, stream=None) -> torch.Tensor:
        """fio_direct: the direct sum of eq. dfio at flat grid indices xi (int64 CUDA tensor);
        returns (nrhs, len(xi)) complex128."""
        f = self._dev_tensor(f, "f")
        if not isinstance(xi, torch.Tensor) or not xi.is_cuda or xi.dtype != torch.int64 or xi.dim() != 1:
            raise TypeError("xi must be a 1-D int64 CUDA tensor")
        xi = xi.contiguous()
        nrhs = f.shape[0]
        out = torch.empty(nrhs, xi.numel(), dtype=torch.complex128, device=f.device)
        _check(lib().fio_direct(self._h, f.data_ptr(), nrhs, xi.data_ptr(), xi.numel(), out.data_ptr(),
                                _stream_ptr(stream)))
        return out

    def set_switch(self, impl: int) -> None:
        """fio_plan_set_switch: 0 = FP32 FMA switch kernel, 1 = tensor-core switch kernel
        (kernel matrix in shared memory), 2 = warp-specialised persistent FP32 FMA switch
        kernel, 3 = tensor-core switch kernel with the kernel matrix in tensor memory, 4 = as 3 with
        two wide MMAs per K-step, 5 and 6 = as 3 and 4 with three split-TF32 products instead of five."""
        _check(lib().fio_plan_set_switch(self._h, int(impl)))
        self.info.switch_impl = int(impl)

    def set_tuning(self, switch_impl: int = -1, switch_rhs_tile: int = -1, trans_rs: int = -1,
                   trans_rs_x: int = -1) -> None:
        """fio_plan_set_tuning: override the autotuner's choices (-1 keeps one)."""
        _check(lib().fio_plan_set_tuning(self._h, int(switch_impl), int(switch_rhs_tile), int(trans_rs),
                                         int(trans_rs_x)))
        _check(lib().fio_plan_info(self._h, ctypes.byref(self.info)))

    def set_wait_limit(self, ns: int) -> None:
        """fio_plan_set_wait_limit: limit of the tensor-memory switch's hand-off waits (0 = normal)."""
        _check(lib().fio_plan_set_wait_limit(self._h, int(ns)))

    def check(self, stream=None) -> None:
        """fio_check: synchronise and raise if a bounded device-side wait expired."""
        _check(lib().fio_check(self._h, _stream_ptr(stream)))

    def workspace_bytes(self, nrhs: int) -> int:
        """fio_workspace_bytes: device bytes of the two state levels for nrhs RHS."""
        return int(lib().fio_workspace_bytes(self._h, int(nrhs)))

    def kernel_launches(self, nrhs: int, adjoint: bool = False) -> int:
        return int(lib().fio_kernel_launches(self._h, nrhs, int(adjoint)))

    def profile(self, enable: bool) -> None:
        """fio_profile: start (clearing the counters) or stop per-kernel event timing."""
        _check(lib().fio_profile(self._h, int(enable)))

    def profile_read(self) -> dict:
        """fio_profile_read: {kernel kind: (launches, total ms)} since profile(True)."""
        buf = (KernelTime * 16)()
        n = ctypes.c_int()
        _check(lib().fio_profile_read(self._h, buf, 16, ctypes.byref(n)))
        return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].ms)) for i in range(n.value)}


class Plan3:
    """The three-dimensional butterfly (include/fio3.h), FP64: fio3_plan(N, q, phase, params,
    nrhs_max, s, e).  Tensors are (nrhs, N, N, N) complex128; f[r, k1+N/2, k2+N/2, k3+N/2] is the
    source at k, u[r, i1, i2, i3] the potential at x = (i1, i2, i3)/N."""

    PHASES3 = {"linear": 0, "sphere": 2}

    def __init__(self, N: int, q: int, phase="sphere", params=(3.0, 1.0, 4.0, 1.0), nrhs_max: int = 1, s: int = -1,
                 e: int = -1):
        self._h = None
        L = lib()
        pid = self.PHASES3[phase] if isinstance(phase, str) else int(phase)
        prm = [] if pid == 0 else list(params)
        arr = (ctypes.c_double * max(1, len(prm)))(*prm)
        h = ctypes.c_void_p()
        _check(L.fio3_plan(ctypes.byref(h), N, q, pid, arr, len(prm), nrhs_max, s, e))
        self._h = h
        self.info = PlanInfo3()
        _check(L.fio3_plan_info(h, ctypes.byref(self.info)))
        self.N, self.q = N, q
        self.dtype = torch.complex128

    def close(self) -> None:
        if self._h is not None and _lib is not None:
            _lib.fio3_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _dev(self, x: torch.Tensor, name: str) -> torch.Tensor:
        if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != torch.complex128:
            raise TypeError("%s must be a complex128 CUDA tensor" % name)
        if x.dim() == 3:
            x = x.unsqueeze(0)
        if tuple(x.shape[-3:]) != (self.N,) * 3:
            raise ValueError("%s must have shape (nrhs, %d, %d, %d)" % ((name,) + (self.N,) * 3))
        return x.contiguous()

    def apply(self, f: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """u = B f (fio3_apply)."""
        f = self._dev(f, "f")
        u = torch.empty_like(f) if out is None else out
        _check(lib().fio3_apply(self._h, f.data_ptr(), u.data_ptr(), f.shape[0], _stream_ptr(stream)))
        return u

    def adjoint(self, g: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        """fbar = B^H g (fio3_apply_adjoint)."""
        g = self._dev(g, "g")
        fb = torch.empty_like(g) if out is None else out
        _check(lib().fio3_apply_adjoint(self._h, g.data_ptr(), fb.data_ptr(), g.shape[0], _stream_ptr(stream)))
        return fb


class Batch:
    """fio_batch_create over FP32 plans: one persistent launch per butterfly step and
    q-group, replayed from a captured CUDA graph.  Inputs and outputs are packed
    complex64 vectors; plan i occupies [offsets[i], offsets[i+1]) as its
    (nrhs[i], N_i, N_i) array.  The plans must stay alive while the batch does."""

    def __init__(self, plans, nrhs, tune: bool = False, serial: bool = False):
        self._h = None
        L = lib()
        self.plans = list(plans)
        n = len(self.plans)
        ph = (ctypes.c_void_p * n)(*[p._h for p in self.plans])
        nr = (ctypes.c_int * n)(*[int(r) for r in nrhs])
        h = ctypes.c_void_p()
        _check(L.fio_batch_create(ctypes.byref(h), n, ph, nr, (1 if tune else 0) | (2 if serial else 0)))
        self._h = h
        off = (ctypes.c_longlong * (n + 1))()
        _check(L.fio_batch_offsets(h, off))
        self.offsets = [int(v) for v in off]
        self.nrhs = [int(r) for r in nrhs]
        self.info = BatchInfo()
        _check(L.fio_batch_info(h, ctypes.byref(self.info)))

    def close(self) -> None:
        if self._h is not None and _lib is not None:
            _lib.fio_batch_destroy(self._h)
        self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _io(self, x: torch.Tensor, out, name: str):
        total = self.offsets[-1]
        if not isinstance(x, torch.Tensor) or not x.is_cuda or x.dtype != torch.complex64:
            raise TypeError("%s must be a complex64 CUDA tensor" % name)
        if x.numel() != total or not x.is_contiguous():
            raise ValueError("%s must be contiguous with %d elements" % (name, total))
        if out is None:
            out = torch.empty(total, dtype=torch.complex64, device=x.device)
        elif out.dtype != torch.complex64 or out.numel() != total or not out.is_contiguous() or not out.is_cuda:
            raise ValueError("out must be a contiguous complex64 CUDA tensor with %d elements" % total)
        return out

    def apply(self, x: torch.Tensor, out: torch.Tensor | None = None, adjoint: bool = False, stream=None):
        """fio_batch_apply on a packed buffer; returns the packed output."""
        out = self._io(x, out, "input")
        _check(lib().fio_batch_apply(self._h, x.data_ptr(), out.data_ptr(), int(adjoint), _stream_ptr(stream)))
        return out

    def profile(self, x: torch.Tensor, adjoint: bool = False, stream=None) -> dict:
        """fio_batch_profile: one eager pass, {kernel kind: (launches, total ms)}."""
        out = self._io(x, None, "input")
        buf = (KernelTime * 16)()
        n = ctypes.c_int()
        _check(lib().fio_batch_profile(self._h, x.data_ptr(), out.data_ptr(), int(adjoint), _stream_ptr(stream), buf,
                                       16, ctypes.byref(n)))
        return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].ms)) for i in range(n.value)}

    def pack(self, tensors) -> torch.Tensor:
        """Concatenate per-plan (nrhs, N, N) complex64 CUDA tensors into one packed buffer."""
        return torch.cat([t.reshape(-1) for t in tensors]).contiguous()

    def unpack(self, packed: torch.Tensor):
        """Per-plan (nrhs, N, N) views of a packed buffer."""
        return [packed[self.offsets[i]:self.offsets[i + 1]].view(self.nrhs[i], p.N, p.N)
                for i, p in enumerate(self.plans)]


def apply_batch(plans, xs, outs=None, adjoint: bool = False, stream=None):
    """fio_apply_batch (adjoint: fio_apply_batch_adjoint): every FP32 plan i applied to its own
    (nrhs_i, N_i, N_i) complex64 CUDA tensor xs[i] in one graph launch (the library keeps the
    batch of these plans and counts for later calls).  Returns the list of outputs."""
    plans = list(plans)
    n = len(plans)
    if len(xs) != n:
        raise ValueError("one input per plan")
    xs = [p._dev_tensor(x, "input %d" % i) for i, (p, x) in enumerate(zip(plans, xs))]
    outs = [torch.empty_like(x) for x in xs] if outs is None else [p._dev_tensor(o, "out") for p, o in zip(plans, outs)]
    ph = (ctypes.c_void_p * n)(*[p._h for p in plans])
    pin = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
    pout = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    nr = (ctypes.c_int * n)(*[x.shape[0] for x in xs])
    fn = lib().fio_apply_batch_adjoint if adjoint else lib().fio_apply_batch
    _check(fn(ph, n, pin, pout, nr, _stream_ptr(stream)))
    return outs


def plan_auto(N: int, target: float, phase="ellipse", params=(2.0, 1.0, 16.0, 1.0), precision="f32",
              nrhs_max: int = 1, s: int = -1, e: int = -1, nsample: int = 256, seed: int = 0):
    """fio_plan_auto: the plan of the smallest q in (3, 5, 7, 9, 11) whose estimated error
    (eq. err on nsample seeded points) meets target.  Returns (plan, q, estimated error)."""
    L = lib()
    pid = PHASES[phase] if isinstance(phase, str) else int(phase)
    prec = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    prm = [] if pid == 0 else list(params)
    arr = (ctypes.c_double * max(1, len(prm)))(*prm)
    h = ctypes.c_void_p()
    q = ctypes.c_int()
    err = ctypes.c_double()
    _check(L.fio_plan_auto(ctypes.byref(h), N, pid, arr, len(prm), prec, nrhs_max, s, e, float(target), nsample,
                           seed, ctypes.byref(q), ctypes.byref(err)))
    plan = Plan.__new__(Plan)
    plan._h = h
    plan.info = PlanInfo()
    _check(L.fio_plan_info(h, ctypes.byref(plan.info)))
    plan.N, plan.q = N, q.value
    plan.dtype = torch.complex128 if prec == F64 else torch.complex64
    return plan, q.value, err.value


def wave_plans(N: int, q: int, a: float, m: float, b: float, t: float, precision="f32", nrhs_max: int = 1,
               s: int = -1, e: int = -1):
    """The two circle-phase plans of the wave propagator at time t (Sec. 1): phases
    x.k + c(x)|k|t and x.k - c(x)|k|t, c(x) = (a + m sin 2 pi x1 sin 2 pi x2)/b."""
    plus = Plan(N, q, "circle", (a * t, m * t, b, 1.0), precision, nrhs_max, s, e)
    minus = Plan(N, q, "circle", (-a * t, -m * t, b, 1.0), precision, nrhs_max, s, e)
    return plus, minus


def apply_wave(plus: Plan, minus: Plan, x: torch.Tensor, w_plus: float = 0.5, w_minus: float = 0.5,
               adjoint: bool = False, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """fio_apply_wave: out = w_plus B_plus x + w_minus B_minus x (or the sum of the adjoints);
    with wave_plans and the default weights 1/2, u(x, t) for u_t(x, 0) = 0."""
    x = plus._dev_tensor(x, "input")
    out = torch.empty_like(x) if out is None else plus._dev_tensor(out, "out")
    _check(lib().fio_apply_wave(plus._h, minus._h, x.data_ptr(), out.data_ptr(), x.shape[0], float(w_plus),
                                float(w_minus), int(adjoint), _stream_ptr(stream)))
    return out


def apply_wave_series(plan: Plan, times, x: torch.Tensor, out: torch.Tensor | None = None, stream=None):
    """fio_apply_wave_series: u(t_k) = (B_{+t_k} x + B_{-t_k} x)/2 for every t_k from one circle-phase
    plan (its params give the speed at t = 1); returns (ntimes, nrhs, N, N)."""
    x = plan._dev_tensor(x, "input")
    times = [float(t) for t in times]
    shape = (len(times),) + tuple(x.shape)
    out = torch.empty(shape, dtype=x.dtype, device=x.device) if out is None else out
    if tuple(out.shape) != shape or out.dtype != x.dtype or not out.is_contiguous():
        raise ValueError("out must be a contiguous %s tensor of shape %s" % (x.dtype, shape))
    ts = (ctypes.c_double * len(times))(*times)
    _check(lib().fio_apply_wave_series(plan._h, ts, len(times), x.data_ptr(), out.data_ptr(), x.shape[0],
                                       _stream_ptr(stream)))
    return out


def peak_probe(kind: str) -> float:
    """fio_peak_probe on the current device: 'fp32' / 'fp64' flop/s or 'sfu' sin/s."""
    v = ctypes.c_double()
    kinds = {"fp32": 0, "fp64": 1, "sfu": 2, "mma_tf32_n64": 3, "mma_bf16_n64": 4, "mma_tf32_n256": 5,
             "mma_bf16_n256": 6, "mma_tf32_n64_smem_a": 7, "mma_bf16_n64_smem_a": 8,
             "mma_tf32_n64_3acc": 9, "mma_tf32_n64_2acc": 10}
    _check(lib().fio_peak_probe(kinds[kind], ctypes.byref(v)))
    return float(v.value)


class FIOFunction(torch.autograd.Function):
    """u = B f with backward grad_f = B^H grad_u (the hand-written adjoint butterfly)."""

    @staticmethod
    def forward(ctx, f, plan):
        ctx.plan = plan
        return plan.apply(f)

    @staticmethod
    def backward(ctx, grad_u):
        return ctx.plan.adjoint(grad_u.contiguous()), None


def fio_apply(f: torch.Tensor, plan: Plan) -> torch.Tensor:
    """Differentiable apply."""
    return FIOFunction.apply(f, plan)
