"""Python access to the FP64 CPU oracle (``fio_oracle.c``) -- TEST INFRASTRUCTURE ONLY.

The oracle is a plain, slow statement of the butterfly FIO method of Candes,
Demanet & Ying (2008) used to check the CUDA library.  Only the tests, the smoke
check and the CPU-baseline leg of the benchmark may import this module; the
library itself never does, and the oracle imports nothing from the library.

Array conventions (numpy, complex128):
  f, fbar : (N, N), f[k1 + N/2, k2 + N/2] is the source at frequency (k1, k2)   (Sec. 1, eq. dfio)
  u, g    : (N, N), u[i1, i2] is the potential at x = (i1/N, i2/N)
Butterfly parameters: q (Chebyshev points per dimension), s (truncation depth,
-1 = 3), lm (switch level, -1 = floor(L/2)), e (angular refinement of T_P: boxes
of width 2^-j in p1 and 2^-(j+e) in p2; e=0 is the square-box statement).
Phase ids: 0 linear x.k, 1 ellipse (eq. ex1 with params [a, m, b, lambda]),
2 circle (eq. ex2 phase with params [a, m, b, lambda]), 3 test-only separable phase.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fio_oracle.c")
_SRC3 = os.path.join(_HERE, "fio_oracle3.c")  # the three-dimensional form
_LIB = os.path.join(_HERE, "liboracle.so")

LINEAR, ELLIPSE, CIRCLE, SEPARABLE = 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile fio_oracle.c and fio_oracle3.c into liboracle.so (gcc, OpenMP) when missing or stale."""
    srcs = [_SRC, _SRC3]
    if force or not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(x) for x in srcs):
        tmp = _LIB + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-o", tmp] + srcs + ["-lm"])
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _L():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        lp = ctypes.POINTER(ctypes.c_long)
        vp = ctypes.c_void_p
        lib.orc_direct.argtypes = [ctypes.c_int, ctypes.c_int, dp, vp, ctypes.c_int, lp, vp]
        lib.orc_direct_adjoint.argtypes = [ctypes.c_int, ctypes.c_int, dp, vp, ctypes.c_int, lp, vp]
        lib.orc_direct_multi.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, vp, ctypes.c_int, lp, vp]
        lib.orc_butterfly.argtypes = [ctypes.c_int] * 3 + [dp] + [ctypes.c_int] * 3 + [vp, vp, ctypes.c_int, vp]
        lib.orc_butterfly_adjoint.argtypes = [ctypes.c_int] * 3 + [dp] + [ctypes.c_int] * 3 + [vp, vp]
        lib.orc_theta_xp.argtypes = [ctypes.c_int, dp, ctypes.c_int] + [ctypes.c_double] * 4
        lib.orc_theta_xp.restype = ctypes.c_double
        lib.orc_phi_k.argtypes = [ctypes.c_int, dp, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int]
        lib.orc_phi_k.restype = ctypes.c_double
        lib.orc_cheb_nodes.argtypes = [ctypes.c_int, dp]
        lib.orc3_spherical_map.argtypes = [ctypes.c_int] * 4 + [dp]
        lib.orc3_theta_xp.argtypes = [ctypes.c_int, dp, ctypes.c_int, dp, dp]
        lib.orc3_theta_xp.restype = ctypes.c_double
        lib.orc3_direct.argtypes = [ctypes.c_int, ctypes.c_int, dp, vp, ctypes.c_int, lp, vp]
        lib.orc3_butterfly.argtypes = [ctypes.c_int] * 3 + [dp] + [ctypes.c_int] * 3 + [vp, vp]
        lib.orc3_butterfly_adjoint.argtypes = [ctypes.c_int] * 3 + [dp] + [ctypes.c_int] * 3 + [vp, vp]
        lib.orc3_direct_adjoint.argtypes = [ctypes.c_int, ctypes.c_int, dp, vp, ctypes.c_int, lp, vp]
        lib.orc_lagrange_row.argtypes = [ctypes.c_int, ctypes.c_double, dp]
        lib.orc_polar_map.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
        lib.orc_num_stages.argtypes = [ctypes.c_int] * 3
        lib.orc_stage_level.argtypes = [ctypes.c_int] * 4
        lib.orc_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def _prm(params):
    p = np.zeros(4, dtype=np.float64)
    p[: len(params)] = params
    return p


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def threads() -> int:
    """OpenMP threads the oracle uses."""
    return int(_L().orc_threads())


def set_threads(n: int) -> None:
    _L().orc_set_threads(int(n))


def cheb_nodes(q: int) -> np.ndarray:
    """Chebyshev grid of order q on [-1/2, 1/2] (Sec. 3.2)."""
    z = np.zeros(q)
    _L().orc_cheb_nodes(q, _dp(z))
    return z


def lagrange(q: int, t: float) -> np.ndarray:
    """[L_0(t), ..., L_{q-1}(t)] on the order-q Chebyshev grid (Sec. 3.2)."""
    out = np.zeros(q)
    _L().orc_lagrange_row(q, float(t), _dp(out))
    return out


def polar(N: int, k1: int, k2: int):
    """p(k) of eq. polar: (p1, p2) in [0,1]^2."""
    p = np.zeros(2)
    _L().orc_polar_map(N, int(k1), int(k2), _dp(p))
    return float(p[0]), float(p[1])


def theta(phase_id, params, N, x, p) -> float:
    """theta(x, p) = N Psi(x, p) (Sec. 1.1)."""
    return float(_L().orc_theta_xp(phase_id, _dp(_prm(params)), N, x[0], x[1], p[0], p[1]))


def phi(phase_id, params, N, x, k) -> float:
    """Phi(x, k) at a lattice frequency k."""
    return float(_L().orc_phi_k(phase_id, _dp(_prm(params)), N, x[0], x[1], int(k[0]), int(k[1])))


def direct(N, phase_id, params, f, xi=None) -> np.ndarray:
    """Direct sum of eq. dfio at flat grid indices xi (default: all N^2 points)."""
    f = np.ascontiguousarray(f, dtype=np.complex128).reshape(N, N)
    xi = np.arange(N * N, dtype=np.int64) if xi is None else np.ascontiguousarray(xi, dtype=np.int64)
    u = np.zeros(len(xi), dtype=np.complex128)
    prm = _prm(params)
    _L().orc_direct(N, phase_id, _dp(prm), f.ctypes.data, len(xi),
                    xi.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), u.ctypes.data)
    return u


def direct_multi(N, phase_id, params, F, xi=None) -> np.ndarray:
    """Direct sum of eq. dfio for every source array of F (R, N, N) at flat grid indices xi;
    returns (R, len(xi)).  Each RHS equals direct() on it bit for bit (same order of terms);
    the phases are evaluated once per (x, k) for all RHS."""
    F = np.ascontiguousarray(F, dtype=np.complex128).reshape(-1, N, N)
    xi = np.arange(N * N, dtype=np.int64) if xi is None else np.ascontiguousarray(xi, dtype=np.int64)
    u = np.zeros((F.shape[0], len(xi)), dtype=np.complex128)
    prm = _prm(params)
    _L().orc_direct_multi(N, phase_id, _dp(prm), F.shape[0], F.ctypes.data, len(xi),
                          xi.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), u.ctypes.data)
    return u


def direct_adjoint(N, phase_id, params, g, ki=None) -> np.ndarray:
    """fbar(k) = sum_x e^{-2 pi i Phi(x,k)} g(x) at flat frequency indices ki (default: all)."""
    g = np.ascontiguousarray(g, dtype=np.complex128).reshape(N, N)
    ki = np.arange(N * N, dtype=np.int64) if ki is None else np.ascontiguousarray(ki, dtype=np.int64)
    out = np.zeros(len(ki), dtype=np.complex128)
    prm = _prm(params)
    _L().orc_direct_adjoint(N, phase_id, _dp(prm), g.ctypes.data, len(ki),
                            ki.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), out.ctypes.data)
    return out


def num_stages(N, s=-1, lm=-1) -> int:
    return int(_L().orc_num_stages(N, s, lm))


def stage_level(N, s, lm, j) -> int:
    return int(_L().orc_stage_level(N, s, lm, j))


def butterfly(N, q, phase_id, params, f, s=-1, lm=-1, e=2, stage=-1):
    """FP64 CPU butterfly (Sec. 4 with the Sec. 5 truncation depth s, switch level lm,
    angular refinement e of the T_P boxes).

    Returns u (N, N), or (u, snapshot) when stage >= 0; the snapshot is the state
    after that stage with shape (2^l, 2^l, 2^(L-l), 2^(L-l+e), q, q), indexed
    [a1, a2, b1, b2, t1, t2] for the pair (A=(a1,a2), B=(b1,b2)) at A-level l."""
    f = np.ascontiguousarray(f, dtype=np.complex128).reshape(N, N)
    u = np.zeros((N, N), dtype=np.complex128)
    snap = np.zeros((N * N * q * q) << e, dtype=np.complex128) if stage >= 0 else None
    prm = _prm(params)
    rc = _L().orc_butterfly(N, q, phase_id, _dp(prm), s, lm, e, f.ctypes.data, u.ctypes.data, stage,
                            snap.ctypes.data if snap is not None else None)
    if rc != 0:
        raise ValueError("oracle butterfly rejected N=%d q=%d s=%d lm=%d" % (N, q, s, lm))
    if snap is None:
        return u
    L = N.bit_length() - 1
    lv = stage_level(N, s, lm, stage)
    nA, nB = 1 << lv, 1 << (L - lv)
    return u, snap.reshape(nA, nA, nB, nB << e, q, q)


def butterfly_adjoint(N, q, phase_id, params, g, s=-1, lm=-1, e=2) -> np.ndarray:
    """Exact conjugate transpose of butterfly(): fbar = B^H g."""
    g = np.ascontiguousarray(g, dtype=np.complex128).reshape(N, N)
    out = np.zeros((N, N), dtype=np.complex128)
    prm = _prm(params)
    rc = _L().orc_butterfly_adjoint(N, q, phase_id, _dp(prm), s, lm, e, g.ctypes.data, out.ctypes.data)
    if rc != 0:
        raise ValueError("oracle adjoint rejected N=%d q=%d s=%d lm=%d" % (N, q, s, lm))
    return out


# ---------------------------------------------------------------- three dimensions
# f[k1 + N/2, k2 + N/2, k3 + N/2] and u[i1, i2, i3] (N, N, N); phases 0 linear and 2 sphere
# (lambda x.k + c(x)|k|, c = (a + m sin sin sin)/b; eq. ex3 is [3, 1, 4, 1]).
SPHERE = 2


def spherical3(N, k) -> np.ndarray:
    """Spherical coordinates (p1, p2, p3) of a lattice frequency k (the 3D polar map)."""
    p = np.zeros(3)
    _L().orc3_spherical_map(N, int(k[0]), int(k[1]), int(k[2]), _dp(p))
    return p


def theta3(phase_id, params, N, x, p) -> float:
    """Phi(x, kappa(p)) in three dimensions."""
    xx = np.ascontiguousarray(x, dtype=np.float64)
    pp = np.ascontiguousarray(p, dtype=np.float64)
    return float(_L().orc3_theta_xp(phase_id, _dp(_prm(params)), N, _dp(xx), _dp(pp)))


def direct3(N, phase_id, params, f, xi=None) -> np.ndarray:
    """3D direct sum u(x) = sum_k e^{2 pi i Phi(x,k)} f(k) at flat indices xi = i1 N^2 + i2 N + i3."""
    f = np.ascontiguousarray(f, dtype=np.complex128).reshape(N, N, N)
    xi = np.arange(N ** 3, dtype=np.int64) if xi is None else np.ascontiguousarray(xi, dtype=np.int64)
    u = np.zeros(len(xi), dtype=np.complex128)
    _L().orc3_direct(N, phase_id, _dp(_prm(params)), f.ctypes.data, len(xi),
                     xi.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), u.ctypes.data)
    return u


def butterfly3(N, q, phase_id, params, f, s=-1, lm=-1, e=1) -> np.ndarray:
    """FP64 CPU butterfly in three dimensions (q^3 Chebyshev grids, 8 children per box)."""
    f = np.ascontiguousarray(f, dtype=np.complex128).reshape(N, N, N)
    u = np.zeros((N, N, N), dtype=np.complex128)
    if _L().orc3_butterfly(N, q, phase_id, _dp(_prm(params)), s, lm, e, f.ctypes.data, u.ctypes.data) != 0:
        raise ValueError("oracle 3D butterfly rejected N=%d q=%d s=%d lm=%d e=%d" % (N, q, s, lm, e))
    return u


def direct3_adjoint(N, phase_id, params, g, ki=None) -> np.ndarray:
    """3D adjoint direct sum fbar(k) = sum_x e^{-2 pi i Phi(x,k)} g(x) at flat indices ki."""
    g = np.ascontiguousarray(g, dtype=np.complex128).reshape(N, N, N)
    ki = np.arange(N ** 3, dtype=np.int64) if ki is None else np.ascontiguousarray(ki, dtype=np.int64)
    out = np.zeros(len(ki), dtype=np.complex128)
    _L().orc3_direct_adjoint(N, phase_id, _dp(_prm(params)), g.ctypes.data, len(ki),
                             ki.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), out.ctypes.data)
    return out


def butterfly3_adjoint(N, q, phase_id, params, g, s=-1, lm=-1, e=1) -> np.ndarray:
    """The exact conjugate transpose of butterfly3."""
    g = np.ascontiguousarray(g, dtype=np.complex128).reshape(N, N, N)
    fb = np.zeros((N, N, N), dtype=np.complex128)
    if _L().orc3_butterfly_adjoint(N, q, phase_id, _dp(_prm(params)), s, lm, e, g.ctypes.data, fb.ctypes.data) != 0:
        raise ValueError("oracle 3D adjoint butterfly rejected N=%d q=%d s=%d lm=%d e=%d" % (N, q, s, lm, e))
    return fb


def wave_params(a, m, b, t, sign) -> list:
    """Circle-phase constants [a, m, b, lambda] of Phi_sign(x, k) = x.k + sign c(x)|k| t with
    c(x) = (a + m sin 2 pi x1 sin 2 pi x2) / b (the speed of eq. ex2), sign = +1 or -1."""
    return [sign * a * t, sign * m * t, b, 1.0]


def wave_direct(N, a, m, b, t, f, xi=None) -> np.ndarray:
    """The wave-equation solution operator as a sum of two FIOs (Sec. 1): for u_tt = c^2 Lap u,
    u(x, 0) = u0, u_t(x, 0) = 0 and f the Fourier coefficients of u0 on the lattice,
        u(x, t) = 1/2 sum_k (e^{2 pi i Phi_+(x,k)} + e^{2 pi i Phi_-(x,k)}) f(k),
    Phi_+-(x, k) = x.k +- c|k| t; exact for constant c (m = 0).  With m != 0 the two phases
    use the variable speed c(x), the form of eq. ex2 (the paper notes the exact phases for
    variable c solve a Hamilton-Jacobi equation; this is the two-phase FIO pair, not them)."""
    up = direct(N, CIRCLE, wave_params(a, m, b, t, +1), f, xi)
    um = direct(N, CIRCLE, wave_params(a, m, b, t, -1), f, xi)
    return 0.5 * (up + um)


def wave_butterfly(N, q, a, m, b, t, f, s=-1, lm=-1, e=2) -> np.ndarray:
    """The same two-phase sum with each FIO applied by the butterfly (Sec. 4)."""
    up = butterfly(N, q, CIRCLE, wave_params(a, m, b, t, +1), f, s=s, lm=lm, e=e)
    um = butterfly(N, q, CIRCLE, wave_params(a, m, b, t, -1), f, s=s, lm=lm, e=e)
    return 0.5 * (up + um)


def rel_l2(a, b) -> float:
    """Relative L2 error of eq. err: ||a - b|| / ||b||."""
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))
