"""Pins for the three-dimensional FP64 CPU oracle (the 3D form of the method, Sec. 5 and
Table 3).  As for the 2D oracle, each test checks it against something other than itself:
the 3D DFT (numpy), the inverse of the spherical map, exactness when the phase does not
depend on x (R^{AB} = 0), the decay of the error with q, its flatness in N, and the
accuracy the paper prints in Table 3."""
import os

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EX3 = [3.0, 1.0, 4.0, 1.0]  # eq. ex3: c(x) = (3 + sin sin sin)/4


def sources3(N, seed):
    rng = np.random.default_rng(seed)
    return rng.standard_normal((N, N, N)) + 1j * rng.standard_normal((N, N, N))


def dft3_of(f):
    """u[i] = sum_k e^{2 pi i (i/N).k} f(k), k = m - N/2, with numpy's inverse FFT."""
    N = f.shape[0]
    i = np.arange(N)
    sign = (-1.0) ** (i[:, None, None] + i[None, :, None] + i[None, None, :])
    return sign * N ** 3 * np.fft.ifftn(f)


def test_direct3_linear_phase_is_a_3d_dft(oracle):
    N = 8
    f = sources3(N, 31)
    u = oracle.direct3(N, 0, [], f).reshape(N, N, N)
    assert oracle.rel_l2(u, dft3_of(f)) < 1e-12


def test_direct3_sphere_phase_with_constant_speed_is_a_dft(oracle):
    N = 8
    f = sources3(N, 32)
    k = np.arange(N) - N // 2
    kk = np.sqrt(k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2)
    u = oracle.direct3(N, oracle.SPHERE, [3.0, 0.0, 4.0, 1.0], f).reshape(N, N, N)
    assert oracle.rel_l2(u, dft3_of(f * np.exp(2j * np.pi * 0.75 * kk))) < 1e-12


def test_spherical_map_inverts_to_the_lattice(oracle):
    # kappa(p(k)) = k: read kappa through the linear phase at the unit vectors, and the
    # coordinates stay in [0, 1] with p1 = 1 at the corner (-N/2, -N/2, -N/2)
    N = 8
    r = np.arange(N) - N // 2
    for k in [(a, b, c) for a in r for b in r for c in r]:
        p = oracle.spherical3(N, k)
        assert 0.0 <= p[0] <= 1.0 + 1e-15 and 0.0 <= p[1] <= 1.0 and 0.0 <= p[2] < 1.0
        back = [oracle.theta3(0, [0, 0, 0, 0], N, e, p) for e in np.eye(3)]
        assert np.allclose(back, k, rtol=0, atol=1e-12), (k, back)
    assert oracle.spherical3(N, (-N // 2,) * 3)[0] == pytest.approx(1.0, abs=1e-15)


@pytest.mark.parametrize("N,s,e", [(8, 0, 0), (8, 1, 1), (16, 0, 1), (16, 2, 0)])
def test_butterfly3_exact_when_the_phase_does_not_depend_on_x(oracle, N, s, e):
    # lambda = m = 0: Phi = c|k|, so R^{AB} vanishes and the interpolations are exact
    f = sources3(N, 33)
    prm = [3.0, 0.0, 4.0, 0.0]
    ub = oracle.butterfly3(N, 3, oracle.SPHERE, prm, f, s=s, e=e)
    ud = oracle.direct3(N, oracle.SPHERE, prm, f).reshape(N, N, N)
    assert oracle.rel_l2(ub, ud) < 1e-12


def test_butterfly3_error_falls_with_q_and_is_flat_in_N(oracle):
    err = {}
    for N, qs in ((8, (3, 5, 7)), (16, (5,))):
        f = sources3(N, 34)
        ud = oracle.direct3(N, oracle.SPHERE, EX3, f).reshape(N, N, N)
        for q in qs:
            err[N, q] = oracle.rel_l2(oracle.butterfly3(N, q, oracle.SPHERE, EX3, f, s=0, e=1), ud)
    assert err[8, 5] < err[8, 3] / 5 and err[8, 7] < err[8, 5] / 5, err
    assert 0.67 < err[16, 5] / err[8, 5] < 1.5, err


def test_butterfly3_accuracy_matches_table3(oracle):
    # Table 3 reports eps_a ~ 3.3e-3 .. 4.1e-3 at q = 7 for N = 64 .. 256, nearly flat in N;
    # the oracle at N = 8 (the size a plain CPU statement finishes in seconds) is within 2x
    rows = np.loadtxt(os.path.join(ROOT, "tests", "golden", "table3_ex3_eps.txt"))
    N, q = 8, 7
    f = sources3(N, 35)
    err = oracle.rel_l2(oracle.butterfly3(N, q, oracle.SPHERE, EX3, f, s=0, e=1),
                        oracle.direct3(N, oracle.SPHERE, EX3, f).reshape(N, N, N))
    for _, qq, eps in rows:
        assert qq == q
        assert eps / 2 < err < 2 * eps, (err, eps)


def test_direct3_adjoint_linear_phase_is_a_forward_dft(oracle):
    # fbar(k) = sum_x e^{-2 pi i x.k} g(x) with x = i/N, k = m - N/2: e^{pi i (i1+i2+i3)}
    # times numpy's forward FFT kernel, i.e. the FFT of (-1)^(i1+i2+i3) g
    N = 8
    g = sources3(N, 36)
    fb = oracle.direct3_adjoint(N, 0, [], g).reshape(N, N, N)
    i = np.arange(N)
    sign = (-1.0) ** (i[:, None, None] + i[None, :, None] + i[None, None, :])
    assert oracle.rel_l2(fb, np.fft.fftn(sign * g)) < 1e-12


@pytest.mark.parametrize("N,q,s,e", [(8, 3, 0, 1), (8, 5, 1, 0), (16, 3, 0, 1)])
def test_butterfly3_dot_test(oracle, N, q, s, e):
    # <g, B f> = <B^H g, f> to rounding: the adjoint is the exact conjugate transpose
    f, g = sources3(N, 37), sources3(N, 38)
    a = np.vdot(g, oracle.butterfly3(N, q, oracle.SPHERE, EX3, f, s=s, e=e))
    b = np.vdot(oracle.butterfly3_adjoint(N, q, oracle.SPHERE, EX3, g, s=s, e=e), f)
    assert abs(a - b) < 1e-12 * abs(a)


def test_butterfly3_adjoint_approximates_the_adjoint_sum(oracle):
    # the adjoint butterfly approximates the adjoint direct sum as the forward does the forward
    N, q = 8, 7
    g = sources3(N, 39)
    fb = oracle.butterfly3_adjoint(N, q, oracle.SPHERE, EX3, g, s=0, e=1)
    ref = oracle.direct3_adjoint(N, oracle.SPHERE, EX3, g).reshape(N, N, N)
    assert oracle.rel_l2(fb, ref) < 1e-2


def test_butterfly3_rejects_bad_arguments(oracle):
    f = np.zeros((8, 8, 8), dtype=np.complex128)
    with pytest.raises(ValueError):
        oracle.butterfly3(8, 1, oracle.SPHERE, EX3, f)
    with pytest.raises(ValueError):
        oracle.butterfly3(8, 5, 1, EX3, f)  # no ellipse phase in 3D
