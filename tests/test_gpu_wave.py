"""GPU parity of the wave propagator as a sum of two FIOs (Sec. 1): fio_apply_wave with the
two circle-phase plans x.k +- c(x)|k|t against the oracle's two-phase butterfly with identical
(q, s, e), forward and adjoint, plus the dot test and argument checks.  Tolerances as for a
single FIO: 1e-12 (FP64 form), 1e-5 (FP32 form)."""
import numpy as np
import pytest
import torch

from paper_0809_0719_gb300.inputs import gaussian_batch

pytestmark = pytest.mark.gpu

A, M, B = 3.0, 1.0, 20.0  # c(x) = (3 + sin 2 pi x1 sin 2 pi x2) / 20, the speed of eq. ex2


@pytest.fixture(scope="module")
def fio():
    from paper_0809_0719_gb300 import fio as F

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    F.lib()
    return F


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5)])
@pytest.mark.parametrize("N,q,t", [(64, 7, 1.0), (128, 5, 0.5)])
def test_wave_matches_oracle_two_phase_butterfly(fio, oracle, prec, tol, N, q, t):
    plus, minus = fio.wave_plans(N, q, A, M, B, t, prec, nrhs_max=3, e=2)
    try:
        F = gaussian_batch(N, range(500, 503))
        f = torch.from_numpy(F).to(plus.dtype).cuda()
        u = fio.apply_wave(plus, minus, f).cpu().numpy()
        g = fio.apply_wave(plus, minus, f, adjoint=True).cpu().numpy()
        plus.check()
        minus.check()
        s = plus.info.s
        pp, pm = oracle.wave_params(A, M, B, t, +1), oracle.wave_params(A, M, B, t, -1)
        for r in range(3):
            fr = F[r].astype(np.complex64).astype(np.complex128) if prec == "f32" else F[r]
            ref = oracle.wave_butterfly(N, q, A, M, B, t, fr, s=s, e=2)
            assert rel(u[r], ref) < tol, (r, rel(u[r], ref))
            refa = 0.5 * (oracle.butterfly_adjoint(N, q, oracle.CIRCLE, pp, fr, s=s, e=2)
                          + oracle.butterfly_adjoint(N, q, oracle.CIRCLE, pm, fr, s=s, e=2))
            assert rel(g[r], refa) < tol, (r, rel(g[r], refa))
    finally:
        plus.close()
        minus.close()


def test_wave_dot_test_and_weights(fio):
    N = 64
    plus, minus = fio.wave_plans(N, 5, A, M, B, 1.0, "f64", nrhs_max=1, e=2)
    try:
        f = torch.from_numpy(gaussian_batch(N, [7])).cuda()
        g = torch.from_numpy(gaussian_batch(N, [8])).cuda()
        w = fio.apply_wave(plus, minus, f, 0.3, -1.7)
        wh = fio.apply_wave(plus, minus, g, 0.3, -1.7, adjoint=True)
        a = torch.vdot(g.flatten(), w.flatten())
        b = torch.vdot(wh.flatten(), f.flatten())
        assert abs(a - b).item() < 1e-12 * abs(a).item()
        # the weighted sum is the sum of the two single-plan applies
        ref = 0.3 * plus.apply(f) - 1.7 * minus.apply(f)
        assert rel(w.cpu().numpy(), ref.cpu().numpy()) < 1e-14
    finally:
        plus.close()
        minus.close()


def test_wave_rejects_mismatched_plans(fio):
    p32 = fio.Plan(32, 5, "circle", (1.0, 0.0, 20.0, 1.0), "f64")
    p64 = fio.Plan(64, 5, "circle", (-1.0, 0.0, 20.0, 1.0), "f64")
    try:
        f = torch.zeros(1, 32, 32, dtype=torch.complex128, device="cuda")
        with pytest.raises(fio.FIOError):
            fio.apply_wave(p32, p64, f)
        with pytest.raises(fio.FIOError):  # in and out may not alias
            fio.apply_wave(p32, p32, f, out=f)
    finally:
        p32.close()
        p64.close()


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_wave_series_from_one_plan(fio, oracle, prec, tol):
    # u(t_k) for several times from ONE circle-phase plan (its tables and state serve all 2 ntimes
    # butterflies): against the oracle's two-phase butterfly at each time, and bit for bit
    # against fio_apply_wave on a separately built pair of plans per time
    N, q, R = 64, 7, 2
    times = [0.3, 1.0, 2.5]
    plan = fio.Plan(N, q, "circle", (A, M, B, 1.0), prec, nrhs_max=R, e=2)
    try:
        F = gaussian_batch(N, range(600, 600 + R))
        f = torch.from_numpy(F).to(plan.dtype).cuda()
        U = fio.apply_wave_series(plan, times, f)
        plan.check()
        Uh = U.cpu().numpy()
        for k, t in enumerate(times):
            plus, minus = fio.wave_plans(N, q, A, M, B, t, prec, nrhs_max=R, e=2)
            try:
                pair = fio.apply_wave(plus, minus, f)
                assert torch.equal(pair, U[k]), (k, t)
            finally:
                plus.close()
                minus.close()
            for r in range(R):
                fr = F[r].astype(np.complex64).astype(np.complex128) if prec == "f32" else F[r]
                ref = oracle.wave_butterfly(N, q, A, M, B, t, fr, s=plan.info.s, e=2)
                assert rel(Uh[k, r], ref) < tol, (k, r, rel(Uh[k, r], ref))
        with pytest.raises(fio.FIOError):  # a linear-phase plan has no speed to propagate with
            lin = fio.Plan(N, q, "linear", (), prec)
            try:
                fio.apply_wave_series(lin, times, f[:1])
            finally:
                lin.close()
    finally:
        plan.close()
