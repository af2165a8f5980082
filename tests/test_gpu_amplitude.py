"""Variable amplitudes (eq. allfio) through fio_apply_amplitude: a(x,k) = sum_t g_t(x) h_t(k).

* parity: equals sum_t g_t (oracle butterfly of h_t f) -- 1e-12 (FP64 form), 1e-5 (FP32);
* accuracy: against the direct sum sum_k a(x,k) e^{2 pi i Phi} f(k), formed from the oracle's
  direct sums of h_t f weighted by g_t, on seeded samples (q = 9);
* the adjoint is the exact conjugate transpose (dot test) and equals
  sum_t conj h_t (oracle adjoint butterfly of conj g_t gin);
* one term with g = h = 1 gives fio_apply itself.
"""
import numpy as np
import pytest
import torch

from paper_0809_0719_gb300.inputs import gaussian_batch, gaussian_sources, sample_indices

pytestmark = pytest.mark.gpu

ELL16 = (2.0, 1.0, 16.0, 1.0)


@pytest.fixture(scope="module")
def fio():
    from paper_0809_0719_gb300 import fio as F

    assert torch.cuda.is_available()
    return F


def amplitude_terms(N, nt):
    """Smooth seeded separated amplitude: g_t(x) = 1 + c_t cos 2 pi (m_t x1 + x2), h_t(k) = exp(-w_t |k|^2 / N^2) e^{i d_t k1 / N}."""
    rng = np.random.default_rng(12)
    i = np.arange(N) / N
    x1, x2 = np.meshgrid(i, i, indexing="ij")
    k = np.arange(N) - N // 2
    k1, k2 = np.meshgrid(k, k, indexing="ij")
    g = np.stack([1 + rng.uniform(0.1, 0.5) * np.cos(2 * np.pi * (rng.integers(1, 4) * x1 + x2)) + 0j for _ in range(nt)])
    h = np.stack([np.exp(-rng.uniform(0.5, 3) * (k1 ** 2 + k2 ** 2) / N ** 2 + 1j * rng.uniform(-2, 2) * k1 / N)
                  for _ in range(nt)])
    return g, h


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-5)])
def test_amplitude_matches_oracle_butterfly(fio, oracle, prec, tol):
    N, q, nt, nrhs = 64, 7, 3, 2
    plan = fio.Plan(N, q, "ellipse", ELL16, prec, nrhs_max=nt * nrhs)
    try:
        g, h = amplitude_terms(N, nt)
        F = gaussian_batch(N, [31, 32])
        dt = plan.dtype
        U = plan.apply_amplitude(torch.from_numpy(F).to(dt).cuda(), torch.from_numpy(g).to(dt).cuda(),
                                 torch.from_numpy(h).to(dt).cuda()).cpu().numpy()
        cast = (lambda a: a) if prec == "f64" else (lambda a: a.astype(np.complex64).astype(np.complex128))
        for r in range(nrhs):
            ref = sum(cast(g)[t] * oracle.butterfly(N, q, 1, list(ELL16), cast(h)[t] * cast(F)[r]) for t in range(nt))
            assert rel(U[r], ref) < tol
        G = plan.apply_amplitude(torch.from_numpy(F).to(dt).cuda(), torch.from_numpy(g).to(dt).cuda(),
                                 torch.from_numpy(h).to(dt).cuda(), adjoint=True).cpu().numpy()
        for r in range(nrhs):
            ref = sum(np.conj(cast(h)[t]) * oracle.butterfly_adjoint(N, q, 1, list(ELL16), np.conj(cast(g)[t]) * cast(F)[r])
                      for t in range(nt))
            assert rel(G[r], ref) < tol
    finally:
        plan.close()


def test_amplitude_accuracy_against_direct_sum(fio, oracle):
    N, q, nt = 128, 9, 3
    plan = fio.Plan(N, q, "ellipse", ELL16, "f64", nrhs_max=nt)
    try:
        g, h = amplitude_terms(N, nt)
        f = gaussian_sources(N, 41)
        u = plan.apply_amplitude(torch.from_numpy(f).cuda()[None], torch.from_numpy(g).cuda(),
                                 torch.from_numpy(h).cuda())[0].cpu().numpy().ravel()
        xi = sample_indices(N, 256, 1000)
        ref = sum(g[t].ravel()[xi] * oracle.direct(N, 1, list(ELL16), h[t] * f, xi) for t in range(nt))
        assert rel(u[xi], ref) < 1e-4
    finally:
        plan.close()


@pytest.mark.parametrize("prec,tol", [("f64", 1e-12), ("f32", 1e-6)])
def test_amplitude_dot_test_and_reduction(fio, prec, tol):
    N, nt = 128, 4
    plan = fio.Plan(N, 7, "ellipse", ELL16, prec, nrhs_max=nt)
    try:
        dt = plan.dtype
        g, h = amplitude_terms(N, nt)
        gt, ht = torch.from_numpy(g).to(dt).cuda(), torch.from_numpy(h).to(dt).cuda()
        f = torch.from_numpy(gaussian_sources(N, 51)).to(dt).cuda()[None]
        w = torch.from_numpy(gaussian_sources(N, 52)).to(dt).cuda()[None]
        Bf = plan.apply_amplitude(f, gt, ht).to(torch.complex128).flatten()
        Bw = plan.apply_amplitude(w, gt, ht, adjoint=True).to(torch.complex128).flatten()
        w64, f64 = w.to(torch.complex128).flatten(), f.to(torch.complex128).flatten()
        a, b = torch.vdot(w64, Bf), torch.vdot(Bw, f64)
        assert abs(a - b).item() < tol * (w64.norm() * Bf.norm()).item()
        one = torch.ones(1, N, N, dtype=dt, device="cuda")
        assert torch.equal(plan.apply_amplitude(f, one, one), plan.apply(f))
    finally:
        plan.close()
