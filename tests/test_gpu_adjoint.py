"""Differentiation through the adjoint butterfly (N=512, q=7, ellipse phase of eq. ex1 scaled by 1/16).

loss(f) = sum_x |u(x) - u*(x)|^2 with u = B f and u* = B f* for a second seeded input.
PyTorch's gradient of a real loss with respect to a complex input is
dL/dRe f + i dL/dIm f = 2 B^H (B f - u*); the backward of FIOFunction applies the
hand-written adjoint butterfly B^H.
  * dot test <B f, g> = <f, B^H g>: 1e-12 (FP64 form), 1e-6 (FP32 form);
  * the complex64 gradient through autograd matches the FP64 gradient to FP32 accuracy;
  * central finite differences on 64 seeded frequencies (h = 1e-3, FP64 form) match the
    gradient; the loss is quadratic, so the differences carry no truncation error, and
    the two losses are subtracted element by element, so they agree to ~1e-10;
  * the adjoint butterfly approximates the direct adjoint sum fbar(k) = sum_x e^{-2 pi i Phi(x,k)} g(x)
    at 256 seeded frequencies to the method's accuracy at q = 7 (~1e-4).
"""
import numpy as np
import pytest
import torch

from paper_0809_0719_gb300.inputs import gaussian_sources, sample_indices

pytestmark = pytest.mark.gpu

N, Q = 512, 7
ELL16 = (2.0, 1.0, 16.0, 1.0)


@pytest.fixture(scope="module")
def fio():
    from paper_0809_0719_gb300 import fio as F

    assert torch.cuda.is_available()
    return F


@pytest.fixture(scope="module")
def plans(fio):
    p64 = fio.Plan(N, Q, "ellipse", ELL16, "f64", nrhs_max=32)
    p32 = fio.Plan(N, Q, "ellipse", ELL16, "f32", nrhs_max=2)
    yield p64, p32
    p64.close()
    p32.close()


def _inputs(dtype):
    f = torch.from_numpy(gaussian_sources(N, 2)).to(dtype).cuda()[None]
    fs = torch.from_numpy(gaussian_sources(N, 3)).to(dtype).cuda()[None]
    return f, fs


def test_dot_test_both_forms(fio, plans):
    for plan, tol in ((plans[0], 1e-12), (plans[1], 1e-6)):
        dt = plan.dtype
        f = torch.from_numpy(gaussian_sources(N, 4)).to(dt).cuda()[None]
        g = torch.from_numpy(gaussian_sources(N, 5)).to(dt).cuda()[None]
        a = torch.vdot(g.to(torch.complex128).flatten(), plan.apply(f).to(torch.complex128).flatten())
        b = torch.vdot(plan.adjoint(g).to(torch.complex128).flatten(), f.to(torch.complex128).flatten())
        assert abs(a - b).item() < tol * abs(a).item(), (dt, abs(a - b).item() / abs(a).item())


def _grad(fio, plan, dtype):
    f, fs = _inputs(dtype)
    with torch.no_grad():
        ustar = plan.apply(fs)
    f = f.clone().requires_grad_(True)
    loss = (fio.fio_apply(f, plan) - ustar).abs().pow(2).sum()
    loss.backward()
    return f.grad.detach()


def test_complex64_gradient_matches_fp64_gradient(fio, plans):
    g64 = _grad(fio, plans[0], torch.complex128)
    g32 = _grad(fio, plans[1], torch.complex64).to(torch.complex128)
    rel = ((g32 - g64).norm() / g64.norm()).item()
    assert rel < 1e-5, rel


def _loss_diff(up, um, ustar):
    """sum |up - u*|^2 - sum |um - u*|^2, formed element by element so that the large,
    equal parts of the two losses cancel before the sum."""
    return ((up - ustar).abs().pow(2) - (um - ustar).abs().pow(2)).sum().item()


def test_central_finite_differences(fio, plans):
    plan = plans[0]
    grad = _grad(fio, plan, torch.complex128)[0].reshape(-1)
    f, fs = _inputs(torch.complex128)
    with torch.no_grad():
        ustar = plan.apply(fs)[0]
        u0 = plan.apply(f)[0]
    ks = sample_indices(N, 64, 1002)
    h = 1e-3
    g = grad[torch.from_numpy(ks).cuda()].cpu().numpy()

    # (a) literal central differences: the butterfly re-applied to f +- h e_k and
    # f +- i h e_k for the first 8 frequencies (32 perturbed inputs in one batch)
    lit = ks[:8]
    batch = f.repeat(32, 1, 1)
    for i, k in enumerate(lit):
        for j, d in enumerate((h, -h, 1j * h, -1j * h)):
            batch[4 * i + j].view(-1)[int(k)] += d
    with torch.no_grad():
        ub = plan.apply(batch)
    fd = np.array([(_loss_diff(ub[4 * i], ub[4 * i + 1], ustar)
                    + 1j * _loss_diff(ub[4 * i + 2], ub[4 * i + 3], ustar)) / (2 * h) for i in range(8)])
    rel = np.linalg.norm(fd - g[:8]) / np.linalg.norm(g[:8])
    assert rel < 1e-8, rel

    # (b) all 64 frequencies: the butterfly is linear in f, so B(f +- h e_k) = u0 +- h B e_k;
    # the unit responses B e_k come from two 32-column applies
    fd = []
    for i0 in (0, 32):
        e = torch.zeros(32, N, N, dtype=torch.complex128, device="cuda")
        for j, k in enumerate(ks[i0:i0 + 32]):
            e[j].view(-1)[int(k)] = 1.0
        with torch.no_grad():
            v = plan.apply(e)
        for j in range(32):
            d_re = _loss_diff(u0 + h * v[j], u0 - h * v[j], ustar)
            d_im = _loss_diff(u0 + 1j * h * v[j], u0 - 1j * h * v[j], ustar)
            fd.append((d_re + 1j * d_im) / (2 * h))
    fd = np.array(fd)
    rel = np.linalg.norm(fd - g) / np.linalg.norm(g)
    assert rel < 1e-8, rel


def test_adjoint_matches_direct_adjoint_sum(fio, plans, oracle):
    plan = plans[0]
    g = gaussian_sources(N, 6)
    fb = plan.adjoint(torch.from_numpy(g).cuda()[None])[0].cpu().numpy().ravel()
    ki = sample_indices(N, 256, 1001)
    ref = oracle.direct_adjoint(N, 1, list(ELL16), g, ki)
    rel = np.linalg.norm(fb[ki] - ref) / np.linalg.norm(ref)
    assert rel < 1e-3, rel
