"""The sampled direct sum on the GPU (fio_direct) and the choice of q from a target
accuracy (fio_plan_auto, the usage Sec. 5 recommends: the error falls geometrically with q).

* fio_direct equals the oracle's FP64 direct sum of eq. dfio: 1e-12 for FP64 plans (every x
  of N = 64, three RHS), 1e-6 for FP32 plans (their phases in double-float, their sin/cos
  in FP32, their sums in FP64) on 512 seeded x of N = 256;
* fio_plan_auto returns the smallest q whose estimated error meets the target: its estimate
  is below the target, the true error on other seeded points is within 3x of the estimate,
  and the plan of the next smaller q misses the target on the same points;
* an FP32 target below FP32 resolution returns the q = 11 plan with its (larger) estimate.
"""
import numpy as np
import pytest
import torch

from paper_0809_0719_gb300.inputs import gaussian_batch, gaussian_sources, sample_indices

pytestmark = pytest.mark.gpu

ELL16 = (2.0, 1.0, 16.0, 1.0)
CIRC20 = (3.0, 1.0, 20.0, 1.0)


@pytest.fixture(scope="module")
def fio():
    from paper_0809_0719_gb300 import fio as F

    assert torch.cuda.is_available()
    return F


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


def test_direct_fp64_matches_oracle_everywhere(fio, oracle):
    N = 64
    plan = fio.Plan(N, 5, "ellipse", ELL16, "f64", nrhs_max=3)
    try:
        F = gaussian_batch(N, [7, 8, 9])
        xi = torch.arange(N * N, dtype=torch.int64, device="cuda")
        got = plan.direct(torch.from_numpy(F).cuda(), xi).cpu().numpy()
        for r in range(3):
            assert rel(got[r], oracle.direct(N, 1, list(ELL16), F[r])) < 1e-12
    finally:
        plan.close()


@pytest.mark.parametrize("phase,prm,pid", [("ellipse", ELL16, 1), ("circle", CIRC20, 2), ("linear", (), 0)])
def test_direct_fp32_matches_oracle_on_samples(fio, oracle, phase, prm, pid):
    N = 256
    plan = fio.Plan(N, 7, phase, prm, "f32", nrhs_max=1)
    try:
        f = gaussian_sources(N, 11)
        xi = sample_indices(N, 512, 1000)
        got = plan.direct(torch.from_numpy(f).to(torch.complex64).cuda()[None],
                          torch.from_numpy(xi).cuda()).cpu().numpy()[0]
        ref = oracle.direct(N, pid, list(prm), f.astype(np.complex64).astype(np.complex128), xi)
        assert rel(got, ref) < 1e-6
    finally:
        plan.close()


def test_plan_auto_picks_the_smallest_sufficient_q(fio, oracle):
    N, target = 128, 1e-3
    plan, q, est = fio.plan_auto(N, target, "ellipse", ELL16, "f32", nsample=256, seed=3)
    try:
        assert q in (3, 5, 7, 9, 11) and est <= target and plan.info.q == q
        f = gaussian_sources(N, 21)
        xi = sample_indices(N, 256, 1000)
        ft = torch.from_numpy(f).to(torch.complex64).cuda()[None]
        u = plan.apply(ft)[0].cpu().numpy().ravel()[xi]
        ref = oracle.direct(N, 1, list(ELL16), f.astype(np.complex64).astype(np.complex128), xi)
        true = rel(u, ref)
        assert est / 3 <= true <= 3 * est
        if q > 3:  # the next smaller q misses the target
            smaller = fio.Plan(N, q - 2, "ellipse", ELL16, "f32")
            try:
                us = smaller.apply(ft)[0].cpu().numpy().ravel()[xi]
                assert rel(us, ref) > target
            finally:
                smaller.close()
    finally:
        plan.close()


def test_plan_auto_unreachable_target_returns_q11(fio):
    plan, q, est = fio.plan_auto(64, 1e-9, "ellipse", ELL16, "f32", nsample=128, seed=5)
    try:
        assert q == 11 and est > 1e-9
    finally:
        plan.close()
