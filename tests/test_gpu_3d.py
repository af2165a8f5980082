"""GPU parity of the three-dimensional butterfly (Sec. 5, eq. ex3, Table 3; include/fio3.h)
against the FP64 CPU oracle (oracle/fio_oracle3.c) on the same seeded inputs.

Tolerance: FP64 throughout, so relative L2 <= 1e-12 against the oracle butterfly with equal
(q, s, e), forward and adjoint (both sides take the source-to-box decisions with the same FP64
expressions); the dot test to 1e-12; and the accuracy against the direct sum within the
oracle butterfly's own error (the GPU result IS that butterfly, to rounding)."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

EX3 = [3.0, 1.0, 4.0, 1.0]  # eq. ex3: c(x) = (3 + sin sin sin)/4


@pytest.fixture(scope="module")
def fio():
    from paper_0809_0719_gb300 import fio as F

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    F.lib()
    return F


def white3(N, seed, nrhs=1):
    rng = np.random.default_rng(seed)
    return np.stack([rng.standard_normal((N, N, N)) + 1j * rng.standard_normal((N, N, N)) for _ in range(nrhs)])


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


# N, q, phase, s, e, nrhs: all three compiled q, s = 0 (the full recursion), 1 and 2,
# e = 0 and 1, both phases, one and several RHS
CASES = [(16, 3, "sphere", 0, 1, 1), (16, 5, "sphere", 1, 1, 2), (8, 7, "sphere", 0, 1, 1),
         (16, 5, "linear", 2, 0, 1), (8, 3, "sphere", 1, 0, 3)]


@pytest.mark.parametrize("N,q,phase,s,e,nrhs", CASES)
def test_3d_forward_and_adjoint_match_oracle(fio, oracle, N, q, phase, s, e, nrhs):
    pid = 2 if phase == "sphere" else 0
    plan = fio.Plan3(N, q, phase, EX3, nrhs_max=nrhs, s=s, e=e)
    try:
        assert (plan.info.s, plan.info.e) == (s, e)
        F = white3(N, 10 + N + q, nrhs)
        G = white3(N, 20 + N + q, nrhs)
        u = plan.apply(torch.from_numpy(F).cuda()).cpu().numpy()
        fb = plan.adjoint(torch.from_numpy(G).cuda()).cpu().numpy()
        for r in range(nrhs):
            ref = oracle.butterfly3(N, q, pid, EX3, F[r], s=s, e=e)
            assert rel(u[r], ref) < 1e-12, (r, rel(u[r], ref))
            refa = oracle.butterfly3_adjoint(N, q, pid, EX3, G[r], s=s, e=e)
            assert rel(fb[r], refa) < 1e-12, (r, rel(fb[r], refa))
    finally:
        plan.close()


def test_3d_dot_test_and_accuracy_at_n32(fio, oracle):
    # N = 32, q = 7, e = 1, eq. ex3, s = 2 (two levels of each recursion): the dot test of the GPU
    # butterfly and its adjoint to 1e-12, and its error against the oracle's direct sum on 128
    # seeded x in the range Table 3 reports for q = 7 (3.3e-3 .. 4.1e-3 at N = 64 .. 256;
    # nearly flat in N)
    N, q = 32, 7
    plan = fio.Plan3(N, q, "sphere", EX3, nrhs_max=1, s=2, e=1)
    try:
        F, G = white3(N, 31), white3(N, 32)
        f, g = torch.from_numpy(F).cuda(), torch.from_numpy(G).cuda()
        u, fb = plan.apply(f), plan.adjoint(g)
        a = torch.vdot(g.flatten(), u.flatten())
        b = torch.vdot(fb.flatten(), f.flatten())
        assert abs(a - b).item() < 1e-12 * abs(a).item()
        xi = np.sort(np.random.default_rng(1000).choice(N ** 3, 128, replace=False)).astype(np.int64)
        ref = oracle.direct3(N, 2, EX3, F[0], xi)
        err = rel(u.cpu().numpy().reshape(-1)[xi], ref)
        assert 1e-4 < err < 8e-3, err
    finally:
        plan.close()


def test_3d_rejects_bad_arguments(fio):
    for kw in (dict(N=12, q=5), dict(N=16, q=9), dict(N=16, q=5, e=4), dict(N=512, q=3)):
        with pytest.raises(fio.FIOError):
            fio.Plan3(kw.pop("N"), kw.pop("q"), "sphere", EX3, **kw)
    plan = fio.Plan3(8, 3, "sphere", EX3, nrhs_max=1)
    try:
        with pytest.raises(fio.FIOError):
            plan.apply(torch.zeros(2, 8, 8, 8, dtype=torch.complex128, device="cuda"))  # nrhs > nrhs_max
    finally:
        plan.close()
