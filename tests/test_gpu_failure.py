"""Failure detection on the GPU without a fault: a bounded device-side wait is made to run
out, the library reports it, and the next apply is correct again.

The tensor-memory switch kernel hands chunks between its producer warps and its MMA warp
through mbarriers, each wait bounded in wall time.  fio_plan_set_wait_limit shrinks that
bound to 1 ns, so the first hand-off wait that is not already complete gives up: the kernel
records status 1, stops issuing, still waits with the normal 2 s bound for the tensor-core
operations it issued, frees its tensor memory and returns.  fio_check must then report
FIO_ETIMEOUT (and clear the word); with the normal bound restored the apply matches the
oracle butterfly.
"""
import numpy as np
import pytest
import torch

from paper_0809_0719_gb300.inputs import gaussian_batch

pytestmark = pytest.mark.gpu

ELL16 = (2.0, 1.0, 16.0, 1.0)


@pytest.fixture(scope="module")
def fio():
    from paper_0809_0719_gb300 import fio as F

    assert torch.cuda.is_available()
    F.lib()
    return F


def rel(a, b):
    return float(np.linalg.norm(np.ravel(a) - np.ravel(b)) / np.linalg.norm(np.ravel(b)))


@pytest.mark.parametrize("adjoint", [False, True])
def test_expired_switch_wait_is_reported_and_the_next_apply_is_correct(fio, oracle, adjoint):
    N, q, R = 64, 5, 4
    plan = fio.Plan(N, q, "ellipse", ELL16, "f32", nrhs_max=R)
    try:
        plan.set_switch(3)
        F = gaussian_batch(N, range(700, 700 + R)).astype(np.complex64)
        f = torch.from_numpy(F).cuda()
        run = plan.adjoint if adjoint else plan.apply
        run(f)
        plan.check()  # a clean apply first
        plan.set_wait_limit(1)
        run(f)
        with pytest.raises(fio.FIOError) as err:
            plan.check()
        assert err.value.code == fio.FIO_ETIMEOUT
        plan.check()  # the word was cleared
        plan.set_wait_limit(0)
        out = run(f).cpu().numpy()
        plan.check()
        for r in range(R):
            Fr = F[r].astype(np.complex128)
            if adjoint:
                ref = oracle.butterfly_adjoint(N, q, 1, list(ELL16), Fr, s=plan.info.s, e=plan.info.e)
            else:
                ref = oracle.butterfly(N, q, 1, list(ELL16), Fr, s=plan.info.s, e=plan.info.e)
            assert rel(out[r], ref) < 1e-5, (r, rel(out[r], ref))
    finally:
        plan.close()
