"""GPU parity: the CUDA butterfly against the FP64 CPU oracle on the same seeded inputs.

Tolerances
  FP64 form : relative L2 <= 1e-12 against the oracle butterfly with equal (q, s, e),
              per stage and end to end (both sides take every integer decision --
              the source-to-box assignment -- with the same FP64 expressions).
  FP32 form : relative L2 <= 1e-5 against the oracle butterfly.  FP32 carries a unit
              roundoff of 6e-8; each of the <= 2L steps multiplies by a Lagrange
              operator of norm ~2-3 and adds a few roundings, and the FP32 sin/cos of
              the FP64-reduced phase adds ~1e-7 per factor, so ~1e-6 is expected and
              1e-5 (the floor of the stated FP32 accuracy bar) leaves a 10x margin.
"""
import numpy as np
import pytest
import torch

from paper_0809_0719_gb300.inputs import gaussian_batch, gaussian_sources, sample_indices

pytestmark = pytest.mark.gpu

ELL16 = (2.0, 1.0, 16.0, 1.0)
CIRC20 = (3.0, 1.0, 20.0, 1.0)
SEP = (0.3, 0.2, 0.25, 0.1)
PH = {"ellipse": (1, ELL16), "circle": (2, CIRC20), "linear": (0, ()), "separable": (3, SEP)}

F64_TOL = 1e-12
F32_TOL = 1e-5

_oracle_cache = {}


@pytest.fixture(scope="module")
def fio():
    from paper_0809_0719_gb300 import fio as F

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    F.lib()
    return F


def oracle_bf(oracle, N, q, phase, f, s, e):
    key = (N, q, phase, s, e, f.tobytes())
    if key not in _oracle_cache:
        pid, prm = PH[phase]
        _oracle_cache[key] = oracle.butterfly(N, q, pid, list(prm), f, s=s, e=e)
    return _oracle_cache[key]


def set_switch(fio, plan, sw, q):
    """Force the FP32 switch kernel; the warp-specialised one needs two q^4 kernel
    buffers in shared memory and does not fit q = 11."""
    try:
        plan.set_switch(sw)
    except fio.FIOError:
        if sw == 2 and q >= 11:
            pytest.skip("the warp-specialised switch does not fit q=%d" % q)
        raise


def rel(a, b):
    a = np.asarray(a).ravel()
    b = np.asarray(b).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


CASES = [
    # N, q, phase, s, e
    (4, 3, "ellipse", 0, 0),
    (8, 11, "ellipse", 0, 4),
    (16, 3, "circle", 0, 0),
    (32, 7, "ellipse", 3, 1),
    (64, 5, "ellipse", 0, 2),
    (64, 5, "ellipse", 3, 2),
    (64, 9, "linear", 3, 2),
    (64, 5, "separable", 3, 2),
    (128, 5, "circle", 3, 2),
    (128, 7, "ellipse", 3, 0),
]


@pytest.mark.parametrize("N,q,phase,s,e", CASES)
@pytest.mark.parametrize("prec,nrhs,sw", [("f64", 1, None), ("f64", 5, None), ("f32", 3, 0), ("f32", 9, 0),
                                          ("f32", 3, 1), ("f32", 33, 1), ("f32", 3, 2), ("f32", 33, 2),
                                          ("f32", 3, 3), ("f32", 33, 3), ("f32", 3, 4), ("f32", 33, 4),
                                          ("f32", 3, 5), ("f32", 33, 5), ("f32", 3, 6), ("f32", 33, 6)])
def test_forward_matches_oracle_butterfly(fio, oracle, N, q, phase, s, e, prec, nrhs, sw):
    # sw: switch kernel of the FP32 form (0 FP32 FMA, 1 tensor cores with the kernel matrix in
    # shared memory, 2 warp-specialised FP32 FMA, 3 tensor cores with it in tensor memory, 4 as
    # 3 with wide MMAs, 5 and 6 as 3 and 4 with three split-TF32 products), forced past the
    # autotuner
    pid, prm = PH[phase]
    plan = fio.Plan(N, q, pid, prm, prec, nrhs_max=nrhs, s=s, e=e)
    try:
        if sw is not None:
            set_switch(fio, plan, sw, q)
        F = gaussian_batch(N, range(100, 100 + nrhs))
        f = torch.from_numpy(F).to(plan.dtype).cuda()
        u = plan.apply(f).cpu().numpy()
        torch.cuda.synchronize()
        plan.check()  # no bounded device-side wait expired
        tol = F64_TOL if prec == "f64" else F32_TOL
        for r in range(nrhs):
            ref = oracle_bf(oracle, N, q, phase, F[r].astype(np.complex64).astype(np.complex128) if prec == "f32" else F[r],
                            plan.info.s, e)
            assert rel(u[r], ref) < tol, (r, rel(u[r], ref))
    finally:
        plan.close()


@pytest.mark.parametrize("N,q,phase,s,e", [(64, 5, "ellipse", 0, 2), (128, 7, "circle", 3, 2), (32, 3, "separable", 0, 1)])
@pytest.mark.parametrize("prec,nrhs,sw", [("f64", 1, None), ("f64", 3, None), ("f32", 10, 0), ("f32", 10, 1),
                                          ("f32", 10, 2), ("f32", 10, 3), ("f32", 10, 4), ("f32", 10, 5),
                                          ("f32", 10, 6)])
def test_adjoint_matches_oracle_adjoint(fio, oracle, N, q, phase, s, e, prec, nrhs, sw):
    pid, prm = PH[phase]
    plan = fio.Plan(N, q, pid, prm, prec, nrhs_max=nrhs, s=s, e=e)
    try:
        if sw is not None:
            set_switch(fio, plan, sw, q)
        G = gaussian_batch(N, range(200, 200 + nrhs))
        g = torch.from_numpy(G).to(plan.dtype).cuda()
        fb = plan.adjoint(g).cpu().numpy()
        plan.check()
        tol = F64_TOL if prec == "f64" else F32_TOL
        for r in range(nrhs):
            gr = G[r].astype(np.complex64).astype(np.complex128) if prec == "f32" else G[r]
            ref = oracle.butterfly_adjoint(N, q, pid, list(prm), gr, s=plan.info.s, e=e)
            assert rel(fb[r], ref) < tol, (r, rel(fb[r], ref))
    finally:
        plan.close()


@pytest.mark.parametrize("N,q,s,e", [(64, 5, 0, 2), (128, 5, 3, 1), (32, 9, 3, 0)])
def test_every_stage_matches_oracle(fio, oracle, N, q, s, e):
    plan = fio.Plan(N, q, "ellipse", ELL16, "f64", nrhs_max=1, s=s, e=e)
    try:
        F = gaussian_sources(N, 7)
        f = torch.from_numpy(F).cuda()
        for st in range(plan.info.nstages):
            got = plan.debug_stage(f, st).cpu().numpy()
            _, ref = oracle.butterfly(N, q, 1, list(ELL16), F, s=plan.info.s, e=e, stage=st)
            assert rel(got, ref) < F64_TOL, (st, rel(got, ref))
    finally:
        plan.close()


@pytest.mark.parametrize("prec,tol,sw", [("f64", 1e-12, None), ("f32", 1e-6, 0), ("f32", 1e-6, 1), ("f32", 1e-6, 2),
                                         ("f32", 1e-6, 3), ("f32", 1e-6, 4), ("f32", 1e-6, 5), ("f32", 1e-6, 6)])
@pytest.mark.parametrize("N,q,e", [(64, 5, 2), (256, 9, 2)])
def test_dot_test(fio, prec, tol, sw, N, q, e):
    plan = fio.Plan(N, q, "ellipse", ELL16, prec, nrhs_max=2, e=e)
    try:
        if sw is not None:
            set_switch(fio, plan, sw, q)
        f = torch.from_numpy(gaussian_batch(N, [1, 2])).to(plan.dtype).cuda()
        g = torch.from_numpy(gaussian_batch(N, [3, 4])).to(plan.dtype).cuda()
        Bf = plan.apply(f).to(torch.complex128)
        Bg = plan.adjoint(g).to(torch.complex128)
        for r in range(2):
            g64 = g[r].to(torch.complex128).flatten()
            a = torch.vdot(g64, Bf[r].flatten())
            b = torch.vdot(Bg[r].flatten(), f[r].to(torch.complex128).flatten())
            # residual against ||g|| ||Bf|| (the Cauchy-Schwarz bound of a rounding-level
            # perturbation) at every size; against |<g, Bf>| itself where the inner
            # product sums enough terms (FP64, or N >= 256) not to be small by chance
            assert abs(a - b).item() < tol * (g64.norm() * Bf[r].norm()).item()
            if prec == "f64" or N >= 256:
                assert abs(a - b).item() < tol * abs(a).item()
    finally:
        plan.close()


@pytest.mark.parametrize("N,q,phase,nrhs", [(64, 9, "ellipse", 33), (128, 5, "circle", 7)])
@pytest.mark.parametrize("sw,tile,rs", [(0, 4, 2), (0, 8, 4), (0, 8, 8), (2, 4, 8), (3, 4, 4), (4, 4, 32), (5, 4, 32),
                                       (6, 4, 8)])
def test_every_tuning_choice_matches_oracle(fio, oracle, N, q, phase, nrhs, sw, tile, rs):
    # the autotuner picks among these per plan; each must give the oracle's result
    pid, prm = PH[phase]
    plan = fio.Plan(N, q, pid, prm, "f32", nrhs_max=nrhs)
    try:
        plan.set_tuning(sw, tile, rs, rs)
        assert (plan.info.switch_impl, plan.info.switch_rhs_tile, plan.info.trans_rs, plan.info.trans_rs_x) == (
            sw, tile, rs, rs)
        F = gaussian_batch(N, range(300, 300 + nrhs))
        U = plan.apply(torch.from_numpy(F).to(plan.dtype).cuda()).cpu().numpy()
        G = plan.adjoint(torch.from_numpy(F).to(plan.dtype).cuda()).cpu().numpy()
        for r in (0, nrhs - 1):
            assert rel(U[r], oracle_bf(oracle, N, q, phase, F[r], -1, 2)) < F32_TOL
            ref = oracle.butterfly_adjoint(N, q, pid, list(prm), F[r])
            assert rel(G[r], ref) < F32_TOL
    finally:
        plan.close()


def test_zero_input_gives_zero_and_linearity(fio):
    N = 64
    plan = fio.Plan(N, 5, "ellipse", ELL16, "f64", nrhs_max=3)
    try:
        z = torch.zeros(1, N, N, dtype=torch.complex128, device="cuda")
        assert plan.apply(z).abs().max().item() == 0.0
        F = torch.from_numpy(gaussian_batch(N, [5, 6])).cuda()
        a, b = 0.3 - 1.1j, 2.0 + 0.5j
        comb = torch.stack([F[0], F[1], a * F[0] + b * F[1]])
        U = plan.apply(comb)
        assert (U[2] - (a * U[0] + b * U[1])).abs().max().item() < 1e-12 * U.abs().max().item()
    finally:
        plan.close()


def test_nrhs_batch_equals_single_calls(fio):
    N = 64
    plan = fio.Plan(N, 7, "circle", CIRC20, "f32", nrhs_max=11)
    try:
        F = torch.from_numpy(gaussian_batch(N, range(11))).to(torch.complex64).cuda()
        U = plan.apply(F)
        # each RHS is independent; the switch splits its inner sums by the number of RHS
        # sharing a CTA, so a RHS applied alone agrees to FP32 rounding, not bit for bit
        for r in (0, 7, 10):
            one = plan.apply(F[r:r + 1])[0]
            assert ((one - U[r]).norm() / U[r].norm()).item() < 1e-6
        assert torch.equal(plan.apply(F)[10], U[10])  # the same call shape is bit-stable
    finally:
        plan.close()


def test_apply_host_matches_device(fio):
    N = 128
    plan = fio.Plan(N, 5, "ellipse", ELL16, "f32", nrhs_max=4)
    try:
        F = torch.from_numpy(gaussian_batch(N, range(4))).to(torch.complex64)
        dev = plan.apply(F.cuda()).cpu()
        out = torch.empty_like(F).pin_memory()
        plan.apply_host(F.pin_memory(), out)
        assert torch.equal(out, dev)
        gb = plan.adjoint(F.cuda()).cpu()
        plan.apply_host(F.pin_memory(), out, adjoint=True)
        assert torch.equal(out, gb)
    finally:
        plan.close()


def test_bad_arguments_raise(fio):
    plan = fio.Plan(64, 5, "ellipse", ELL16, "f32", nrhs_max=2)
    try:
        with pytest.raises(fio.FIOError):
            plan.apply(torch.zeros(3, 64, 64, dtype=torch.complex64, device="cuda"))
        with pytest.raises(TypeError):
            plan.apply(torch.zeros(1, 64, 64, dtype=torch.complex128, device="cuda"))
        with pytest.raises(fio.FIOError):
            plan.debug_stage(torch.zeros(1, 64, 64, dtype=torch.complex64, device="cuda"), 99)
    finally:
        plan.close()
    for kw in (dict(N=96, q=5), dict(N=64, q=4), dict(N=64, q=5, e=5)):
        with pytest.raises(fio.FIOError):
            fio.Plan(kw.pop("N"), kw.pop("q"), "ellipse", ELL16, "f32", **kw)


def test_autograd_backward_is_adjoint(fio):
    N = 64
    plan = fio.Plan(N, 5, "ellipse", ELL16, "f64", nrhs_max=1)
    try:
        f = torch.from_numpy(gaussian_sources(N, 8))[None].cuda().requires_grad_(True)
        ustar = torch.from_numpy(gaussian_sources(N, 9))[None].cuda()
        loss = (fio.fio_apply(f, plan) - ustar).abs().pow(2).sum()
        loss.backward()
        with torch.no_grad():
            ref = 2.0 * plan.adjoint(plan.apply(f) - ustar)
        assert (f.grad - ref).abs().max().item() < 1e-12 * ref.abs().max().item()
    finally:
        plan.close()


def test_accuracy_against_direct_sum_medium(fio, oracle):
    # both forms against eq. dfio on sampled x; the FP32 form meets max(2 x FP64 error, 1e-5).
    # At q=9 the oracle butterfly's own error for this phase is ~4e-6 (Sec. 5 behaviour).
    N, q = 256, 9
    F = gaussian_sources(N, 1)
    xi = sample_indices(N, 512, 1000)
    ref = oracle.direct(N, 1, list(ELL16), F, xi)
    errs = {}
    for prec in ("f64", "f32"):
        plan = fio.Plan(N, q, "ellipse", ELL16, prec, nrhs_max=1)
        try:
            u = plan.apply(torch.from_numpy(F).to(plan.dtype).cuda()).cpu().numpy().reshape(-1)
            errs[prec] = rel(u[xi], ref)
        finally:
            plan.close()
    assert errs["f64"] < 3e-5
    assert errs["f32"] <= max(2 * errs["f64"], 1e-5)


@pytest.mark.parametrize("N,q,nrhs", [(256, 9, 32), (256, 9, 7), (128, 11, 32), (256, 5, 40)])
def test_tensor_memory_switch_matches_fma_switch(fio, N, q, nrhs):
    # the persistent tensor-core switch walks hundreds of pairs per CTA (its tensor-memory
    # and shared-memory rings wrap many times); forward and adjoint must agree with the FFMA
    # switch on the same plan within the FP32 tolerance, with no bounded wait expiring
    plan = fio.Plan(N, q, "ellipse", ELL16, "f32", nrhs_max=nrhs)
    try:
        f = torch.from_numpy(gaussian_batch(N, range(400, 400 + nrhs))).to(plan.dtype).cuda()
        out = {}
        for sw in (0, 3, 4, 5, 6):
            plan.set_switch(sw)
            out[sw] = (plan.apply(f).to(torch.complex128), plan.adjoint(f).to(torch.complex128))
            plan.check()
        for k in range(2):
            for sw in (3, 4, 5, 6):
                a, b = out[sw][k], out[0][k]
                for r in range(nrhs):
                    assert rel(a[r].cpu().numpy(), b[r].cpu().numpy()) < 2e-6, (sw, k, r)
    finally:
        plan.close()


# register-tiled translations (trans_rs 32 for the p-shape, trans_rs_x 32 for the x-shape),
# each shape also beside the other's subtile kernel.  Cases cover the
# bulk-copy staging (even RHS counts), the cp.async fallback (odd counts), full and
# partial 32-RHS tiles, several tiles, s = 0 (three levels of each recursion) and
# every phase
REG_CASES = [(64, 9, "ellipse", 32, 3, 2), (128, 7, "circle", 10, 3, 2), (64, 5, "ellipse", 33, 0, 2),
             (32, 3, "separable", 2, 0, 1), (128, 9, "linear", 64, 3, 0)]


@pytest.mark.parametrize("N,q,phase,nrhs,s,e", REG_CASES)
@pytest.mark.parametrize("rs,rsx", [(32, 32), (32, 4), (8, 32)])
def test_register_tiled_translations_match_oracle(fio, oracle, N, q, phase, nrhs, s, e, rs, rsx):
    pid, prm = PH[phase]
    plan = fio.Plan(N, q, pid, prm, "f32", nrhs_max=nrhs, s=s, e=e)
    try:
        plan.set_tuning(-1, -1, rs, rsx)
        assert (plan.info.trans_rs, plan.info.trans_rs_x) == (rs, rsx)
        F = gaussian_batch(N, range(500, 500 + nrhs))
        f = torch.from_numpy(F).to(plan.dtype).cuda()
        U = plan.apply(f).cpu().numpy()
        G = plan.adjoint(f).cpu().numpy()
        plan.check()  # no bounded wait on the staging expired
        for r in sorted({0, nrhs // 2, nrhs - 1}):
            Fr = F[r].astype(np.complex64).astype(np.complex128)
            assert rel(U[r], oracle_bf(oracle, N, q, phase, Fr, plan.info.s, e)) < F32_TOL, r
            ref = oracle.butterfly_adjoint(N, q, pid, list(prm), Fr, s=plan.info.s, e=e)
            assert rel(G[r], ref) < F32_TOL, r
    finally:
        plan.close()
