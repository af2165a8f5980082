"""Batches of FP32 plans (fio_batch_*): one persistent launch per butterfly step and
(q, s) group, replayed from captured CUDA graphs.

* every plan's slice of a batched apply (forward and adjoint) equals, bit for bit,
  fio_apply / fio_apply_adjoint of that plan alone with the FP32 FMA switch and the
  RHS-subtile translations (the kernels a batch runs): the
  batched kernels run the same per-unit code, only the assignment of units to
  CTAs differs;
* the uneven-batch workload (96 plans, N in {64..512}, q in {5, 7, 9}, 1-8 RHS,
  ellipse and c(x)|k| phases, seed 4) is checked the same way, and plans of every
  (N <= 128, q) class against the oracle's FP64 butterfly at equal q;
* replays with other buffers, autotuned grids, and the dot test of every plan of the
  batch, normalised by ||g|| ||B f||.
"""
import numpy as np
import pytest
import torch

from paper_0809_0719_gb300.inputs import gaussian_batch, uneven_batch_sources, uneven_batch_specs

pytestmark = pytest.mark.gpu

SEP = (0.3, 0.2, 0.25, 0.1)
PARAMS = {"ellipse": (2.0, 1.0, 16.0, 1.0), "circle": (3.0, 1.0, 20.0, 1.0), "linear": (), "separable": SEP}
PID = {"linear": 0, "ellipse": 1, "circle": 2, "separable": 3}

# (N, q, phase, nrhs): several q and s groups (N = 8: s = 1; N = 16, 32: s = 2), an
# nrhs above 32 (two RHS tiles per unit), all four phases
SMALL = [(16, 3, "ellipse", 2), (32, 5, "circle", 1), (64, 7, "linear", 3), (32, 5, "separable", 33),
         (64, 5, "ellipse", 4), (8, 3, "circle", 1), (128, 7, "ellipse", 2), (64, 9, "circle", 5)]


@pytest.fixture(scope="module")
def fio():
    from paper_0809_0719_gb300 import fio as F

    assert torch.cuda.is_available()
    return F


def _plans(fio, specs):
    # the kernels a batch runs: the FFMA switch and the RHS-subtile translations (a plan alone
    # may otherwise be tuned to the register-tiled translations, which sum in another order)
    plans = []
    for N, q, phase, nrhs in specs:
        p = fio.Plan(N, q, phase, PARAMS[phase], "f32", nrhs_max=nrhs)
        p.set_tuning(0, -1, 8, 8)
        plans.append(p)
    return plans


def _sources(specs, base):
    return [torch.from_numpy(gaussian_batch(N, [base + 100 * i + r for r in range(nrhs)])).to(torch.complex64).cuda()
            for i, (N, q, phase, nrhs) in enumerate(specs)]


def _check_equal_singles(batch, plans, xs, adjoint):
    y = batch.unpack(batch.apply(batch.pack(xs), adjoint=adjoint))
    torch.cuda.synchronize()
    for i, p in enumerate(plans):
        ref = p.adjoint(xs[i]) if adjoint else p.apply(xs[i])
        assert torch.equal(y[i], ref), (i, p.N, p.q, adjoint, (y[i] - ref).abs().max().item())


@pytest.mark.parametrize("tune", [False, True])
def test_small_mixed_batch_equals_single_plans(fio, tune):
    plans = _plans(fio, SMALL)
    batch = fio.Batch(plans, [s[3] for s in SMALL], tune=tune)
    try:
        assert batch.info.ngroups == len({(q, min(3, (N.bit_length() - 1) // 2)) for N, q, _, _ in SMALL})
        assert batch.info.tuned == int(tune)
        for base, adj in ((1, False), (2, True), (3, False)):  # third call: new buffers through the io slot
            _check_equal_singles(batch, plans, _sources(SMALL, base), adj)
    finally:
        batch.close()
        for p in plans:
            p.close()


def test_batch_profile_counts_the_schedule(fio):
    plans = _plans(fio, SMALL)
    batch = fio.Batch(plans, [s[3] for s in SMALL])
    try:
        x = batch.pack(_sources(SMALL, 4))
        for adj in (False, True):
            prof = batch.profile(x, adjoint=adj)
            n = sum(v[0] for v in prof.values())
            assert n == (batch.info.launches_adj if adj else batch.info.launches_fwd)
            assert all(k.startswith("b_") for k in prof)
    finally:
        batch.close()
        for p in plans:
            p.close()


def test_batch_rejects_bad_arguments(fio):
    p64 = fio.Plan(16, 3, "ellipse", PARAMS["ellipse"], "f64", nrhs_max=1)
    p32 = fio.Plan(16, 3, "ellipse", PARAMS["ellipse"], "f32", nrhs_max=2)
    try:
        with pytest.raises(fio.FIOError):
            fio.Batch([p64], [1])          # FP64 plans cannot be batched
        with pytest.raises(fio.FIOError):
            fio.Batch([p32], [3])          # nrhs above nrhs_max
        with pytest.raises(fio.FIOError):
            fio.Batch([p32, p32], [1, 1])  # the same plan twice
        b = fio.Batch([p32], [2])
        with pytest.raises(ValueError):
            b.apply(torch.zeros(5, dtype=torch.complex64, device="cuda"))
        b.close()
    finally:
        p64.close()
        p32.close()


@pytest.fixture(scope="module")
def uneven(fio):
    specs = uneven_batch_specs()
    plans = []
    for sp in specs:
        p = fio.Plan(sp["N"], sp["q"], sp["phase"], sp["params"], "f32", nrhs_max=sp["nrhs"])
        p.set_tuning(0, -1, 8, 8)
        plans.append(p)
    batch = fio.Batch(plans, [sp["nrhs"] for sp in specs], tune=True)
    xs = [torch.from_numpy(uneven_batch_sources(sp, i)).to(torch.complex64).cuda() for i, sp in enumerate(specs)]
    yield specs, plans, batch, xs
    batch.close()
    for p in plans:
        p.close()


def test_uneven_batch_equals_single_plans(uneven):
    specs, plans, batch, xs = uneven
    assert batch.info.nplans == 96 and batch.info.ngroups == 3
    assert batch.offsets[-1] == sum(sp["nrhs"] * sp["N"] ** 2 for sp in specs)
    _check_equal_singles(batch, plans, xs, False)
    _check_equal_singles(batch, plans, xs, True)


def test_uneven_batch_against_oracle_butterfly(uneven, oracle):
    specs, plans, batch, xs = uneven
    y = batch.unpack(batch.apply(batch.pack(xs)))
    seen = set()
    for i, sp in enumerate(specs):
        key = (sp["N"], sp["q"])
        if sp["N"] > 128 or key in seen:
            continue
        seen.add(key)
        f = xs[i][0].cpu().numpy().astype(np.complex128)
        ref = oracle.butterfly(sp["N"], sp["q"], PID[sp["phase"]], sp["params"], f)
        err = oracle.rel_l2(y[i][0].cpu().numpy(), ref)
        assert err < 1e-5, (i, key, err)
    assert len(seen) == 6


def test_uneven_batch_dot_test(uneven):
    specs, plans, batch, xs = uneven
    gs = [torch.from_numpy(gaussian_batch(sp["N"], [777 + 100 * i + r for r in range(sp["nrhs"])])).to(torch.complex64).cuda()
          for i, sp in enumerate(specs)]
    bf = batch.unpack(batch.apply(batch.pack(xs)))
    bg = batch.unpack(batch.apply(batch.pack(gs), adjoint=True))
    # |<g, B f> - <B^H g, f>| against ||g|| ||B f||: by Cauchy-Schwarz the FP32 rounding
    # of either apply (relative ~4e-7 per output) contributes at most that fraction
    for i in range(len(specs)):
        g64, f64 = gs[i].flatten().to(torch.complex128), xs[i].flatten().to(torch.complex128)
        bf64, bg64 = bf[i].flatten().to(torch.complex128), bg[i].flatten().to(torch.complex128)
        a, b = torch.vdot(g64, bf64), torch.vdot(bg64, f64)
        r = abs(a - b).item() / (g64.norm() * bf64.norm()).item()
        assert r < 1e-6, (i, r)


def test_apply_batch_with_one_pointer_per_plan(fio):
    # fio_apply_batch(plans, nplans, f[], u[], nrhs[], stream): each plan's own input and
    # output pointer; bit-identical to each plan alone (FFMA switch, subtile translations),
    # forward and adjoint,
    # on repeated calls (the kept batch) and after a plan of the list is destroyed and the
    # list rebuilt (the kept batch is dropped with it)
    plans = _plans(fio, SMALL)
    try:
        for base, adj in ((4, False), (5, True), (6, False)):
            xs = _sources(SMALL, base)
            ys = fio.apply_batch(plans, xs, adjoint=adj)
            torch.cuda.synchronize()
            for i, p in enumerate(plans):
                ref = p.adjoint(xs[i]) if adj else p.apply(xs[i])
                assert torch.equal(ys[i], ref), (i, adj)
        # drop one plan and rebuild it: the library's kept batch for the old list must go
        plans[1].close()
        N, q, phase, nrhs = SMALL[1]
        plans[1] = fio.Plan(N, q, phase, PARAMS[phase], "f32", nrhs_max=nrhs)
        plans[1].set_tuning(0, -1, 8, 8)
        xs = _sources(SMALL, 7)
        ys = fio.apply_batch(plans, xs)
        torch.cuda.synchronize()
        for i, p in enumerate(plans):
            assert torch.equal(ys[i], p.apply(xs[i])), i
        # the workspace figure is the two state levels of 2^e N^2 q^2 complex64 per RHS
        p = plans[0]
        assert p.workspace_bytes(2) == 2 * (p.N * p.N << p.info.e) * 2 * p.q * p.q * 8
    finally:
        for p in plans:
            p.close()
