"""Weighted harmonic-average boundary dielectric (Sec. 2.7) on the GPU against the
FP64 oracle: the FP64 edge arrays bit-exact (the same interval arithmetic,
rounded operation by operation), the operator, FP64 PCG and FP32 refinement
parity, the Born ion converging, and the argument errors."""
import numpy as np
import pytest

import oracle
from paper_1704_02745_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

COULOMB = 332.0637


@pytest.fixture(scope="module")
def pbm():
    from paper_1704_02745_gb300 import build, pb
    build.build()
    pb.load()
    return pb


@pytest.fixture(scope="module")
def ctx(pbm):
    c = pbm.Context(0)
    yield c
    c.close()


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype).cuda()


def rel_max(a, b):
    return float(np.max(np.abs(np.asarray(a) - np.asarray(b))) / max(np.max(np.abs(np.asarray(b))), 1e-300))


MAKERS = [lambda: inputs.random_small(5, 7, 9, 11, n_atoms=40),
          lambda: inputs.random_small(6, 37, 29, 45, n_atoms=120),
          lambda: inputs.small_33()]


def harmonic(p, coef="f64"):
    return p.grid.replace(eps_model="harmonic", coef=coef)


@pytest.mark.parametrize("maker", MAKERS)
def test_setup_arrays(pbm, ctx, maker):
    p = maker()
    spec = harmonic(p)
    s = oracle.setup(spec, p.atoms)
    with pbm.Grid(ctx, spec, p.atoms) as g:
        assert np.array_equal(g.export("eps_x"), s.ex)
        assert np.array_equal(g.export("eps_y"), s.ey)
        assert np.array_equal(g.export("eps_z"), s.ez)
        assert np.array_equal(g.export("lambda"), s.lam)
        assert rel_max(g.export("b"), s.b) < 1e-13
    partial = (s.ex > spec.eps_in) & (s.ex < spec.eps_out)
    assert partial.any()


@pytest.mark.parametrize("maker", MAKERS[:2])
def test_apply(pbm, ctx, maker):
    p = maker()
    s = oracle.setup(harmonic(p), p.atoms)
    u = np.random.default_rng(2).normal(size=p.grid.shape)
    want = oracle.apply(s, u)
    with pbm.Grid(ctx, harmonic(p, "f64"), p.atoms) as g:
        du = dev(u)
        dau = torch.empty_like(du)
        g.apply(du, dau, pbm.PB_F64)
        assert rel_max(dau.cpu().numpy(), want) < 1e-13
    with pbm.Grid(ctx, harmonic(p, "f32"), p.atoms) as g:
        du = dev(u, torch.float32)
        dau = torch.empty_like(du)
        g.apply(du, dau, pbm.PB_F32)
        assert rel_max(dau.cpu().numpy(), want) < 2e-6


def test_pcg_f64_parity(pbm, ctx):
    p = inputs.small_33()
    s = oracle.setup(harmonic(p), p.atoms)
    ref = oracle.pcg(s, tol=1e-10)
    e_ref = oracle.energy(s, ref.phi)
    phi = torch.zeros(p.grid.shape, dtype=torch.float64, device="cuda")
    with pbm.Grid(ctx, harmonic(p), p.atoms) as g:
        info = g.solve(phi, precision="f64", tol=1e-10)
        e = g.energy(phi)
    assert info.status == 0
    assert rel_max(phi.cpu().numpy(), ref.phi) <= 1e-8
    assert abs(e - e_ref) <= 1e-8 * abs(e_ref)
    assert abs(info.iterations - ref.iters) <= max(1, 0.02 * ref.iters)


@pytest.mark.parametrize("coef", ["f32", "bf16", "f64"])
def test_refinement_parity(pbm, ctx, coef):
    """The FP32 inner solve on FP32 / BF16 copies (or packed-free FP32 copies of
    the FP64 edges), the FP64 residual on the FP64 edges: refinement reaches
    the FP64 solution."""
    p = inputs.random_small(6, 37, 29, 45, n_atoms=120)
    s = oracle.setup(harmonic(p), p.atoms)
    ref = oracle.pcg(s, tol=1e-11)
    e_ref = oracle.energy(s, ref.phi)
    phi = torch.zeros(p.grid.shape, dtype=torch.float64, device="cuda")
    with pbm.Grid(ctx, harmonic(p, coef), p.atoms) as g:
        info = g.solve(phi, precision="f32_refine", tol=1e-9, inner_tol=1e-3)
        e = g.energy(phi)
    assert info.status == 0 and info.relres_true < 1e-9
    assert abs(e - e_ref) <= 1e-7 * abs(e_ref)


def test_born_ion_harmonic_on_the_gpu(pbm, ctx):
    a, ein, eout = 2.0, 1.0, 80.0
    exact = COULOMB / (2 * a) * (1 / eout - 1 / ein)
    errs = []
    for n, h in ((41, 0.5), (81, 0.25), (161, 0.125)):
        p = inputs.single_charge(n, h, ionic_strength=0.0)
        spec = p.grid.replace(eps_model="harmonic", coef="f32")
        phi = torch.zeros(spec.shape, dtype=torch.float64, device="cuda")
        out = ctx.solvation(spec, p.atoms, phi, precision="f32_refine", tol=1e-9)
        errs.append(abs(out.dG - exact) / abs(exact))
        if n == 41:
            want = oracle.solvation_energy(spec, p.atoms, tol=1e-11)[0]
            assert abs(out.dG - want) <= 1e-6 * abs(want)
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] < 0.02


def test_harmonic_argument_errors(pbm, ctx):
    p = inputs.random_small(3, 12, 12, 12, n_atoms=4)
    for bad in (harmonic(p, "packed"), harmonic(p).replace(periodic=True)):
        with pytest.raises(pbm.PbError) as ei:
            pbm.Grid(ctx, bad, p.atoms)
        assert ei.value.status == pbm.PB_ERR_ARG
    with pbm.Server(ctx, 1 << 30) as srv:
        with pytest.raises(pbm.PbError) as ei:
            srv.submit(1, harmonic(p), p.atoms)
        assert ei.value.status == pbm.PB_ERR_ARG
