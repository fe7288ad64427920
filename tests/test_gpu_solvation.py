"""Electrostatic solvation energy (Sec. 3.1, Figs. 1-2) through pb_solvation_energy:
the solvated system minus the reference system (eps_in everywhere, no salt),
against the FP64 oracle, and the Born ion's analytic value as h shrinks."""
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


def phi_for(spec):
    return torch.zeros(spec.shape, dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("precision,tol,bound", [("f64", 1e-10, 1e-8), ("f32_refine", 1e-9, 1e-7)])
def test_solvation_matches_oracle(pbm, ctx, precision, tol, bound):
    p = inputs.small_33()
    dG, e1, e0 = oracle.solvation_energy(p.grid, p.atoms, tol=1e-11)
    phi = phi_for(p.grid)
    out = ctx.solvation(p.grid, p.atoms, phi, precision=precision, tol=tol)
    scale = max(abs(e1), abs(e0))
    assert abs(out.e_solv - e1) <= bound * scale
    assert abs(out.e_ref - e0) <= bound * scale
    assert abs(out.dG - dG) <= 2 * bound * scale
    assert out.dG == out.e_solv - out.e_ref
    # phi holds the solvated potential
    s = oracle.setup(p.grid, p.atoms)
    assert oracle.relres(s, phi.cpu().numpy()) < 10 * tol
    assert out.solv.status == 0 and out.ref.status == 0


def test_born_ion_on_the_gpu(pbm, ctx):
    a, ein, eout = 2.0, 1.0, 80.0
    exact = COULOMB / (2 * a) * (1 / eout - 1 / ein)
    errs = []
    for n, h in ((41, 0.5), (81, 0.25), (161, 0.125)):
        p = inputs.single_charge(n, h, ionic_strength=0.0)
        out = ctx.solvation(p.grid, p.atoms, phi_for(p.grid), precision="f32_refine", tol=1e-9)
        errs.append(abs(out.dG - exact) / abs(exact))
        if n == 41:  # the same discrete problem as the oracle's
            want = oracle.solvation_energy(p.grid, p.atoms, tol=1e-11)[0]
            assert abs(out.dG - want) <= 1e-6 * abs(want)
    assert errs[0] > errs[1] > errs[2]
    assert errs[1] < 0.02
