"""pb_energy_noalloc: the energy for callers that cannot allocate device memory
(an MD engine whose allocator owns all device memory, or a time-critical loop
where cudaMalloc/cudaFree and their device synchronisation are not allowed).

Called through the C ABI with the caller's device arrays only, it must give
what pb_energy gives, on two calls in a row (the second reuses the library's
fixed scratch array left over from the first).  This file is collected last."""
import numpy as np
import pytest

from paper_1704_02745_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_energy_noalloc_matches_pb_energy_twice():
    from paper_1704_02745_gb300 import build, pb
    build.build()
    pb.load()
    p = inputs.random_small(31, 37, 29, 41, n_atoms=700)
    q = inputs.random_small(32, 37, 29, 41, n_atoms=300)
    rng = np.random.default_rng(5)
    with pb.Context(0) as ctx:
        stream = torch.cuda.current_stream().cuda_stream
        for prob in (p, q):
            with pb.Grid(ctx, prob.grid, prob.atoms) as g:
                phi = torch.as_tensor(rng.normal(size=prob.grid.shape)).cuda()
                want = g.energy(phi)  # the existing entry point (library scratch)
                xyzq = torch.as_tensor(np.concatenate([prob.atoms.xyz, prob.atoms.q[:, None]], 1)).cuda()
                out = torch.zeros(1, dtype=torch.float64, device="cuda")
                pb.pb_energy_noalloc(xyzq.contiguous(), prob.grid, phi, out, stream)
                torch.cuda.synchronize()
                got = float(out.item())
                assert abs(got - want) <= 1e-12 * max(abs(want), 1.0)
    # sizes beyond the fixed array are refused before any device work
    import ctypes
    org = (ctypes.c_double * 3)(0.0, 0.0, 0.0)
    st = pb.load().pb_energy_noalloc(4096 * 256 + 1, None, 4, 4, 4, 0.5, org, None, None, None)
    assert st == pb.PB_ERR_ARG
