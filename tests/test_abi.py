"""C ABI checks that need no GPU: libpb builds for sm_103a, loads, exports
every entry point that include/*.h declares, and the binding's struct layouts
match the C header."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1704_02745_gb300 import build as pbbuild
from paper_1704_02745_gb300 import pb

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        txt = open(os.path.join(ROOT, "include", h)).read()
        txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
        names.update(re.findall(r"\b(pb_\w+)\s*\(", txt))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    pbbuild.build()
    return pb.load()


def test_exports_every_declared_symbol(lib):
    decl = declared_functions()
    assert "pb_pcg_solve" in decl and "pb_setup_grid" in decl
    out = subprocess.run(["nm", "-D", "--defined-only", pbbuild.LIB], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r"\bT (pb_\w+)", out))
    missing = [n for n in decl if n not in exported]
    assert not missing, missing
    for n in decl:
        getattr(lib, n)
    assert set(pb.EXPORTED) <= set(decl)


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "sz.c"
    src.write_text("""
#include <stdio.h>
#include <stddef.h>
#include "pb.h"
int main(void) {
  printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\\n", sizeof(pb_grid_desc), sizeof(pb_solve_opts),
         sizeof(pb_solve_info), offsetof(pb_grid_desc, dh_precision),
         offsetof(pb_solve_opts, profile), offsetof(pb_solve_info, n_resid),
         sizeof(pb_request), sizeof(pb_result), sizeof(pb_kernel_profile), sizeof(pb_solvation),
         offsetof(pb_solvation, ref), sizeof(pb_tune_info), offsetof(pb_tune_info, us_best));
  return 0;
}
""")
    exe = tmp_path / "sz"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    want = [ctypes.sizeof(pb.GridDesc), ctypes.sizeof(pb.SolveOpts), ctypes.sizeof(pb.SolveInfo),
            pb.GridDesc.dh_precision.offset, pb.SolveOpts.profile.offset,
            pb.SolveInfo.n_resid.offset, ctypes.sizeof(pb.Request), ctypes.sizeof(pb.Result),
            ctypes.sizeof(pb.KernelProfile), ctypes.sizeof(pb.Solvation), pb.Solvation.ref.offset,
            ctypes.sizeof(pb.TuneInfo), pb.TuneInfo.us_best.offset]
    assert got == want


def test_errors_are_reported_without_gpu(lib):
    # no GPU in this container: the call must fail with a CUDA error, not crash
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    with pytest.raises(pb.PbError) as ei:
        pb.pb_create(0)
    assert ei.value.status in (pb.PB_ERR_CUDA, pb.PB_ERR_ARG)
    # argument checks that run before any CUDA call
    assert lib.pb_setup_grid(None, None, 0, None, None, None, None) == pb.PB_ERR_ARG
    assert lib.pb_pcg_solve(None, None, None, None) == pb.PB_ERR_ARG
    assert lib.pb_grid_bytes(None, 0) == 0
    assert lib.pb_grid_autotune(None, 0, None) == pb.PB_ERR_ARG
    assert lib.pb_pinned_alloc(16, None) == pb.PB_ERR_ARG
    assert lib.pb_pinned_free(None) == pb.PB_OK
    p = pb._P()
    st = lib.pb_pinned_alloc(4096, ctypes.byref(p))
    if st == pb.PB_OK:  # some drivers pin host memory without a GPU
        assert lib.pb_pinned_free(p) == pb.PB_OK
    else:
        assert st == pb.PB_ERR_OOM and not p.value


def test_grid_bytes_model(lib):
    from paper_1704_02745_gb300 import inputs
    d = pb.grid_desc(inputs.centered_grid(129, 0.5))
    n = 132 * 129 * 129
    b32 = pb.pb_grid_bytes(d, "f32_refine")
    b64 = pb.pb_grid_bytes(d, "f64")
    assert 40 * n < b32 < 60 * n
    assert b64 > b32


def test_pinned_pool_size_classes():
    """Page-locked phi buffers are pooled in size classes: a class holds the
    request, wastes at most a quarter of itself, and is a multiple of 4 KB;
    nearby grid sizes share a class (no GPU needed: only the arithmetic)."""
    from paper_1704_02745_gb300.pb import PinnedPool
    sizes = [8 * n ** 3 for n in range(9, 200, 2)] + [1, 7, 4096, 4097, 1 << 30]
    for b in sizes:
        c = PinnedPool.size_class(b)
        assert c >= b and c % 4096 == 0
        assert c <= max(4096, 1.25 * b) + 4096
        assert PinnedPool.size_class(c) == c  # a class is its own class
    assert PinnedPool.size_class(8 * 125 ** 3) == PinnedPool.size_class(8 * 127 ** 3)
    classes = [PinnedPool.size_class(b) for b in sorted(sizes)]
    assert classes == sorted(classes)
