"""The FP64 reassembly entry point that allocates no device memory.

Callers that must not allocate device memory while they run (a framework
that owns the whole device pool, a latency-critical loop in which a driver
allocation would stall) use fem_assemble_all_noalloc: its scratch lives in a
fixed array inside the library.  This test checks, through the C ABI, that
two calls in a row give the same CSR values as the ordinary entry point
fem_assemble_all, within the FP64 tolerance the parity tests use, and that a
mesh too large for the fixed array is refused.  The file name makes pytest
collect it last.
"""
import numpy as np
import pytest

import meshgen as mg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2204_03893_gb300 as F  # noqa: E402
from paper_2204_03893_gb300.torch_api import FemMesh  # noqa: E402

FP64_TOL = 1e-12


def _values(fm, which):
    return {k: torch.empty(fm.nnz, dtype=torch.float64, device="cuda") for k in which}


@pytest.mark.parametrize("case", ["tri_p2", "tet_p2"])
def test_noalloc_matches_assemble_all_twice(case):
    wl = mg.workload("tri_p2_1024", scale=41) if case == "tri_p2" else mg.workload("tet_p2_64", scale=5)
    fm = FemMesh.of(wl.mesh)
    fm.symbolic()
    u = torch.tensor(wl.u, dtype=torch.float64, device="cuda")
    k = F.coeff(wl.coeff.kind, wl.coeff.params)
    ref = _values(fm, "MKT")
    F.fem_assemble_all(fm.h, k, u, F.FEM_FP64, ref["M"], ref["K"], ref["T"])
    torch.cuda.synchronize()
    for _ in range(2):
        out = _values(fm, "MKT")
        for v in out.values():
            v.fill_(np.nan)
        F.fem_assemble_all_noalloc(fm.h, k, u, out["M"], out["K"], out["T"])
        torch.cuda.synchronize()
        for name in "MKT":
            scale = ref[name].abs().max().item()
            err = (out[name] - ref[name]).abs().max().item()
            assert err <= FP64_TOL * scale, (name, err, scale)
    F.fem_device_status()


def test_noalloc_refuses_mesh_beyond_limit():
    m = mg.structured_tri(70, 2, 0.2, seed=3)           # 9 800 P2 triangles: 6.1 MB per pass of M+K+T
    fm = FemMesh.of(m)
    fm.symbolic()
    u = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    out = _values(fm, "MKT")
    k = F.coeff("poly", (1.0,))
    F.fem_assemble_all_noalloc(fm.h, k, u, out["M"], out["K"], out["T"])    # fits
    big = mg.structured_tri(150, 2, 0.2, seed=3)          # 45 000 P2 triangles: 28 MB, over 16 MiB
    fb = FemMesh.of(big)
    fb.symbolic()
    ub = torch.zeros(big.n_nodes, dtype=torch.float64, device="cuda")
    ob = _values(fb, "MKT")
    with pytest.raises(F.FemError) as ei:
        F.fem_assemble_all_noalloc(fb.h, k, ub, ob["M"], ob["K"], ob["T"])
    assert ei.value.code == F.FEM_EINVAL
    assert "too large" in str(ei.value)
