"""The FP64 reassembly entry point that allocates no device memory.

Some callers cannot allocate device memory while they run: a framework that
owns the whole device pool and hands out fixed budgets, or a latency-critical
solver loop in which a driver allocation (which can synchronise the device)
would stall.  fem_assemble_all_noalloc serves them: its scratch lives in a
fixed array inside the library.  These tests check, through the C ABI, that
two calls in a row give the same CSR values as the ordinary entry point
fem_assemble_all bit for bit (both run the same FP64 element kernel and the
same fixed-order CSR sum, so any difference is a layout mistake), for all
three matrices and for each one alone; that no device memory is taken by the
calls after the first; that host pointers and a mesh too large for the array
are refused.  The file name makes pytest collect it last.
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


def _values(fm, which):
    return {k: torch.empty(fm.nnz, dtype=torch.float64, device="cuda") for k in which}


def _setup(case):
    wl = mg.workload("tri_p2_1024", scale=41) if case == "tri_p2" else mg.workload("tet_p2_64", scale=5)
    fm = FemMesh.of(wl.mesh)
    fm.symbolic()
    u = torch.tensor(wl.u, dtype=torch.float64, device="cuda")
    k = F.coeff(wl.coeff.kind, wl.coeff.params)
    return fm, u, k


@pytest.mark.parametrize("which", ["MKT", "M", "K", "T"])
@pytest.mark.parametrize("case", ["tri_p2", "tet_p2"])
def test_noalloc_matches_assemble_all_twice(case, which):
    fm, u, k = _setup(case)
    ref = _values(fm, which)
    F.fem_assemble_all(fm.h, k, u, F.FEM_FP64, ref.get("M"), ref.get("K"), ref.get("T"))
    torch.cuda.synchronize()
    u_arg = None if which == "M" else u     # M alone needs no nodal values
    # the first call on the device loads the library's fixed array (a one-time
    # driver allocation); the calls after it must take no device memory at all
    warm = _values(fm, which)
    F.fem_assemble_all_noalloc(fm.h, k, u_arg, warm.get("M"), warm.get("K"), warm.get("T"))
    torch.cuda.synchronize()
    outs = [_values(fm, which) for _ in range(2)]
    for o in outs:
        for v in o.values():
            v.fill_(np.nan)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    mesh_bytes0 = F.fem_mesh_get_info(fm.h).device_bytes
    for o in outs:
        F.fem_assemble_all_noalloc(fm.h, k, u_arg, o.get("M"), o.get("K"), o.get("T"))
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert F.fem_mesh_get_info(fm.h).device_bytes == mesh_bytes0
    for o in outs:
        for name in which:
            assert torch.equal(o[name], ref[name]), name
    F.fem_device_status()


def test_noalloc_refuses_host_pointers():
    fm, u, k = _setup("tri_p2")
    out = _values(fm, "MKT")
    host = np.zeros(fm.nnz, dtype=np.float64)
    with pytest.raises(F.FemError) as ei:
        F.fem_assemble_all_noalloc(fm.h, k, u, host, out["K"], out["T"])
    assert ei.value.code == F.FEM_EINVAL
    u_host = u.cpu().numpy()
    with pytest.raises(F.FemError) as ei:
        F.fem_assemble_all_noalloc(fm.h, k, u_host, out["M"], out["K"], out["T"])
    assert ei.value.code == F.FEM_EINVAL
    assert not np.any(host)


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
