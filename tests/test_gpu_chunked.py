"""Reassembly over ranges (fem_chunk_plan, fem_form_elements_range,
fem_sum_elements_range): element ranges formed and the slots they complete
summed range by range.  The plan's slot ranges must be exactly the slots whose
contributors are all formed, and the ranged values must equal one formation
followed by one sum bit for bit (same kernels, same per-slot order)."""
import numpy as np
import pytest

import meshgen as mg

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2204_03893_gb300 as F  # noqa: E402
from paper_2204_03893_gb300.torch_api import PRECISIONS, FemMesh  # noqa: E402


def mesh_of(name):
    if name == "tri_p2":
        return mg.structured_tri(48, 2, 0.2, seed=61)
    if name == "tet_p1":
        return mg.structured_tet(12, 1, 0.15, seed=62)
    if name == "tet_p3":
        return mg.structured_tet(5, 3, 0.15, seed=63)
    raise KeyError(name)


def whole(fm, k, u, prec, which=7):
    dt = torch.float64 if prec == "fp64" else torch.float32
    out = {c: torch.full((fm.nnz,), float("nan"), dtype=dt, device="cuda") for c in "MKT"}
    F.fem_form_elements(fm.h, k, u, PRECISIONS[prec], which, None)
    F.fem_sum_elements(fm.h, PRECISIONS[prec], out["M"] if which & 1 else None, out["K"] if which & 2 else None,
                       out["T"] if which & 4 else None, None)
    torch.cuda.synchronize()
    return out


@pytest.mark.parametrize("name", ["tri_p2", "tet_p1", "tet_p3"])
def test_plan_slot_ranges_are_the_completed_slots(name):
    m = mesh_of(name)
    fm = FemMesh.of(m)
    fm.symbolic()
    eb, sb = F.fem_chunk_plan(fm.h, F.FEM_TF32X3, 64 << 10, 64)
    E, nnz = m.n_elems, fm.nnz
    assert len(eb) == len(sb) >= 3
    assert eb[0] == 0 and eb[-1] == E and sb[0] == 0 and sb[-1] == nnz
    assert all(a < b for a, b in zip(eb, eb[1:])) and all(a <= b for a, b in zip(sb, sb[1:]))
    assert all(e % 128 == 0 for e in eb[:-1])
    # the largest contributing element of every slot, from the slot map
    slot = fm.slot_map().cpu().numpy().reshape(E, -1)
    maxe = np.full(nnz, -1, dtype=np.int64)
    np.maximum.at(maxe, slot.ravel(), np.repeat(np.arange(E), slot.shape[1]))
    for c in range(len(eb) - 1):
        ready = maxe[: sb[c + 1]]
        assert (ready < eb[c + 1]).all()                       # all contributors formed
        if sb[c + 1] < nnz:
            assert maxe[sb[c + 1]] >= eb[c + 1]                 # the prefix cannot grow


@pytest.mark.parametrize("prec", ["tf32x3", "fp32", "fp64", "bf16x3", "bf16x6"])
@pytest.mark.parametrize("name", ["tri_p2", "tet_p1", "tet_p3"])
@pytest.mark.parametrize("which", [7, 1, 6])
def test_ranges_equal_whole(prec, name, which):
    if prec.startswith("bf16") and name == "tet_p3":
        pytest.skip("no BF16 tile for P3 tetrahedra")
    m = mesh_of(name)
    fm = FemMesh.of(m)
    fm.symbolic()
    u = torch.tensor(mg.fourier_field(m.coords, 64), dtype=torch.float64, device="cuda")
    k = F.coeff("sin", (2.0, 1.0, 3.0))
    ref = whole(fm, k, u, prec, which)
    p = PRECISIONS[prec]
    eb, sb = F.fem_chunk_plan(fm.h, p, 32 << 10, 64)
    dt = torch.float64 if prec == "fp64" else torch.float32
    out = {c: torch.full((fm.nnz,), float("nan"), dtype=dt, device="cuda") for c in "MKT"}
    for c in range(len(eb) - 1):
        F.fem_form_elements_range(fm.h, k, u, p, which, eb[c], eb[c + 1], None)
        F.fem_sum_elements_range(fm.h, p, sb[c], sb[c + 1], out["M"] if which & 1 else None,
                                 out["K"] if which & 2 else None, out["T"] if which & 4 else None, None)
    torch.cuda.synchronize()
    F.fem_device_status()
    for i, c in enumerate("MKT"):
        if which & (1 << i):
            assert torch.equal(out[c], ref[c]), (prec, name, c)


@pytest.mark.parametrize("prec", ["tf32x3", "fp64"])
def test_default_plan_of_a_large_mesh(prec):
    """V of 400^2 x 2 P2 triangles is 100 MB (FP32): the default plan (48 MB
    ranges) splits it, and its ranges reproduce fem_assemble_all bit for bit."""
    m = mg.structured_tri(400, 2, 0.2, seed=65)
    fm = FemMesh.of(m)
    fm.symbolic()
    p = PRECISIONS[prec]
    eb, sb = F.fem_chunk_plan(fm.h, p, 0, 64)
    assert len(eb) - 1 >= 2
    u = torch.tensor(mg.fourier_field(m.coords, 66), dtype=torch.float64, device="cuda")
    k = F.coeff("poly", (1.0, 0.0, 1.0))
    ref = {c: v.clone() for c, v in fm.assemble(u, "poly", (1.0, 0.0, 1.0), prec).items()}
    dt = torch.float64 if prec == "fp64" else torch.float32
    out = {c: torch.full((fm.nnz,), float("nan"), dtype=dt, device="cuda") for c in "MKT"}
    for c in range(len(eb) - 1):
        F.fem_form_elements_range(fm.h, k, u, p, 7, eb[c], eb[c + 1], None)
        F.fem_sum_elements_range(fm.h, p, sb[c], sb[c + 1], out["M"], out["K"], out["T"], None)
    torch.cuda.synchronize()
    for c in "MKT":
        assert torch.equal(out[c], ref[c]), c


def test_range_errors():
    m = mesh_of("tri_p2")
    fm = FemMesh.of(m)
    fm.symbolic()
    u = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    k = F.coeff("poly", (1.0,))
    with pytest.raises(F.FemError) as ei:
        F.fem_form_elements_range(fm.h, k, u, F.FEM_TF32X3, 7, 64, 256, None)    # begin not a multiple of 128
    assert ei.value.code == F.FEM_EINVAL
    with pytest.raises(F.FemError) as ei:
        F.fem_form_elements_range(fm.h, k, u, F.FEM_TF32X3, 7, 128, m.n_elems + 1, None)
    assert ei.value.code == F.FEM_EINVAL
    F.fem_form_elements_range(fm.h, k, u, F.FEM_TF32X3, 1, 0, 128, None)
    with pytest.raises(F.FemError) as ei:                                          # other matrices than range 0
        F.fem_form_elements_range(fm.h, k, u, F.FEM_TF32X3, 7, 128, 256, None)
    assert ei.value.code == F.FEM_ESTATE
    out = torch.empty(fm.nnz, device="cuda")
    with pytest.raises(F.FemError) as ei:
        F.fem_sum_elements_range(fm.h, F.FEM_TF32X3, 0, fm.nnz + 1, out, None, None, None)
    assert ei.value.code == F.FEM_EINVAL


@pytest.mark.parametrize("name", ["tri_p2", "tet_p1", "fan"])
def test_sum_ranges_at_arbitrary_slots(name):
    """Slot ranges cut anywhere (inside long segments' neighbourhoods, one
    slot wide, empty) sum to the same bits as one whole sum: every slot's
    additions follow the fixed groups of 32 contributions, whatever range
    or launch covers it."""
    m = mg.fan_tri(300, seed=2) if name == "fan" else mesh_of(name)
    fm = FemMesh.of(m)
    fm.symbolic()
    u = torch.tensor(mg.fourier_field(m.coords, 67), dtype=torch.float64, device="cuda")
    k = F.coeff("poly", (1.0, 0.5, 0.25))
    ref = whole(fm, k, u, "tf32x3")
    nnz = fm.nnz
    rng = np.random.default_rng(68)
    cuts = sorted(set([0, nnz, 1, nnz - 1, nnz // 2, nnz // 2 + 1] + list(rng.integers(0, nnz, 9))))
    out = {c: torch.full((nnz,), float("nan"), device="cuda") for c in "MKT"}
    for a, b in zip(cuts, cuts[1:]):
        F.fem_sum_elements_range(fm.h, F.FEM_TF32X3, int(a), int(b), out["M"], out["K"], out["T"], None)
    F.fem_sum_elements_range(fm.h, F.FEM_TF32X3, 5, 5, out["M"], out["K"], out["T"], None)   # empty
    torch.cuda.synchronize()
    for c in "MKT":
        assert torch.equal(out[c], ref[c]), c
