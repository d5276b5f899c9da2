"""GPU parity with an anisotropic conductivity tensor (fem_mesh_set_conductivity,
Section 7: A_e = B_e^-1 c B_e^-T, conductivity k(u) c) against the oracle
with the same tensor, through the C ABI: FEM_FP64 within 1e-12 * absum per
entry, FEM_TF32X3 / FEM_BF16X6 within 1e-6 relative Frobenius; resetting
to the identity restores the isotropic bits; batches read the same cache."""
import numpy as np
import pytest

import meshgen as mg
import oracle as orc
from fp64bar import check_fp64

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2204_03893_gb300 as F  # noqa: E402
from paper_2204_03893_gb300.torch_api import FemMesh  # noqa: E402

C2 = [[2.0, 0.6], [0.6, 0.8]]
C3 = [[2.0, 0.5, -0.3], [0.5, 1.2, 0.4], [-0.3, 0.4, 0.9]]
MESHES = {
    "tri_p1": lambda: mg.structured_tri(20, 1, 0.2, seed=101),
    "tri_p2": lambda: mg.structured_tri(17, 2, 0.2, seed=102),
    "tri_p3": lambda: mg.structured_tri(9, 3, 0.2, seed=103),
    "tet_p1": lambda: mg.structured_tet(6, 1, 0.15, seed=104),
    "tet_p2": lambda: mg.structured_tet(4, 2, 0.15, seed=105),
    "tet_p3": lambda: mg.structured_tet(5, 3, 0.15, seed=106),
}
LAW = mg.Coeff("sin", (2.0, 1.0, 3.0))


def frob(g, o):
    return np.linalg.norm(g - o) / np.linalg.norm(o)


@pytest.mark.parametrize("name", list(MESHES))
def test_anisotropic_parity(name):
    m = MESHES[name]()
    c = C2 if m.d == 2 else C3
    u = mg.fourier_field(m.coords, 107)
    o = orc.Oracle.of(m).set_conductivity(np.array(c)).assemble(u, LAW)
    fm = FemMesh.of(m).set_conductivity(c)
    du = torch.tensor(u, dtype=torch.float64, device="cuda")
    precs = ("fp64", "tf32x3") + (("bf16x6",) if name != "tet_p3" else ())
    for prec in precs:
        g = {k: v.double().cpu().numpy() for k, v in fm.assemble(du, LAW.kind, LAW.params, prec).items()}
        torch.cuda.synchronize()
        for k in ("M", "K", "T"):
            if prec == "fp64":
                check_fp64(g[k], o[k], o["abs" + k], (prec, k))
            else:
                assert frob(g[k], o[k]) <= 1e-6, (prec, k, frob(g[k], o[k]))
    F.fem_device_status()


def test_reset_restores_isotropic_bits_and_batches_follow():
    m = MESHES["tri_p2"]()
    u = torch.tensor(mg.fourier_field(m.coords, 108), dtype=torch.float64, device="cuda")
    iso = {k: v.clone() for k, v in FemMesh.of(m).assemble(u, LAW.kind, LAW.params, "tf32x3").items()}
    fm = FemMesh.of(m)
    fm.symbolic()
    b = F.fem_batch_create([fm.h], F.fem_batch_opts(F.FEM_TF32X3, 0, 1, 0))
    try:
        fm.set_conductivity(C2)
        an = {k: v.clone() for k, v in fm.assemble(u, LAW.kind, LAW.params, "tf32x3").items()}
        outs = {k: torch.full((fm.nnz,), float("nan"), device="cuda") for k in "MKT"}
        F.fem_batch_launch(b, [F.coeff(LAW.kind, LAW.params)], [u], [outs["M"]], [outs["K"]], [outs["T"]])
        torch.cuda.synchronize()
        for k in "MKT":
            assert torch.equal(outs[k], an[k]), k
        assert torch.equal(an["M"], iso["M"]) and not torch.equal(an["K"], iso["K"])
        fm.set_conductivity(None)
        back = fm.assemble(u, LAW.kind, LAW.params, "tf32x3")
        torch.cuda.synchronize()
        for k in "MKT":
            assert torch.equal(back[k], iso[k]), k
    finally:
        F.fem_batch_destroy(b)
    F.fem_device_status()


def test_invalid_tensors():
    m = MESHES["tet_p1"]()
    fm = FemMesh.of(m)
    for bad in ([[1.0, 0.2, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]],      # not symmetric
                [[1.0, 2.0, 0.0], [2.0, 1.0, 0.0], [0.0, 0.0, 1.0]],      # indefinite
                [[1.0, 0.0, 0.0], [0.0, float("nan"), 0.0], [0.0, 0.0, 1.0]]):
        with pytest.raises(F.FemError) as ei:
            fm.set_conductivity(bad)
        assert ei.value.code == F.FEM_EINVAL
