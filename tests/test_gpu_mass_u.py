"""GPU parity of the u-dependent mass M(u) and the mass-tensor term
Mt = (mass tensor) o_2 (u - us) (fem_assemble_mass_u) against the oracle,
through the C ABI.  Bars: FEM_FP64 |gpu - oracle| <= 1e-12 * absum per
entry (absum: the oracle's sum of the magnitudes of the expanded terms);
FEM_FP32 relative Frobenius error <= 1e-5 and FEM_TF32X3 (tcgen05 tile,
P1-P3 triangles, P1-P2 tetrahedra) <= 1e-6 per matrix; repeatable bits."""
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

MESHES = {
    "tri_p1": lambda: mg.structured_tri(20, 1, 0.2, seed=51),     # 800 elements (ragged last tile)
    "tri_p2": lambda: mg.structured_tri(17, 2, 0.2, seed=52),
    "tri_p3": lambda: mg.structured_tri(9, 3, 0.2, seed=53),
    "tet_p1": lambda: mg.structured_tet(6, 1, 0.15, seed=54),
    "tet_p2": lambda: mg.structured_tet(4, 2, 0.15, seed=55),
    "tet_p3": lambda: mg.structured_tet(3, 3, 0.15, seed=56),
}
LAWS = [("poly", (1.0, 0.5, 0.25)), ("sin", (2.0, 1.0, 3.0)), ("pwlin", (0.0, 0.4, 1.0, 1.0, 2.0, 1.5))]


def fields(m, seed):
    u = mg.fourier_field(m.coords, seed)
    us = u - 0.05 * np.random.default_rng(seed).standard_normal(m.n_nodes)
    return u, us


def frob(g, o):
    return np.linalg.norm(g - o) / np.linalg.norm(o)


@pytest.mark.parametrize("law", range(3))
@pytest.mark.parametrize("name", list(MESHES))
def test_mass_u_parity(name, law):
    m = MESHES[name]()
    kind, params = LAWS[law]
    u, us = fields(m, 60 + law)
    o = orc.Oracle.of(m).assemble_mass_u(u, us, mg.Coeff(kind, params))
    fm = FemMesh.of(m)
    du, dus = (torch.tensor(x, dtype=torch.float64, device="cuda") for x in (u, us))
    g64 = {k: v.cpu().numpy() for k, v in fm.assemble_mass_u(du, dus, kind, params, "fp64").items()}
    g32 = {k: v.double().cpu().numpy() for k, v in fm.assemble_mass_u(du, dus, kind, params, "fp32").items()}
    if name == "tet_p3":
        with pytest.raises(F.FemError) as ei:                   # no tensor-core tile for P3 tetrahedra
            fm.assemble_mass_u(du, dus, kind, params, "tf32x3")
        assert ei.value.code == F.FEM_EINVAL
        gtc = None
    else:
        gtc = {k: v.double().cpu().numpy() for k, v in fm.assemble_mass_u(du, dus, kind, params, "tf32x3").items()}
    torch.cuda.synchronize()
    F.fem_device_status()
    for k in ("Mu", "Mt"):
        check_fp64(g64[k], o[k], o["abs" + k], k, rel_factor=10.0)
        assert frob(g32[k], o[k]) <= 1e-5, (k, frob(g32[k], o[k]))
        if gtc is not None:
            assert frob(gtc[k], o[k]) <= 1e-6, ("tf32x3", k, frob(gtc[k], o[k]))


@pytest.mark.parametrize("prec", ["fp32", "tf32x3"])
def test_mass_u_single_output_and_repeatable(prec):
    m = MESHES["tri_p2"]()
    u, us = fields(m, 70)
    fm = FemMesh.of(m)
    du, dus = (torch.tensor(x, dtype=torch.float64, device="cuda") for x in (u, us))
    both = {k: v.clone() for k, v in fm.assemble_mass_u(du, dus, "poly", (1.0, 0.5), prec).items()}
    only = fm.assemble_mass_u(du, None, "poly", (1.0, 0.5), prec, which=("Mu",))
    assert torch.equal(only["Mu"], both["Mu"])
    for _ in range(3):
        again = fm.assemble_mass_u(du, dus, "poly", (1.0, 0.5), prec)
        for k in both:
            assert torch.equal(again[k], both[k]), k
    torch.cuda.synchronize()
    F.fem_device_status()


def test_mass_u_errors_and_scratch_state():
    m = MESHES["tri_p1"]()
    u, us = fields(m, 71)
    fm = FemMesh.of(m)
    fm.symbolic()
    du, dus = (torch.tensor(x, dtype=torch.float64, device="cuda") for x in (u, us))
    out = torch.empty(fm.nnz, dtype=torch.float64, device="cuda")
    k = F.coeff("poly", (1.0, 0.5))
    with pytest.raises(F.FemError) as ei:                                   # BF16 splits
        F.fem_assemble_mass_u(fm.h, k, du, dus, F.FEM_BF16X3, out, None, None)
    assert ei.value.code == F.FEM_EINVAL
    with pytest.raises(F.FemError) as ei:                                   # Mt without u^s
        F.fem_assemble_mass_u(fm.h, k, du, None, F.FEM_FP64, None, out, None)
    assert ei.value.code == F.FEM_EINVAL
    host = np.zeros(fm.nnz)
    with pytest.raises(F.FemError) as ei:                                   # host output
        F.fem_assemble_mass_u(fm.h, k, du, dus, F.FEM_FP64, host, None, None)
    assert ei.value.code == F.FEM_EINVAL
    # formed matrices are gone once the scratch served the mass-u call
    F.fem_form_elements(fm.h, k, du, F.FEM_FP64, 7, None)
    F.fem_assemble_mass_u(fm.h, k, du, dus, F.FEM_FP64, out, None, None)
    with pytest.raises(F.FemError) as ei:
        F.fem_sum_elements(fm.h, F.FEM_FP64, out, None, None, None)
    assert ei.value.code == F.FEM_ESTATE
    # and the usual path still agrees with the oracle afterwards
    r = orc.Oracle.of(m).assemble(u, mg.Coeff("poly", (1.0, 0.5)))
    g = fm.assemble(du, "poly", (1.0, 0.5), "fp64")
    torch.cuda.synchronize()
    for c in ("M", "K", "T"):
        assert (np.abs(g[c].cpu().numpy() - r[c]) <= 1e-12 * r["abs" + c] + 1e-300).all(), c
    F.fem_device_status()
