"""GPU parity of the per-quadrature-point geometry (Section 7: isoparametric
mappings, conductivity tensors per point) against the CPU oracle, through
the C ABI.

  * curved meshes (meshgen.curved) mapped isoparametrically, a varying
    conductivity field, and both together: FEM_FP64 within the FP64 bar of
    tests/fp64bar.py per entry, FEM_FP32 within 1e-5 relative Frobenius, on
    six element types; the u-dependent mass likewise;
  * switching the mapping off restores the affine results bit for bit, and
    the allocation-free FP64 call gives the same bits as fem_assemble_all;
  * the paths that do not read per-point geometry refuse such meshes.
"""
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

CASES = [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2), (3, 3)]
LAW = mg.Coeff("poly", (1.0, 0.6, 0.3))


def _mesh(d, p, seed=71):
    m = mg.structured_tri(9, p, 0.2, seed=seed) if d == 2 else mg.structured_tet(3, p, 0.15, seed=seed)
    return mg.curved(m, 0.05, seed=seed + 1)


def _field(m, phi):
    """A conductivity field c(x) evaluated at the physical quadrature points
    x_q = sum_i x_i phi_i(xhat_q) of a rule (phi: (n_q, n_p) basis values at
    its points): the oracle's rule for the oracle, the library's rule (its
    points and their order are the library's own) for the library."""
    X = np.einsum("qi,eid->eqd", phi, m.coords[m.conn])          # physical points
    d = m.d
    cf = np.zeros(X.shape[:2] + (d, d))
    for i in range(d):
        cf[..., i, i] = 1.0 + 0.5 * i + 0.3 * np.sin(3 * X[..., i])
    cf[..., 0, 1] = cf[..., 1, 0] = 0.2 * X[..., 1]
    return cf


def _gpu(fm, u, prec):
    du = torch.tensor(u, dtype=torch.float64, device="cuda")
    g = fm.assemble(du, LAW.kind, LAW.params, prec)
    torch.cuda.synchronize()
    F.fem_device_status()
    return {k: v.double().cpu().numpy() for k, v in g.items()}


@pytest.mark.parametrize("mode", ["iso", "field", "both"])
@pytest.mark.parametrize("d,p", CASES)
def test_per_point_parity(d, p, mode):
    m = _mesh(d, p)
    u = mg.fourier_field(m.coords, 73)
    o = orc.Oracle.of(m)
    fm = FemMesh.of(m)
    fm.symbolic()
    if mode in ("iso", "both"):
        o.set_isoparametric(True)
        F.fem_mesh_set_isoparametric(fm.h, True)
    if mode in ("field", "both"):
        xo, _ = orc.rule(m.d, 2 * m.p)
        o.set_conductivity_field(_field(m, np.array([orc.basis(m.d, m.p, x)[0] for x in xo])))
        F.fem_mesh_set_conductivity_field(fm.h, _field(m, F.fem_reference_tables(m.d, m.p)[2]))
    ref = o.assemble(u, LAW)
    g64 = _gpu(fm, u, "fp64")
    for k in ("M", "K", "T"):
        check_fp64(g64[k], ref[k], ref["abs" + k], (mode, k))
    g32 = _gpu(fm, u, "fp32")
    for k in ("M", "K", "T"):
        assert np.linalg.norm(g32[k] - ref[k]) <= 1e-5 * np.linalg.norm(ref[k]), (mode, k)


@pytest.mark.parametrize("d,p", [(2, 2), (3, 2)])
def test_per_point_mass_u(d, p):
    m = _mesh(d, p)
    u, us = mg.fourier_field(m.coords, 74), mg.fourier_field(m.coords, 75)
    mk = mg.Coeff("poly", (1.0, 0.5, 0.25))
    ref = orc.Oracle.of(m).set_isoparametric(True).assemble_mass_u(u, us, mk)
    fm = FemMesh.of(m)
    fm.symbolic()
    F.fem_mesh_set_isoparametric(fm.h, True)
    du, dus = (torch.tensor(x, dtype=torch.float64, device="cuda") for x in (u, us))
    g = {k: v.cpu().numpy() for k, v in fm.assemble_mass_u(du, dus, mk.kind, mk.params, "fp64").items()}
    for k in ("Mu", "Mt"):
        check_fp64(g[k], ref[k], ref["abs" + k], k, rel_factor=10.0)


def test_switching_off_restores_affine_bits_and_noalloc_agrees():
    m = _mesh(3, 2)
    u = mg.fourier_field(m.coords, 76)
    fm = FemMesh.of(m)
    fm.symbolic()
    affine = _gpu(fm, u, "fp64")
    F.fem_mesh_set_isoparametric(fm.h, True)
    curved = _gpu(fm, u, "fp64")
    assert any(not np.array_equal(curved[k], affine[k]) for k in "MKT")
    du = torch.tensor(u, dtype=torch.float64, device="cuda")
    out = {k: torch.empty(fm.nnz, dtype=torch.float64, device="cuda") for k in "MKT"}
    F.fem_assemble_all_noalloc(fm.h, F.coeff(LAW.kind, LAW.params), du, out["M"], out["K"], out["T"])
    torch.cuda.synchronize()
    for k in "MKT":
        assert np.array_equal(out[k].cpu().numpy(), curved[k]), k
    F.fem_mesh_set_isoparametric(fm.h, False)
    again = _gpu(fm, u, "fp64")
    for k in "MKT":
        assert np.array_equal(again[k], affine[k]), k


def test_paths_without_per_point_geometry_refuse():
    m = _mesh(2, 2)
    fm = FemMesh.of(m)
    fm.symbolic()
    F.fem_mesh_set_isoparametric(fm.h, True)
    du = torch.tensor(mg.fourier_field(m.coords, 77), dtype=torch.float64, device="cuda")
    for prec in ("tf32x3", "bf16x6"):
        with pytest.raises(F.FemError) as ei:
            fm.assemble(du, LAW.kind, LAW.params, prec)
        assert ei.value.code == F.FEM_EINVAL
    with pytest.raises(F.FemError) as ei:
        F.fem_batch_create([fm.h], F.fem_batch_opts(F.FEM_FP64, 0, 1, 0))
    assert ei.value.code == F.FEM_EINVAL
    vB = torch.empty(fm.nnz, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FemError) as ei:
        F.fem_assemble_boundary(fm.h, F.coeff("poly", (1.0, 2.0)), du, None, vB, None)
    assert ei.value.code == F.FEM_EINVAL
