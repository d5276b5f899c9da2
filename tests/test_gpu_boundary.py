"""GPU parity of the boundary terms and the Newton step (Section 5; Section 6,
Experiment 2) against the CPU oracle, through the C ABI.

  * boundary facets: the same (element, face) list as the oracle, bit for bit;
  * B(u) and the boundary load b(u): |gpu - oracle| <= 1e-12 absum per entry
    (the FP64 bar of tests/fp64bar.py);
  * residual F = M (u - u^s) + dt K u - dt b from the GPU's own M, K, b: the
    same bar against the oracle's residual of the oracle's matrices, with the
    error scale of the matrices carried through; ||F||_2 and ||F||_inf within
    1e-12 relative of the oracle's F, and bitwise repeatable;
  * Jacobian Mt + M + dt (K + T) - dt B likewise;
  * y = A x against a dense product, and at full size (12.6 million
    tetrahedra) the facet count 12 N^2, the boundary total
    sum B = g' |dOmega| and vanishing interior residual rows for a linear u.
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

EXP2 = ("poly", (10.0 * 1000.0 + 0.8 * 5.670373e-8 * 1000.0 ** 4, -10.0, 0.0, 0.0, -0.8 * 5.670373e-8))
KLAW = ("poly", (1.5, -0.004, 3e-6))
DT = 10.0
MASS = 2.4e6   # c rho of Experiment 2

MESHES = {
    "tri_p1": lambda: mg.structured_tri(9, 1, 0.2, seed=51),
    "tri_p2": lambda: mg.structured_tri(7, 2, 0.2, seed=52),
    "tri_p3": lambda: mg.structured_tri(5, 3, 0.2, seed=53),
    "tet_p1": lambda: mg.structured_tet(5, 1, 0.15, seed=54),
    "tet_p2": lambda: mg.structured_tet(3, 2, 0.15, seed=55),
    "tet_p3": lambda: mg.structured_tet(2, 3, 0.15, seed=56),
}


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def _mesh(name, mass=1.0):
    m = MESHES[name]()
    fm = FemMesh.of(m, mass=mass)
    fm.symbolic()
    return m, fm


@pytest.mark.parametrize("name", list(MESHES))
def test_boundary_facets_match_oracle(name):
    m, fm = _mesh(name)
    nb = F.fem_boundary_facets(fm.h)
    fe = torch.empty(max(nb, 1), dtype=torch.int32, device="cuda")
    ff = torch.empty_like(fe)
    F.fem_get_boundary_facets(fm.h, fe, ff)
    torch.cuda.synchronize()
    oe, of = orc.Oracle.of(m).boundary_facets()
    assert nb == len(oe)
    assert np.array_equal(fe[:nb].cpu().numpy(), oe) and np.array_equal(ff[:nb].cpu().numpy(), of)


@pytest.mark.parametrize("name", list(MESHES))
def test_boundary_matrix_and_load(name):
    m, fm = _mesh(name)
    u = 600.0 * mg.fourier_field(m.coords, 57)
    ref = orc.Oracle.of(m).boundary(u, mg.Coeff(*EXP2))
    vB = torch.full((fm.nnz,), np.nan, dtype=torch.float64, device="cuda")
    b = torch.full((m.n_nodes,), np.nan, dtype=torch.float64, device="cuda")
    g = F.coeff(*EXP2)
    F.fem_assemble_boundary(fm.h, g, _dev(u), None, vB, b)
    torch.cuda.synchronize()
    check_fp64(vB.cpu().numpy(), ref["B"], ref["absB"], "B")
    check_fp64(b.cpu().numpy(), ref["b"], ref["absb"], "b")
    # all facets selected by the mask = no mask, bit for bit; no facet: zero
    vB2, b2 = torch.empty_like(vB), torch.empty_like(b)
    nb = F.fem_boundary_facets(fm.h)
    ones = torch.ones(nb, dtype=torch.uint8, device="cuda")
    F.fem_assemble_boundary(fm.h, g, _dev(u), ones, vB2, b2)
    torch.cuda.synchronize()
    assert torch.equal(vB, vB2) and torch.equal(b, b2)
    F.fem_assemble_boundary(fm.h, g, _dev(u), torch.zeros_like(ones), vB2, b2)
    torch.cuda.synchronize()
    assert not vB2.any() and not b2.any()


@pytest.mark.parametrize("name", ["tri_p1", "tri_p2", "tet_p1", "tet_p2", "tri_p3", "tet_p3"])
def test_residual_and_jacobian(name):
    m, fm = _mesh(name, mass=MASS)
    o = orc.Oracle.of(m)
    us = 400.0 * mg.fourier_field(m.coords, 58)
    u = us + 30.0 * mg.fourier_field(m.coords, 59)
    klaw = mg.Coeff(*KLAW)
    r = o.assemble(u, klaw, m=MASS)
    rb = o.boundary(u, mg.Coeff(*EXP2))
    oF, aF_terms = o.residual(r["M"], r["K"], rb["b"], u, us, DT)
    # error scale of F: the residual of the matrices' and load's scales
    aF, _ = o.residual(r["absM"], r["absK"], -rb["absb"], np.abs(u), -np.abs(us), DT)
    oJ = o.jacobian(r["M"], None, r["K"], r["T"], rb["B"], DT)
    aJ = o.jacobian(r["absM"], None, r["absK"], r["absT"], -rb["absB"], DT)

    du, dus = _dev(u), _dev(us)
    g = fm.assemble(du, klaw.kind, klaw.params, "fp64")
    vB = torch.empty(fm.nnz, dtype=torch.float64, device="cuda")
    b = torch.empty(m.n_nodes, dtype=torch.float64, device="cuda")
    F.fem_assemble_boundary(fm.h, F.coeff(*EXP2), du, None, vB, b)
    Fv = torch.empty(m.n_nodes, dtype=torch.float64, device="cuda")
    norms = torch.empty(2, dtype=torch.float64, device="cuda")
    F.fem_residual(fm.h, g["M"], g["K"], b, du, dus, DT, Fv, norms)
    J = torch.empty(fm.nnz, dtype=torch.float64, device="cuda")
    F.fem_jacobian(fm.h, DT, g["M"], None, g["K"], g["T"], vB, J)
    torch.cuda.synchronize()
    check_fp64(Fv.cpu().numpy(), oF, aF + aF_terms, "F")
    check_fp64(J.cpu().numpy(), oJ, aJ, "J")
    n2, ninf = norms.cpu().numpy()
    assert abs(n2 - np.linalg.norm(oF)) <= 1e-12 * np.linalg.norm(aF + aF_terms)
    assert abs(ninf - np.abs(oF).max()) <= 1e-12 * np.abs(aF + aF_terms).max()
    norms2 = torch.empty_like(norms)
    F.fem_residual(fm.h, g["M"], g["K"], b, du, dus, DT, Fv, norms2)
    torch.cuda.synchronize()
    assert torch.equal(norms, norms2)


def test_spmv_against_dense():
    m, fm = _mesh("tri_p2")
    rp, ci = (t.cpu().numpy() for t in fm.pattern())
    rng = np.random.default_rng(60)
    vals, x, y0 = rng.standard_normal(fm.nnz), rng.standard_normal(m.n_nodes), rng.standard_normal(m.n_nodes)
    A = orc.csr_to_dense(rp, ci, vals, m.n_nodes)
    y = _dev(y0)
    F.fem_csr_spmv(fm.h, _dev(vals), 2.0, _dev(x), -0.5, y)
    torch.cuda.synchronize()
    ref = 2.0 * (A @ x) - 0.5 * y0
    assert np.abs(y.cpu().numpy() - ref).max() <= 1e-13 * (2 * np.abs(A) @ np.abs(x) + np.abs(y0)).max()


def test_errors():
    m, fm = _mesh("tri_p1")
    host = np.zeros(m.n_nodes)
    with pytest.raises(F.FemError) as ei:
        F.fem_assemble_boundary(fm.h, F.coeff(*EXP2), host, None, None, _dev(host))
    assert ei.value.code == F.FEM_EINVAL
    fresh = FemMesh.of(m)
    with pytest.raises(F.FemError) as ei:
        F.fem_boundary_facets(fresh.h)
    assert ei.value.code == F.FEM_ESTATE


def test_full_size_tet_p1_128_newton_step():
    """The 12 582 912-tetrahedron mesh: 12 N^2 boundary triangles, the
    boundary total sum B = g' |dOmega| = 6 g' for g = 2 - 3u, and interior
    residual rows that vanish for a linear u = u^s with constant k and no
    boundary term."""
    wl = mg.workload("tet_p1_128")
    N = 128
    fm = FemMesh.of(wl.mesh)
    fm.symbolic()
    assert F.fem_boundary_facets(fm.h) == 12 * N * N
    u = _dev(0.2 + wl.mesh.coords @ np.array([0.3, -1.1, 0.7]))
    vB = torch.empty(fm.nnz, dtype=torch.float64, device="cuda")
    F.fem_assemble_boundary(fm.h, F.coeff("poly", (2.0, -3.0)), u, None, vB, None)
    torch.cuda.synchronize()
    assert abs(vB.sum().item() - (-3.0) * 6.0) <= 1e-11 * 18.0
    g = fm.assemble(u, "poly", (2.0,), "fp64")
    Fv = torch.empty_like(u)
    norms = torch.empty(2, dtype=torch.float64, device="cuda")
    F.fem_residual(fm.h, g["M"], g["K"], None, u, u, DT, Fv, norms)
    torch.cuda.synchronize()
    X = wl.mesh.coords
    interior = torch.tensor(np.all((X > 1e-9) & (X < 1 - 1e-9), axis=1), device="cuda")
    scale = DT * 2.0 * 3 * (0.3 ** 2 + 1.1 ** 2 + 0.7 ** 2) ** 0.5 / N   # |K_ij u_j| ~ k |grad u| h
    assert Fv[interior].abs().max().item() <= 1e-9 * scale
    assert Fv[~interior].abs().max().item() > 1e-4 * scale   # boundary rows carry the flux
