"""GPU solve of the heat problem (Section 5 Newton step; Section 6,
Experiment 2) against the CPU oracle, through the C ABI.

  * fem_bicgstab on an Experiment-2 Jacobian: the solution of a sparse
    direct solve (scipy) within 1e-9 relative, bitwise repeatable;
  * fem_heat_step: a few implicit Euler steps from T = 0 agree with the
    oracle's steps (Newton with sparse direct solves) within 1e-9 of the
    temperature scale, and each GPU step balances the energy;
  * errors: host pointers, isoparametric meshes.
"""
import numpy as np
import pytest

import meshgen as mg
import oracle as orc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2204_03893_gb300 as F  # noqa: E402
from paper_2204_03893_gb300.torch_api import FemMesh  # noqa: E402

KLAW = ("pwlin", (0.0, 200.0, 1000.0, 1.5, 0.7, 0.5))
HC, HR, TA = 10.0, 0.8 * 5.670373e-8, 1000.0
GLAW = ("poly", (HC * TA + HR * TA ** 4, -HC, 0.0, 0.0, -HR))
RHOC = 1000.0 * 2400.0
DT = 10.0


def _mesh(N=8):
    m = mg.structured_tri(N, 2, 0.2, seed=91)
    return mg.Mesh(m.d, m.p, 0.2 * m.coords, m.conn)


def _dev(x):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


@pytest.mark.parametrize("N", [8, 100])
def test_bicgstab_against_direct_solve(N):
    """A small (n = 289) and a larger (n = 40 401) Experiment-2 system."""
    import scipy.sparse as sp
    import scipy.sparse.linalg as spl
    m = _mesh(N)
    o = orc.Oracle.of(m)
    u = 300.0 * mg.fourier_field(m.coords / 0.2, 92)
    r = o.assemble(u, mg.Coeff(*KLAW), m=RHOC, want_abs=False)
    bd = o.boundary(u, mg.Coeff(*GLAW))
    J = o.jacobian(r["M"], None, r["K"], r["T"], bd["B"], DT)
    rp, ci = o.pattern()
    rhs = mg.fourier_field(m.coords / 0.2, 93) - 0.5
    ref = spl.spsolve(sp.csr_matrix((J, ci, rp), shape=(m.n_nodes,) * 2).tocsc(), rhs)
    fm = FemMesh.of(m, mass=RHOC)
    fm.symbolic()
    xs = []
    for _ in range(2):
        x = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
        it, rr = F.fem_bicgstab(fm.h, _dev(J), _dev(rhs), x, 1e-14, 500)
        torch.cuda.synchronize()
        assert rr <= 1e-14 and it > 0
        xs.append(x.cpu().numpy())
    assert np.linalg.norm(xs[0] - ref) <= 1e-9 * np.linalg.norm(ref)
    assert np.array_equal(xs[0], xs[1])


def test_heat_steps_match_oracle_and_balance_energy():
    m = _mesh()
    o = orc.Oracle.of(m)
    fm = FemMesh.of(m, mass=RHOC)
    fm.symbolic()
    k, g = F.coeff(*KLAW), F.coeff(*GLAW)
    u_o = np.zeros(m.n_nodes)
    du = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    rp, ci = o.pattern()
    for step in range(5):
        dus = du.clone()
        rep = F.fem_heat_step(fm.h, k, g, None, DT, dus, du, 1e-12, 20, 1e-13, 1000)
        torch.cuda.synchronize()
        assert rep.converged == 1 and rep.newton_iters >= 1
        u_o, info = o.heat_step(mg.Coeff(*KLAW), mg.Coeff(*GLAW), u_o, DT, RHOC)
        ug = du.cpu().numpy()
        assert np.abs(ug - u_o).max() <= 1e-9 * TA, (step, np.abs(ug - u_o).max())
        # energy balance of the GPU step: sum M (u - u^s) = dt sum b(u)
        r = o.assemble(ug, mg.Coeff(*KLAW), m=RHOC, want_abs=False)
        M = orc.csr_to_dense(rp, ci, r["M"], m.n_nodes)
        b = o.boundary(ug, mg.Coeff(*GLAW))["b"]
        lhs, rhs = (M @ (ug - dus.cpu().numpy())).sum(), DT * b.sum()
        assert abs(lhs - rhs) <= 1e-8 * abs(rhs)


def test_heat_step_errors():
    m = _mesh(4)
    fm = FemMesh.of(m, mass=RHOC)
    fm.symbolic()
    k, g = F.coeff(*KLAW), F.coeff(*GLAW)
    host = np.zeros(m.n_nodes)
    with pytest.raises(F.FemError) as ei:
        F.fem_heat_step(fm.h, k, g, None, DT, host, host)
    assert ei.value.code == F.FEM_EINVAL
    du = torch.zeros(m.n_nodes, dtype=torch.float64, device="cuda")
    F.fem_mesh_set_isoparametric(fm.h, True)
    with pytest.raises(F.FemError) as ei:
        F.fem_heat_step(fm.h, k, g, None, DT, du.clone(), du)
    assert ei.value.code == F.FEM_EINVAL
