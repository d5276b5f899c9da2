"""Host-side checks of libfem that need no GPU: the library builds and loads,
exports every symbol include/fem.h declares, validates arguments before any
device work, and its reference tables (quadrature + Lagrange basis, derived
by its own construction) satisfy the same pins as the oracle's."""
import ctypes as C
import itertools
import math
import os
import re

import numpy as np
import pytest

import meshgen as mg
import oracle as orc

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def fem():
    from paper_2204_03893_gb300 import build
    build.build()
    import paper_2204_03893_gb300 as F
    return F


def header_functions():
    src = open(os.path.join(ROOT, "include", "fem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fem_[a-z_0-9]+)\s*\(", src)))


def test_exports_every_declared_symbol(fem):
    names = header_functions()
    assert len(names) >= 15
    L = C.CDLL(fem.library_path())
    for n in names:
        assert hasattr(L, n), n
    assert "sm_103a" in fem.fem_version()


def test_binding_names_match_header(fem):
    for n in header_functions():
        assert hasattr(fem, n), n


@pytest.mark.parametrize("d,deg,nq", [(2, 2, 3), (2, 4, 6), (2, 6, 12), (3, 2, 4), (3, 4, 11), (3, 6, 24)])
def test_library_rules_exact(fem, d, deg, nq):
    xq, wq, phi, grad = fem.fem_reference_tables(d, deg // 2)
    assert len(wq) == nq
    for alpha in itertools.product(range(deg + 1), repeat=d):
        if sum(alpha) > deg:
            continue
        q = np.sum(wq * np.prod(xq ** np.array(alpha), axis=1))
        ex = math.prod(math.factorial(a) for a in alpha) / math.factorial(sum(alpha) + d)
        assert abs(q - ex) < 1e-15
    # same rule as the oracle's (as a point set, up to order): compare sorted weights
    # and the integrals of random smooth functions
    xo, wo = orc.rule(d, deg)
    np.testing.assert_allclose(np.sort(wq), np.sort(wo), rtol=0, atol=1e-14)
    rng = np.random.default_rng(0)
    for _ in range(5):
        a = rng.normal(size=d)
        f = lambda x: np.exp(x @ a)
        assert abs(np.sum(wq * f(xq)) - np.sum(wo * f(xo))) < 1e-14


@pytest.mark.parametrize("d,p", [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2), (3, 3)])
def test_library_basis_matches_oracle(fem, d, p):
    xq, wq, phi, grad = fem.fem_reference_tables(d, p)
    for q in range(len(wq)):
        po, go = orc.basis(d, p, xq[q])
        np.testing.assert_allclose(phi[q], po, atol=1e-13)
        np.testing.assert_allclose(grad[q], go, atol=1e-12)
    assert np.abs(phi.sum(1) - 1).max() < 1e-13
    assert np.abs(grad.sum(1)).max() < 1e-12


def test_argument_validation_without_device(fem):
    desc = fem.fem_mesh_desc()
    desc.dim, desc.order, desc.n_nodes, desc.n_elems = 4, 1, 3, 1
    with pytest.raises(fem.FemError) as ei:
        fem.fem_mesh_create(desc)
    assert ei.value.code == fem.FEM_EINVAL
    desc.dim, desc.order, desc.qdeg = 2, 1, 5
    with pytest.raises(fem.FemError) as ei:
        fem.fem_mesh_create(desc)
    assert ei.value.code == fem.FEM_EINVAL
    with pytest.raises(fem.FemError):
        fem.fem_reference_tables(2, 4)
    al = fem.fem_allocator()
    with pytest.raises(fem.FemError):
        fem.fem_set_allocator(al)          # NULL callbacks refused
    fem.fem_set_allocator(None)


def test_no_device_reports_cuda_error(fem):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    m = mg.structured_tri(2, 1)
    from paper_2204_03893_gb300.torch_api import FemMesh
    with pytest.raises(fem.FemError) as ei:
        FemMesh.of(m)
    assert ei.value.code in (fem.FEM_ECUDA, fem.FEM_ENOMEM)
