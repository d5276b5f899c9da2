"""Batched reassembly (one CUDA graph of persistent kernels over many meshes)
against the same meshes reassembled one by one, through the C ABI.

The batch must give bit-identical CSR values to single-mesh calls with the
same precision (the per-slot summation order and the element products are
the same code), for every element type, for ragged mesh sizes, with and
without the launch-shape tuner, and across graph replays with new inputs.
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
from paper_2204_03893_gb300.torch_api import PRECISIONS, FemMesh  # noqa: E402


def mixed_meshes():
    """One mesh of every element type, sizes with ragged last tiles."""
    out = []
    for i, (d, p, N) in enumerate([(2, 1, 23), (2, 2, 17), (2, 3, 9), (3, 1, 7), (3, 2, 4), (3, 3, 3)]):
        m = mg.structured_tri(N, p, 0.2, seed=10 + i) if d == 2 else mg.structured_tet(N, p, 0.15, seed=10 + i)
        u = mg.fourier_field(m.coords, 20 + i)
        a, b = 0.2 + 0.1 * i, 0.5 - 0.05 * i
        out.append(mg.Workload(f"mix{i}", m, u, mg.Coeff("poly", (1.0, a, b, 0.0, 0.0))))
    return out


def single(fm, wl, prec, u=None):
    uu = torch.tensor(wl.u if u is None else u, dtype=torch.float64, device="cuda")
    return {k: v.clone() for k, v in fm.assemble(uu, wl.coeff.kind, wl.coeff.params, prec).items()}


def run_batch(batch, fms, wls, prec, us=None, which="MKT"):
    dt = torch.float64 if prec == "fp64" else torch.float32
    outs = [{k: torch.full((fm.nnz,), float("nan"), dtype=dt, device="cuda") for k in "MKT"} for fm in fms]
    uu = [torch.tensor(wl.u if us is None else us[i], dtype=torch.float64, device="cuda") for i, wl in enumerate(wls)]
    ks = [F.coeff(wl.coeff.kind, wl.coeff.params) for wl in wls]
    F.fem_batch_launch(batch, ks, uu, [o["M"] if "M" in which else None for o in outs],
                       [o["K"] if "K" in which else None for o in outs],
                       [o["T"] if "T" in which else None for o in outs])
    torch.cuda.synchronize()
    F.fem_device_status()
    return outs


@pytest.mark.parametrize("prec", ["tf32x3", "fp64", "fp32"])
@pytest.mark.parametrize("tune", [0, 1])
def test_batch_equals_single_meshes(prec, tune):
    wls = mixed_meshes()
    fms = [FemMesh.of(w.mesh) for w in wls]
    for fm in fms:
        fm.symbolic()
    # references first: single-mesh calls with the same precision
    refs = [single(fm, wl, prec) for fm, wl in zip(fms, wls)]
    opts = F.fem_batch_opts(PRECISIONS[prec], tune, 1, 0)
    b = F.fem_batch_create([fm.h for fm in fms], opts)
    try:
        for rep in range(2):
            outs = run_batch(b, fms, wls, prec)
            for i, (o, r) in enumerate(zip(outs, refs)):
                for k in "MKT":
                    assert torch.equal(o[k], r[k]), (prec, tune, rep, i, k)
        info = F.fem_batch_get_info(b)
        assert info.n_meshes == 6 and info.graph == 1 and info.tuned == tune
        # one tensor-core launch per type (P3 tetrahedra: the chunked kernel), one
        # SIMT walker otherwise, and one CSR-sum launch per n_p present (3, 4, 6, 10, 20)
        expect = {"tf32x3": 6 + 5, "fp32": 1 + 5, "fp64": 1 + 5}[prec]
        assert info.kernels_per_launch == expect
    finally:
        F.fem_batch_destroy(b)


def test_batch_accuracy_against_oracle():
    wls = mixed_meshes()
    fms = [FemMesh.of(w.mesh) for w in wls]
    for fm in fms:
        fm.symbolic()
    b = F.fem_batch_create([fm.h for fm in fms], F.fem_batch_opts(F.FEM_TF32X3, 0, 1, 0))
    try:
        outs = run_batch(b, fms, wls, "tf32x3")
    finally:
        F.fem_batch_destroy(b)
    for o, wl in zip(outs, wls):
        r = orc.Oracle.of(wl.mesh).assemble(wl.u, wl.coeff)
        for k in "MKT":
            g = o[k].double().cpu().numpy()
            assert np.linalg.norm(g - r[k]) <= 1e-6 * np.linalg.norm(r[k]), (wl.name, k)


def test_batch_new_inputs_and_partial_requests():
    """Replays with a new u per mesh, and M only for some meshes."""
    wls = mixed_meshes()[:4]
    fms = [FemMesh.of(w.mesh) for w in wls]
    for fm in fms:
        fm.symbolic()
    b = F.fem_batch_create([fm.h for fm in fms], F.fem_batch_opts(F.FEM_TF32X3, 0, 1, 0))
    try:
        for s in range(3):
            us = [mg.fourier_field(w.mesh.coords, 100 + 7 * s + i) for i, w in enumerate(wls)]
            outs = run_batch(b, fms, wls, "tf32x3", us=us)
            for i, (fm, wl) in enumerate(zip(fms, wls)):
                r = single(fm, wl, "tf32x3", u=us[i])
                for k in "MKT":
                    assert torch.equal(outs[i][k], r[k]), (s, i, k)
        outs = run_batch(b, fms, wls, "tf32x3", which="M")
        for i, (fm, wl) in enumerate(zip(fms, wls)):
            r = single(fm, wl, "tf32x3")
            assert torch.equal(outs[i]["M"], r["M"])
            assert torch.isnan(outs[i]["K"]).all()       # not requested: untouched
    finally:
        F.fem_batch_destroy(b)


def test_batch_errors():
    m = mg.structured_tri(4, 1)
    fm = FemMesh.of(m)
    with pytest.raises(F.FemError) as ei:
        F.fem_batch_create([fm.h])
    assert ei.value.code == F.FEM_ESTATE
    fm.symbolic()
    b = F.fem_batch_create([fm.h])
    try:
        out = torch.empty(fm.nnz, device="cuda")
        with pytest.raises(F.FemError) as ei:
            F.fem_batch_launch(b, None, None, None, [out], None)
        assert ei.value.code == F.FEM_EINVAL
    finally:
        F.fem_batch_destroy(b)
