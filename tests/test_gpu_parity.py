"""GPU parity of libfem against the CPU FP64 oracle, through the C ABI.

Bars (per matrix M, K(u), T(u)):
  * pattern (row_ptr, col_idx) and slot map: bit-exact;
  * FEM_FP64: |gpu - oracle| <= 1e-12 * absum per entry, absum = the
    oracle's sum of the magnitudes of the expanded quadrature terms of the
    slot (entries that cancel are judged against the size of what cancelled),
    and the plain relative error |gpu - oracle| / |oracle| <= 1e-12 where
    |oracle| >= 0.1 absum, <= 1e-10 where |oracle| >= 1e-3 absum;
  * FEM_TF32X3: relative Frobenius error <= 1e-6 per matrix;
  * FEM_FP32 (SIMT reference point): relative Frobenius error <= 1e-5;
  * FEM_BF16X6: relative Frobenius error <= 1e-6 (three BF16 parts carry
    the 24 bits of an FP32 value; the dropped products are of order 2^-24);
  * FEM_BF16X3: relative Frobenius error <= 2e-4: two parts leave each
    operand within 2^-16 of its value and drop x1 q1, so a product term is
    within about 3 * 2^-16 = 4.6e-5 of |x||q|, and the sums over the
    quadrature points (signed terms in K and T) lose up to a small factor
    more relative to the entry;
  * every precision: bitwise identical results run to run.
Sizes span several 128-element tiles with a ragged last tile.
"""
import math

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
from paper_2204_03893_gb300.torch_api import PRECISIONS, FemMesh  # noqa: E402

TF32_TOL = 1e-6
FP32_TOL = 1e-5
BF16X6_TOL = 1e-6
BF16X3_TOL = 2e-4
BF_TOL = {"bf16x3": BF16X3_TOL, "bf16x6": BF16X6_TOL}


def wl_small(name):
    return {
        "tri_p1": lambda: mg.workload("tri_p1_64"),
        "tri_p2": lambda: mg.workload("tri_p2_1024", scale=41),
        "tet_p1": lambda: mg.workload("tet_p1_128", scale=9),
        "tet_p2": lambda: mg.workload("tet_p2_64", scale=5),
        "tri_p3": lambda: _p3(2),
        "tet_p3": lambda: _p3(3),
    }[name]()


def _p3(d):
    m = mg.structured_tri(13, 3, 0.2, seed=77) if d == 2 else mg.structured_tet(3, 3, 0.15, seed=77)
    return mg.Workload(f"p3_{d}", m, mg.fourier_field(m.coords, 78), mg.Coeff("poly", (1.0, 0.3, 0.6, 0.0, 0.0)))


def gpu_assemble(fm, wl, prec):
    u = torch.tensor(wl.u, dtype=torch.float64, device="cuda")   # u is FP64 in every precision
    out = fm.assemble(u, wl.coeff.kind, wl.coeff.params, prec)
    torch.cuda.synchronize()
    return {k: v.double().cpu().numpy() for k, v in out.items()}


_ORACLE_CACHE = {}


def oracle_result(name, wl):
    if name not in _ORACLE_CACHE:
        o = orc.Oracle.of(wl.mesh)
        _ORACLE_CACHE[name] = (o.pattern(), o.assemble(wl.u, wl.coeff, m=wl.mass_coeff))
    return _ORACLE_CACHE[name]


def frob(g, o):
    return np.linalg.norm(g - o) / np.linalg.norm(o)


CASES = ["tri_p1", "tri_p2", "tet_p1", "tet_p2", "tri_p3", "tet_p3"]


@pytest.mark.parametrize("name", CASES)
def test_pattern_and_slot_map_bit_exact(name):
    wl = wl_small(name)
    (rp_o, ci_o), _ = oracle_result(name, wl)
    fm = FemMesh.of(wl.mesh)
    rp, ci = fm.pattern()
    assert np.array_equal(rp.cpu().numpy(), rp_o)
    assert np.array_equal(ci.cpu().numpy(), ci_o)
    # slot map: entry c = (e n_p + i) n_p + j lands on (conn[e][i], conn[e][j])
    slot = fm.slot_map().cpu().numpy().astype(np.int64)
    conn = wl.mesh.conn.astype(np.int64)
    npl = conn.shape[1]
    rows = np.repeat(conn, npl, axis=1).ravel()
    cols = np.tile(conn, (1, npl)).ravel()
    row_of_slot = np.repeat(np.arange(len(rp_o) - 1), np.diff(rp_o))
    assert np.array_equal(row_of_slot[slot], rows)
    assert np.array_equal(ci_o[slot], cols)


@pytest.mark.parametrize("name", CASES)
def test_fp64_parity_per_entry(name):
    wl = wl_small(name)
    _, o = oracle_result(name, wl)
    fm = FemMesh.of(wl.mesh)
    g = gpu_assemble(fm, wl, "fp64")
    for k in ("M", "K", "T"):
        check_fp64(g[k], o[k], o["abs" + k], k)


@pytest.mark.parametrize("name", CASES)
def test_tf32x3_parity_frobenius(name):
    wl = wl_small(name)
    _, o = oracle_result(name, wl)
    fm = FemMesh.of(wl.mesh)
    g = gpu_assemble(fm, wl, "tf32x3")
    F.fem_device_status()
    for k in ("M", "K", "T"):
        assert frob(g[k], o[k]) <= TF32_TOL, (k, frob(g[k], o[k]))


@pytest.mark.parametrize("which", ["MKT", "M", "K", "T", "KT"])
def test_tf32x3_chunked_p3_tet(which):
    """P3 tetrahedra take the chunked tensor-core product (Q streamed
    through shared memory by quadrature-point chunks): 1296 elements (11
    tiles, ragged last tile), every subset of matrices, repeatable bits."""
    m = mg.structured_tet(6, 3, 0.15, seed=91)
    u = mg.fourier_field(m.coords, 92)
    wl = mg.Workload("tet_p3_chunked", m, u, mg.Coeff("sin", (2.0, 1.0, 3.0)))
    o = orc.Oracle.of(m).assemble(u, wl.coeff)
    fm = FemMesh.of(m)
    fm.symbolic()
    uu = torch.tensor(u, dtype=torch.float64, device="cuda")
    r1 = {k: v.clone() for k, v in fm.assemble(uu, "sin", (2.0, 1.0, 3.0), "tf32x3", which=tuple(which)).items()}
    r2 = fm.assemble(uu, "sin", (2.0, 1.0, 3.0), "tf32x3", which=tuple(which))
    torch.cuda.synchronize()
    F.fem_device_status()
    assert set(r1) == set(which)
    for k in which:
        assert torch.equal(r1[k], r2[k])
        g = r1[k].double().cpu().numpy()
        assert frob(g, o[k]) <= TF32_TOL, (k, frob(g, o[k]))


@pytest.mark.parametrize("name", CASES)
def test_fp32_simt_parity_frobenius(name):
    wl = wl_small(name)
    _, o = oracle_result(name, wl)
    fm = FemMesh.of(wl.mesh)
    g = gpu_assemble(fm, wl, "fp32")
    for k in ("M", "K", "T"):
        assert frob(g[k], o[k]) <= FP32_TOL, (k, frob(g[k], o[k]))


@pytest.mark.parametrize("prec", ["bf16x3", "bf16x6"])
@pytest.mark.parametrize("name", ["tri_p1", "tri_p2", "tet_p1", "tet_p2", "tri_p3"])
def test_bf16_split_parity_frobenius(prec, name):
    """The BF16 split products (kind::f16 tensor-core MMAs) against the
    oracle; tet_p3 has no BF16 tile (test_bf16_unavailable_cases)."""
    wl = wl_small(name)
    _, o = oracle_result(name, wl)
    fm = FemMesh.of(wl.mesh)
    g = gpu_assemble(fm, wl, prec)
    F.fem_device_status()
    for k in ("M", "K", "T"):
        assert frob(g[k], o[k]) <= BF_TOL[prec], (k, frob(g[k], o[k]))


def test_bf16x6_closer_than_bf16x3():
    """The third part must bring the error down to the FP32 floor of the
    formation (X in FP32, FP32 accumulation), well below BF16X3's: a slip in
    the x2 / q2 operands would leave BF16X6 at or above BF16X3's level."""
    wl = wl_small("tet_p2")
    _, o = oracle_result("tet_p2", wl)
    fm = FemMesh.of(wl.mesh)
    g3 = gpu_assemble(fm, wl, "bf16x3")
    g6 = gpu_assemble(fm, wl, "bf16x6")
    errs = {k: (frob(g3[k], o[k]), frob(g6[k], o[k])) for k in ("M", "K", "T")}
    for k, (e3, e6) in errs.items():
        assert e6 * 4 < e3 and e6 <= BF16X6_TOL, errs


def test_bf16_unavailable_cases():
    """P3 tetrahedra (their BF16 tile exceeds shared memory) and batches
    refuse the BF16 modes with FEM_EINVAL and leave the device usable."""
    wl = wl_small("tet_p3")
    fm = FemMesh.of(wl.mesh)
    u = torch.tensor(wl.u, dtype=torch.float64, device="cuda")
    for prec in ("bf16x3", "bf16x6"):
        with pytest.raises(F.FemError) as ei:
            fm.assemble(u, wl.coeff.kind, wl.coeff.params, prec)
        assert ei.value.code == F.FEM_EINVAL
        with pytest.raises(F.FemError) as ei:
            F.fem_batch_create([fm.h], F.fem_batch_opts(PRECISIONS[prec], 0, 1, 0))
        assert ei.value.code == F.FEM_EINVAL
    fm.assemble(u, wl.coeff.kind, wl.coeff.params, "tf32x3")
    torch.cuda.synchronize()
    F.fem_device_status()


@pytest.mark.parametrize("prec", ["fp64", "tf32x3", "fp32", "bf16x3", "bf16x6"])
def test_run_to_run_bitwise(prec):
    wl = wl_small("tri_p2")
    fm = FemMesh.of(wl.mesh)
    u = torch.tensor(wl.u, dtype=torch.float64, device="cuda")
    a = fm.assemble(u, wl.coeff.kind, wl.coeff.params, prec)
    a = {k: v.clone() for k, v in a.items()}
    for _ in range(3):
        b = fm.assemble(u, wl.coeff.kind, wl.coeff.params, prec)
        for k in a:
            assert torch.equal(a[k], b[k]), k


def test_separate_entry_points_match_all():
    wl = wl_small("tet_p2")
    fm = FemMesh.of(wl.mesh)
    u = torch.tensor(wl.u, dtype=torch.float64, device="cuda")
    both = fm.assemble(u, wl.coeff.kind, wl.coeff.params, "tf32x3")
    both = {k: v.clone() for k, v in both.items()}
    for k in ("M", "K", "T"):
        one = fm.assemble(u, wl.coeff.kind, wl.coeff.params, "tf32x3", which=(k,))
        assert torch.equal(one[k], both[k]), k
    vals = torch.empty(fm.nnz, dtype=torch.float32, device="cuda")
    F.fem_assemble_mass(fm.h, F.FEM_TF32X3, vals)
    torch.cuda.synchronize()
    assert torch.equal(vals, both["M"])


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_host_pointer_path_matches_device(prec):
    wl = wl_small("tri_p2")
    fm = FemMesh.of(wl.mesh)
    fm.symbolic()
    dt = np.float64 if prec == "fp64" else np.float32
    uh = np.ascontiguousarray(wl.u, dtype=np.float64)
    outs = {k: np.zeros(fm.nnz, dtype=dt) for k in "MKT"}
    F.fem_assemble_all(fm.h, F.coeff(wl.coeff.kind, wl.coeff.params), uh, F.torch_api.PRECISIONS[prec],
                       outs["M"], outs["K"], outs["T"])
    ud = torch.tensor(uh, device="cuda")
    d = fm.assemble(ud, wl.coeff.kind, wl.coeff.params, prec)
    for k in "MKT":
        assert np.array_equal(outs[k], d[k].cpu().numpy()), k


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_pinned_host_outputs_match_device(prec):
    """Page-locked and pageable host outputs, mixed in one call, carry the
    same bits as device outputs."""
    wl = wl_small("tet_p1")
    fm = FemMesh.of(wl.mesh)
    fm.symbolic()
    dt = torch.float64 if prec == "fp64" else torch.float32
    uh = torch.tensor(wl.u, dtype=torch.float64).pin_memory()
    pinned = {k: torch.full((fm.nnz,), float("nan"), dtype=dt).pin_memory() for k in "MK"}
    pageable = np.full(fm.nnz, np.nan, dtype=np.float64 if prec == "fp64" else np.float32)
    F.fem_assemble_all(fm.h, F.coeff(wl.coeff.kind, wl.coeff.params), uh, F.torch_api.PRECISIONS[prec],
                       pinned["M"], pinned["K"], pageable)
    d = fm.assemble(torch.tensor(wl.u, device="cuda"), wl.coeff.kind, wl.coeff.params, prec)
    torch.cuda.synchronize()
    assert torch.equal(pinned["M"], d["M"].cpu()) and torch.equal(pinned["K"], d["K"].cpu())
    assert np.array_equal(pageable, d["T"].cpu().numpy())


@pytest.mark.parametrize("prec,N", [("fp64", 48), ("tf32x3", 64)])
def test_host_outputs_through_the_chunk_pipeline(prec, N):
    """Host outputs of a mesh whose element scratch spans several chunk-plan
    chunks (each chunk formed, its completed slots summed and copied while
    the next chunk is formed) carry the same bits as device outputs."""
    m = mg.structured_tet(N, 1, 0.15, seed=12)
    fm = FemMesh.of(m)
    fm.symbolic()
    law = ("sin", (2.0, 1.0, 3.0))
    dt = torch.float64 if prec == "fp64" else torch.float32
    u = mg.fourier_field(m.coords, 13)
    uh = torch.tensor(u, dtype=torch.float64).pin_memory()
    outs = {k: torch.full((fm.nnz,), float("nan"), dtype=dt).pin_memory() for k in "MKT"}
    nb = (fm.nnz * (8 if prec == "fp64" else 4))
    assert m.n_elems * 36 * (8 if prec == "fp64" else 4) > 3 * (48 << 20) and nb > 0   # several chunks
    F.fem_assemble_all(fm.h, F.coeff(*law), uh, F.torch_api.PRECISIONS[prec], outs["M"], outs["K"], outs["T"])
    d = fm.assemble(torch.tensor(u, device="cuda"), law[0], law[1], prec)
    torch.cuda.synchronize()
    for k in "MKT":
        assert torch.equal(outs[k], d[k].cpu()), k
    fm.close()


def test_coefficient_laws():
    """sin and piecewise-linear laws against the oracle (FP64 per entry)."""
    m = mg.structured_tri(12, 2, 0.2, seed=5)
    u = 1200.0 * mg.fourier_field(m.coords, 6) - 100.0       # spans all pwlin branches
    o = orc.Oracle.of(m)
    fm = FemMesh.of(m)
    for c in (mg.Coeff("sin", (2.0, 1.0, 3.0)), mg.Coeff("pwlin", (0.0, 200.0, 1000.0, 1.5, 0.7, 0.5)),
              mg.Coeff("poly", (0.5, -0.25, 0.125, 0.01, -0.001))):
        uu = u if c.kind == "pwlin" else u / 1200.0
        r = o.assemble(uu, c)
        g = fm.assemble(torch.tensor(uu, device="cuda"), c.kind, c.params, "fp64")
        for k in ("K", "T"):
            gk = g[k].cpu().numpy()
            check_fp64(gk, r[k], r["abs" + k], (c.kind, k))


@pytest.mark.parametrize("law", [("sin", (2.0, 1.0, 3.0), 1.0, 0.0),
                                 ("pwlin", (0.0, 200.0, 1000.0, 1.5, 0.7, 0.5), 1200.0, -100.0)])
def test_tf32x3_coefficient_laws(law):
    kind, params, scale, shift = law
    m = mg.structured_tet(5, 2, 0.15, seed=8)
    u = scale * mg.fourier_field(m.coords, 9) + shift
    c = mg.Coeff(kind, params)
    r = orc.Oracle.of(m).assemble(u, c)
    g = FemMesh.of(m).assemble(torch.tensor(u, device="cuda"), kind, params, "tf32x3")
    for k in ("M", "K", "T"):
        assert frob(g[k].double().cpu().numpy(), r[k]) <= TF32_TOL, k


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_form_and_sum_phases(prec):
    """fem_form_elements + fem_sum_elements == fem_assemble_all, bit for bit;
    summing with another precision than was formed is refused."""
    wl = wl_small("tri_p3")
    fm = FemMesh.of(wl.mesh)
    u = torch.tensor(wl.u, dtype=torch.float64, device="cuda")
    ref = {k: v.clone() for k, v in fm.assemble(u, wl.coeff.kind, wl.coeff.params, prec).items()}
    dt = torch.float64 if prec == "fp64" else torch.float32
    out = {k: torch.empty(fm.nnz, dtype=dt, device="cuda") for k in "MKT"}
    pc = F.torch_api.PRECISIONS[prec]
    F.fem_form_elements(fm.h, F.coeff(wl.coeff.kind, wl.coeff.params), u, pc, F.FEM_MAT_M | F.FEM_MAT_K | F.FEM_MAT_T)
    F.fem_sum_elements(fm.h, pc, out["M"], out["K"], out["T"])
    torch.cuda.synchronize()
    for k in "MKT":
        assert torch.equal(out[k], ref[k]), k
    other = F.FEM_FP32 if prec == "fp64" else F.FEM_FP64
    with pytest.raises(F.FemError) as ei:
        F.fem_sum_elements(fm.h, other, out["M"], None, None)
    assert ei.value.code == F.FEM_ESTATE


@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
@pytest.mark.parametrize("fan", [100, 300])
def test_long_rows_fallback_paths(prec, fan):
    """Triangle fans: the centre row has fan + 1 entries and its diagonal
    slot `fan` contributors.  With 300 triangles the symbolic phase sorts
    the centre's 300 incidences and the row's 900 keys without staging them
    in shared memory; with 100 it ranks the incidences over several keys
    per lane and stages the row's 300 keys."""
    m = mg.fan_tri(fan, seed=2)
    u = mg.uniform_field(m.n_nodes, 3)
    c = mg.Coeff("poly", (1.0, 0.5, 0.25, 0.0, 0.0))
    o = orc.Oracle.of(m)
    rp_o, ci_o = o.pattern()
    r = o.assemble(u, c)
    fm = FemMesh.of(m)
    rp, ci = fm.pattern()
    assert np.array_equal(rp.cpu().numpy(), rp_o) and np.array_equal(ci.cpu().numpy(), ci_o)
    g = fm.assemble(torch.tensor(u, device="cuda"), c.kind, c.params, prec)
    for k in ("M", "K", "T"):
        gk = g[k].double().cpu().numpy()
        if prec == "fp64":
            check_fp64(gk, r[k], r["abs" + k], k)
        else:
            assert frob(gk, r[k]) <= TF32_TOL, k


def test_mass_coefficient_scales():
    m = mg.structured_tet(3, 2, 0.15, seed=1)
    f1, f2 = FemMesh.of(m, mass=1.0), FemMesh.of(m, mass=2.5)
    a = f1.assemble(None, "poly", (1.0,), "fp64", which=("M",))["M"]
    b = f2.assemble(None, "poly", (1.0,), "fp64", which=("M",))["M"]
    torch.testing.assert_close(b, 2.5 * a, rtol=1e-15, atol=0)
    assert abs(a.sum().item() - 1.0) < 1e-12


def test_errors_and_edge_cases():
    m = mg.structured_tri(3, 1, 0.0)
    fm = FemMesh.of(m)
    vals = torch.empty(100, dtype=torch.float64, device="cuda")
    with pytest.raises(F.FemError) as ei:              # before symbolic
        F.fem_assemble_mass(fm.h, F.FEM_FP64, vals)
    assert ei.value.code == F.FEM_ESTATE
    fm.symbolic()
    with pytest.raises(F.FemError) as ei:              # u missing
        F.fem_assemble_stiffness(fm.h, F.coeff("poly", (1.0,)), None, F.FEM_FP64, vals)
    assert ei.value.code == F.FEM_EINVAL
    with pytest.raises(F.FemError) as ei:              # bad law
        F.fem_assemble_stiffness(fm.h, F.coeff("pwlin", (1.0, 0.0, 2.0, 3.0)), vals, F.FEM_FP64, vals)
    assert ei.value.code == F.FEM_EINVAL
    bad = mg.Mesh(2, 1, m.coords, m.conn.copy())
    bad.conn[3, 1] = m.n_nodes + 5
    with pytest.raises(F.FemError) as ei:
        FemMesh.of(bad)
    assert ei.value.code == F.FEM_EINVAL
    deg = mg.Mesh(2, 1, m.coords.copy(), m.conn)
    deg.coords[m.conn[4, 1]] = deg.coords[m.conn[4, 0]]     # collapse an element
    with pytest.raises(F.FemError) as ei:
        FemMesh.of(deg)
    assert ei.value.code == F.FEM_EDEGENERATE
    # empty mesh: no elements, empty rows
    empty = FemMesh(2, 1, m.coords, np.zeros((0, 3), dtype=np.int32))
    empty.symbolic()
    assert empty.nnz == 0
    empty.assemble(torch.zeros(m.n_nodes, device="cuda", dtype=torch.float64), "poly", (1.0,), "fp64")


def _single_simplex(d, p, n_elems):
    """n_elems copies of one skewed simplex sharing no nodes (one element:
    n_p^2 contributions, fewer than one 64-contribution group for P1/P2; an
    odd count for P1 triangles)."""
    K = mg.local_nodes(d, p).astype(np.float64) / p          # barycentric
    verts = np.array([[0.1, 0.2], [1.3, 0.1], [0.4, 0.9]]) if d == 2 else \
        np.array([[0.1, 0.2, 0.0], [1.2, 0.1, 0.3], [0.3, 1.1, 0.2], [0.2, 0.4, 1.3]])
    one = K @ verts                                           # (n_p, d)
    n_p = one.shape[0]
    coords = np.concatenate([one + 2.0 * e for e in range(n_elems)])
    conn = np.arange(n_elems * n_p, dtype=np.int32).reshape(n_elems, n_p)
    return mg.Mesh(d=d, p=p, coords=coords, conn=conn, name=f"single_{d}{p}")


@pytest.mark.parametrize("d,p,n", [(2, 1, 1), (2, 1, 3), (2, 2, 1), (2, 3, 1), (3, 1, 1), (3, 2, 2), (3, 3, 1)])
def test_tiny_meshes(d, p, n):
    """Meshes far below one tile and one contribution group, in every
    precision, against the oracle."""
    m = _single_simplex(d, p, n)
    u = mg.uniform_field(m.n_nodes, 11 + d * 3 + p)
    c = mg.Coeff("poly", (1.0, 0.5, 0.25, 0.0, 0.0))
    r = orc.Oracle.of(m).assemble(u, c)
    fm = FemMesh.of(m)
    precs = ("fp64", "tf32x3", "fp32") + (("bf16x3", "bf16x6") if (d, p) != (3, 3) else ())
    tol = {"tf32x3": TF32_TOL, "fp32": FP32_TOL, **BF_TOL}
    for prec in precs:
        g = fm.assemble(torch.tensor(u, device="cuda"), c.kind, c.params, prec)
        torch.cuda.synchronize()
        for k in ("M", "K", "T"):
            gk = g[k].double().cpu().numpy()
            if prec == "fp64":
                check_fp64(gk, r[k], r["abs" + k], (prec, k))
            else:
                assert frob(gk, r[k]) <= tol[prec], (prec, k, frob(gk, r[k]))
    F.fem_device_status()


def test_sliver_elements_use_fp64_geometry():
    m = mg.sliver_tri(16, 0.05, seed=3)
    fm = FemMesh.of(m)
    assert fm.info().n_flagged > 0
    u = mg.uniform_field(m.n_nodes, 4)
    c = mg.Coeff("poly", (1.0, 0.5, 0.25, 0.0, 0.0))
    o = orc.Oracle.of(m).assemble(u, c)
    g = fm.assemble(torch.tensor(u, dtype=torch.float64, device="cuda"), c.kind, c.params, "tf32x3")
    for k in ("M", "K", "T"):
        assert frob(g[k].double().cpu().numpy(), o[k]) <= TF32_TOL, k


def test_torch_caching_allocator_and_failure_injection():
    """The allocator hook bound to torch's caching allocator; an allocator
    that fails at the N-th request makes the call return FEM_ENOMEM and the
    library stays usable."""
    state = {"n": 0, "fail_at": None, "live": {}}

    def alloc(size, stream, ctx):
        state["n"] += 1
        if state["fail_at"] is not None and state["n"] >= state["fail_at"]:
            return None
        p = torch.cuda.caching_allocator_alloc(size, stream=stream or 0)
        state["live"][p] = size
        return p

    def free(ptr, size, stream, ctx):
        state["live"].pop(ptr, None)
        torch.cuda.caching_allocator_delete(ptr)

    a = F.fem_allocator(F.ALLOC_FN(alloc), F.FREE_FN(free), None)
    F.fem_set_allocator(a)
    try:
        wl = wl_small("tri_p2")
        fm = FemMesh.of(wl.mesh)
        g1 = gpu_assemble(fm, wl, "fp64")
        fm.close()
        assert not state["live"]
        state["n"], state["fail_at"] = 0, 4
        with pytest.raises(F.FemError) as ei:
            fm2 = FemMesh.of(wl.mesh)
            fm2.symbolic()
        assert ei.value.code == F.FEM_ENOMEM
    finally:
        F.fem_set_allocator(None)
    fm3 = FemMesh.of(wl.mesh)
    g3 = gpu_assemble(fm3, wl, "fp64")
    for k in g1:
        assert np.array_equal(g1[k], g3[k])


# ------------------------------------------------------------------ full size
@pytest.mark.parametrize("prec", ["fp64", "tf32x3"])
def test_full_size_tri_p2_1024_sampled(prec):
    """2 097 152 P2 triangles in the launch configuration the benchmark
    times: nnz by its closed form, sampled rows' patterns from the element
    definition, sampled entries against the oracle computed one by one."""
    wl = mg.workload("tri_p2_1024")
    N = 1024
    fm = FemMesh.of(wl.mesh)
    fm.symbolic()
    assert fm.nnz == 46 * N * N + 16 * N + 1
    rp, ci = (t.cpu().numpy() for t in fm.pattern())
    conn = wl.mesh.conn
    rng = np.random.default_rng(123)
    rows = rng.choice(wl.mesh.n_nodes, 40, replace=False)
    for r in rows:
        els = np.nonzero((conn == r).any(axis=1))[0]
        assert np.array_equal(ci[rp[r]:rp[r + 1]], np.unique(conn[els]))
    g = gpu_assemble(fm, wl, prec)
    slots = rng.choice(fm.nnz, 3000, replace=False)
    row_of = np.searchsorted(rp, slots, side="right") - 1
    s = orc.Oracle.of(wl.mesh).entries(row_of, ci[slots], wl.u, wl.coeff)
    for k in ("M", "K", "T"):
        if prec == "fp64":
            check_fp64(g[k][slots], s[k], s["abs" + k], k)
        else:
            err = np.abs(g[k][slots] - s[k])
            assert (err <= 2e-6 * s["abs" + k] + 1e-300).all(), (k, (err / s["abs" + k]).max())


_TET_FULL = {"tet_p1_128": (128, lambda N: 15 * N**3 + 21 * N**2 + 9 * N + 1),
             "tet_p2_64": (64, lambda N: 230 * N**3 + 138 * N**2 + 24 * N + 1)}


@pytest.mark.parametrize("name,prec", [("tet_p1_128", "tf32x3"), ("tet_p1_128", "fp64"), ("tet_p2_64", "tf32x3"),
                                       ("tet_p2_64", "fp64")])
def test_full_size_tetrahedra_sweep_sampled(name, prec):
    """12 582 912 P1 / 1 572 864 P2 tetrahedra in the benchmark's launch
    configuration, reassembled with fresh fields on one symbolic pattern
    (Newton-style sweep): nnz by its closed form, sampled rows' patterns
    from the element definition, the last reassembly's sampled entries
    against the oracle computed one by one, and the first field reassembled
    again at the end equal bit for bit to its first reassembly."""
    wl = mg.workload(name)
    N, nnz_of = _TET_FULL[name]
    fm = FemMesh.of(wl.mesh)
    fm.symbolic()
    assert fm.nnz == nnz_of(N)
    rp, ci = (t.cpu().numpy() for t in fm.pattern())
    conn = wl.mesh.conn
    rng = np.random.default_rng(321)
    flat = conn.ravel()
    perm = np.argsort(flat, kind="stable")
    order = perm // conn.shape[1]                                  # elements, grouped by node
    starts = np.searchsorted(flat[perm], np.arange(wl.mesh.n_nodes + 1))
    for r in rng.choice(wl.mesh.n_nodes, 10, replace=False):
        els = order[starts[r]:starts[r + 1]]
        assert np.array_equal(ci[rp[r]:rp[r + 1]], np.unique(conn[els]))
    fields = [mg.fourier_field(wl.mesh.coords, 3 + s) for s in range(3)]
    first = None
    for f in fields:
        g = gpu_assemble(fm, mg.Workload(wl.name, wl.mesh, f, wl.coeff), prec)
        if first is None:
            first = g
    again = gpu_assemble(fm, mg.Workload(wl.name, wl.mesh, fields[0], wl.coeff), prec)
    F.fem_device_status()
    for k in ("M", "K", "T"):
        assert np.array_equal(again[k], first[k]), k
    slots = rng.choice(fm.nnz, 2000, replace=False)
    row_of = np.searchsorted(rp, slots, side="right") - 1
    s = orc.Oracle.of(wl.mesh).entries(row_of, ci[slots], fields[-1], wl.coeff)
    for k in ("M", "K", "T"):
        if prec == "fp64":
            check_fp64(g[k][slots], s[k], s["abs" + k], k)
        else:
            err = np.abs(g[k][slots] - s[k])
            assert (err <= 2e-6 * s["abs" + k] + 1e-300).all(), (k, (err / s["abs" + k]).max())
