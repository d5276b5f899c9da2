"""The request server (fem_serve_*): results of requests served concurrently
over several streams equal fem_assemble_all of the same mesh, u and law at
the same precision bit for bit; requests of one mesh run in submission
order; admission respects the device-memory budget; errors are reported at
submit or in the result."""
import numpy as np
import pytest

import meshgen as mg
import oracle as orc

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2204_03893_gb300 as F  # noqa: E402
from paper_2204_03893_gb300.torch_api import PRECISIONS, FemMesh, FemServer  # noqa: E402


def meshes():
    out = []
    for i, (d, p, N) in enumerate([(2, 1, 19), (2, 2, 13), (3, 1, 6), (3, 2, 4), (2, 3, 7), (3, 3, 3)]):
        m = mg.structured_tri(N, p, 0.2, seed=40 + i) if d == 2 else mg.structured_tet(N, p, 0.15, seed=40 + i)
        out.append(m)
    return out


def single(m, u, kind, params, prec):
    fm = FemMesh.of(m)
    fm.symbolic()
    r = fm.assemble(torch.tensor(u, dtype=torch.float64, device="cuda"), kind, params, prec)
    torch.cuda.synchronize()
    out = {k: v.clone() for k, v in r.items()}
    fm.close()
    return out


@pytest.mark.parametrize("fuse_min", [0, 2])
@pytest.mark.parametrize("prec", ["tf32x3", "fp64"])
def test_serve_matches_single_calls(prec, fuse_min):
    ms = meshes()
    S = FemServer(prec, budget_bytes=2 << 30, max_inflight=4, n_streams=3, fuse_min=fuse_min)
    try:
        # ASSEMBLE every mesh, then interleave 3 REASSEMBLE rounds with new u over all meshes
        tick = [S.assemble(m, "poly", (1.0, 0.3, 0.2), mg.fourier_field(m.coords, 1 + i)) for i, m in enumerate(ms)]
        ids = []
        for i, (m, t) in enumerate(zip(ms, tick)):
            r, vals = S.result(t)
            assert r.status == 0, F._err()
            ids.append(r.mesh_id)
            assert r.prec == PRECISIONS[prec]
            ref = single(m, mg.fourier_field(m.coords, 1 + i), "poly", (1.0, 0.3, 0.2), prec)
            for k in "MKT":
                assert torch.equal(vals[k], ref[k]), (i, k)
        pend = []
        for s in range(3):
            for i, m in enumerate(ms):
                u = mg.fourier_field(m.coords, 100 + 10 * s + i)
                law = ("sin", (2.0, 1.0, 3.0)) if s == 1 else ("poly", (1.0, 0.0, 1.0))
                pend.append((i, u, law, S.reassemble(ids[i], law[0], law[1], u)))
        for i, u, law, t in pend:
            r, vals = S.result(t)
            assert r.status == 0
            m = ms[i]
            ref = single(m, u, law[0], law[1], prec)
            for k in "MKT":
                assert torch.equal(vals[k], ref[k]), (i, k)
        st = S.stats()
        assert st.pending == 0 and st.inflight == 0 and st.resident_meshes == len(ms)
        assert st.peak_bytes <= 2 << 30
        assert st.single_launches + st.fused_requests == len(ms) * 4
        if fuse_min == 0:
            assert st.fused_launches == 0
    finally:
        S.close()


@pytest.mark.parametrize("prec", ["tf32x3", "fp64", "fp32"])
def test_serve_fused_launches(prec):
    """Requests of many meshes queued at once start as fused batch launches
    (fewer launches than requests, several requests per launch); partial
    matrix subsets and meshes skipped in a launch; results equal single-mesh
    calls bit for bit; a mesh assembled later joins the batch (rebuilt), an
    evicted one leaves it."""
    ms = meshes()
    S = FemServer(prec, budget_bytes=4 << 30, max_inflight=64, n_streams=2, fuse_min=2)
    try:
        ids = []
        for i, m in enumerate(ms[:5]):
            r, _ = S.result(S.assemble(m, "poly", (1.0,), mg.fourier_field(m.coords, 300 + i), which="M"))
            assert r.status == 0
            ids.append(r.mesh_id)
        subsets = ["MKT", "M", "KT", "T", "MK"]
        todo = []
        for rnd in range(3):
            for i in range(5):
                if rnd == 1 and i == 2:
                    continue           # mesh 2 skipped in this round's launches
                u = mg.fourier_field(ms[i].coords, 400 + 10 * rnd + i)
                law = ("sin", (2.0, 1.0, 3.0)) if (i + rnd) % 2 else ("poly", (1.0, 0.3, 0.2))
                todo.append((i, u, law, subsets[(i + rnd) % len(subsets)]))
        # a larger ASSEMBLE first keeps the scheduler busy (it builds the
        # pattern synchronously) while the requests queue up behind it
        tb = S.assemble(mg.structured_tri(200, 2, 0.2, seed=9), which="M")
        pend = [(i, u, law, which, S.reassemble(ids[i], law[0], law[1], u, which=which))
                for i, u, law, which in todo]
        assert S.result(tb)[0].status == 0
        for i, u, law, which, t in pend:
            r, vals = S.result(t)
            assert r.status == 0, F._err()
            assert set(vals) == set(which)
            ref = single(ms[i], u, law[0], law[1], prec)
            for k in which:
                assert torch.equal(vals[k], ref[k]), (i, which, k)
        st = S.stats()
        assert st.fused_launches >= 1 and st.fused_requests >= 2 * st.fused_launches
        assert st.fused_launches < st.fused_requests
        builds = st.batch_builds
        # the resident set changes: one mesh more, one fewer
        r, _ = S.result(S.assemble(ms[5], "poly", (1.0,), mg.fourier_field(ms[5].coords, 305), which="M"))
        ids.append(r.mesh_id)
        S.evict(ids[0])
        us = {i: mg.fourier_field(ms[i].coords, 500 + i) for i in range(1, 6)}
        tb = S.assemble(mg.structured_tri(200, 2, 0.2, seed=10), which="M")
        pend = [(i, us[i], S.reassemble(ids[i], "poly", (1.0, 0.0, 1.0), us[i])) for i in range(1, 6)]
        assert S.result(tb)[0].status == 0
        for i, u, t in pend:
            r, vals = S.result(t)
            assert r.status == 0, F._err()
            ref = single(ms[i], u, "poly", (1.0, 0.0, 1.0), prec)
            for k in "MKT":
                assert torch.equal(vals[k], ref[k]), (i, k)
        st = S.stats()
        assert st.batch_builds > builds and st.resident_meshes == 7
        assert st.pending == 0 and st.inflight == 0
    finally:
        S.close()


def test_serve_accuracy_against_oracle():
    m = mg.structured_tri(11, 2, 0.2, seed=5)
    u = mg.fourier_field(m.coords, 6)
    S = FemServer("tf32x3")
    try:
        r, vals = S.result(S.assemble(m, "poly", (1.0, 0.0, 1.0), u))
    finally:
        S.close()
    ref = orc.Oracle.of(m).assemble(u, mg.Coeff("poly", (1.0, 0.0, 1.0)))
    for k in "MKT":
        g = vals[k].double().cpu().numpy()
        assert np.linalg.norm(g - ref[k]) <= 1e-6 * np.linalg.norm(ref[k]), k


def test_serve_same_mesh_in_order_and_partial():
    """Many requests of one mesh queued at once: each result belongs to its
    own u (no request sees another's nodal values or outputs)."""
    m = mg.structured_tet(4, 2, 0.15, seed=8)
    S = FemServer("tf32x3", max_inflight=8, n_streams=4)
    try:
        r, _ = S.result(S.assemble(m, which="M"))
        mid = r.mesh_id
        us = [mg.fourier_field(m.coords, 200 + s) for s in range(8)]
        ts = [S.reassemble(mid, "poly", (1.0, 0.5), u, which="KT" if s % 2 else "T") for s, u in enumerate(us)]
        for s, (u, t) in enumerate(zip(us, ts)):
            r, vals = S.result(t)
            assert r.status == 0
            assert set(vals) == ({"K", "T"} if s % 2 else {"T"})
            ref = single(m, u, "poly", (1.0, 0.5), "tf32x3")
            for k in vals:
                assert torch.equal(vals[k], ref[k]), (s, k)
            assert r.t_submit_us <= r.t_start_us <= r.t_done_us
    finally:
        S.close()


def test_serve_budget_admission_and_eviction():
    m1 = mg.structured_tri(40, 2, 0.2, seed=1)
    m2 = mg.structured_tri(40, 2, 0.2, seed=2)
    # a budget that holds one of these meshes (with its outputs), not two
    probe = FemServer("tf32x3")
    try:
        r, _ = probe.result(probe.assemble(m1, which="M"))
        one = probe.stats().peak_bytes
    finally:
        probe.close()
    S = FemServer("tf32x3", budget_bytes=int(one * 1.2))
    try:
        with pytest.raises(F.FemError) as ei:
            S.assemble(mg.structured_tri(80, 2, 0.2, seed=3), which="M")
        assert ei.value.code == F.FEM_EBUSY
        t1 = S.assemble(m1, which="M")
        t2 = S.assemble(m2, which="M")
        r1, _ = S.result(t1)
        assert r1.status == 0
        # the second mesh does not fit while the first is resident
        assert F.fem_serve_poll(S.h, t2, 0) is None
        with pytest.raises(F.FemError) as ei:
            F.fem_serve_poll(S.h, t2, 20000)
        assert ei.value.code == F.FEM_ETIMEOUT
        assert S.stats().pending == 1
        S.evict(r1.mesh_id)
        r2, vals = S.result(t2)
        assert r2.status == 0 and r2.mesh_id != r1.mesh_id
        ref = single(m2, np.zeros(m2.coords.shape[0]), "poly", (1.0,), "tf32x3")
        assert torch.equal(vals["M"], ref["M"])
        assert S.stats().peak_bytes <= int(one * 1.2)
    finally:
        S.close()


def test_serve_errors():
    S = FemServer("fp64")
    try:
        m = mg.structured_tri(4, 1)
        with pytest.raises(F.FemError) as ei:
            F.fem_serve_submit(S.h, 7)
        assert ei.value.code == F.FEM_EINVAL
        with pytest.raises(F.FemError) as ei:
            S.reassemble(12345, "poly", (1.0,), np.zeros(m.coords.shape[0]))
        assert ei.value.code == F.FEM_EINVAL
        with pytest.raises(F.FemError) as ei:
            S.assemble(m, "poly", (1.0,), None, which="K")       # K without u
        assert ei.value.code == F.FEM_EINVAL
        with pytest.raises(F.FemError) as ei:
            F.fem_serve_release(S.h, 999)
        assert ei.value.code == F.FEM_EINVAL
        # a degenerate mesh fails in the result, not at submit
        bad = mg.structured_tri(3, 1)
        bad.coords[:] = 0.0
        r, vals = S.result(S.assemble(bad, which="M"))
        assert r.status == F.FEM_EDEGENERATE and not vals
        t = S.assemble(m, which="M")
        r, _ = S.result(t, release=False)
        with pytest.raises(F.FemError) as ei:
            F.fem_serve_evict(S.h, 424242)
        assert ei.value.code == F.FEM_EINVAL
        F.fem_serve_release(S.h, t)
    finally:
        S.close()


def test_serve_next_done_completion_order():
    """fem_serve_next_done hands out every finished, unreleased request once,
    in completion order; a released request is never handed out."""
    ms = meshes()[:4]
    S = FemServer("fp32", max_inflight=8, n_streams=2)
    try:
        ids = []
        for m in ms:
            r, _ = S.result(S.assemble(m, which="M"))
            ids.append(r.mesh_id)
        # the ASSEMBLE results were taken by ticket and released: none is pending here
        assert F.fem_serve_next_done(S.h, 0) is None
        want = {}
        for s in range(3):
            for i, m in enumerate(ms):
                u = mg.fourier_field(m.coords, 600 + 10 * s + i)
                want[S.reassemble(ids[i], "poly", (1.0, 0.5), u, which="KT")] = (i, u)
        got = []
        while len(got) < len(want):
            t = F.fem_serve_next_done(S.h, 10_000_000)
            assert t in want and t not in got
            got.append(t)
            r = F.fem_serve_poll(S.h, t, 0)
            assert r is not None and r.status == 0
        assert F.fem_serve_next_done(S.h, 0) is None
        # requests of one mesh finish in submission order
        for i in range(len(ms)):
            mine = [t for t in got if want[t][0] == i]
            assert mine == sorted(mine)
        for t in got[:3]:
            i, u = want[t]
            r, vals = S.result(t)
            ref = single(ms[i], u, "poly", (1.0, 0.5), "fp32")
            for k in "KT":
                assert torch.equal(vals[k], ref[k])
        for t in got[3:]:
            F.fem_serve_release(S.h, t)
        with pytest.raises(F.FemError) as ei:
            F.fem_serve_next_done(S.h, 1000)
        assert ei.value.code == F.FEM_ETIMEOUT
    finally:
        S.close()
