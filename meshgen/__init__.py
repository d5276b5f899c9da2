"""Seeded synthetic inputs for the finite element assembly path.

This module is the only code shared by the CPU oracle and the CUDA library's
tests and benchmarks.  It generates *inputs* only: structured simplex meshes
with Lagrange P1-P3 degree-of-freedom numbering, vertex jitter, nodal fields
and coefficient parameters.  It holds none of the method's arithmetic (no
quadrature, no basis functions, no element matrices, no sparsity pattern).

Mesh conventions (shared input format, stated in ``include/fem.h`` too):

* Reference simplex vertices: v0 = 0, v_k = e_k (unit vectors).
* Local node order inside an element, as barycentric multi-indices
  (k_0..k_d) with sum p: the d+1 vertices; then edge nodes, edges in
  lexicographic order of their vertex pairs (a<b), and for p=3 the node
  nearer vertex a first; then face nodes (p=3 only), faces in lexicographic
  order of their vertex triples.
* Structured meshes of the unit square / cube, N cells per side, every
  square split along the (0,0)-(1,1) diagonal, every cube split into the six
  Kuhn (path) tetrahedra, positively oriented.
* Global dofs are the points of the p-times refined lattice ((pN+1)^d
  points), numbered x-fastest.  Higher-order nodes sit at the affine images
  of their barycentric positions (straight edges).
* Vertex jitter: interior vertices move by U[-alpha h, alpha h] in every
  coordinate; boundary vertices only tangentially; corners stay fixed, so
  the domain measure stays exactly 1.
"""
from __future__ import annotations

import itertools
import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "local_nodes", "Mesh", "structured_tri", "structured_tet", "fourier_field",
    "uniform_field", "Coeff", "Workload", "workload", "n_local",
    "batched_meshes", "sliver_tri", "fan_tri",
]


def n_local(d: int, p: int) -> int:
    """Number of Lagrange nodes of a degree-p simplex in dimension d."""
    return math.comb(p + d, d)


def local_nodes(d: int, p: int) -> np.ndarray:
    """Barycentric multi-indices of the local nodes, shape (n_p, d+1), in the
    local order described in the module docstring."""
    if d not in (2, 3) or p not in (1, 2, 3):
        raise ValueError("d must be 2 or 3 and p in 1..3")
    nv = d + 1
    out = []
    for a in range(nv):
        k = [0] * nv
        k[a] = p
        out.append(k)
    if p >= 2:
        for a, b in itertools.combinations(range(nv), 2):
            if p == 2:
                k = [0] * nv
                k[a] = 1
                k[b] = 1
                out.append(k)
            else:  # p == 3: two nodes per edge, nearer a first
                k = [0] * nv
                k[a] = 2
                k[b] = 1
                out.append(k)
                k = [0] * nv
                k[a] = 1
                k[b] = 2
                out.append(k)
    if p == 3:
        for a, b, c in itertools.combinations(range(nv), 3):
            k = [0] * nv
            k[a] = k[b] = k[c] = 1
            out.append(k)
    arr = np.asarray(out, dtype=np.int64)
    assert arr.shape[0] == n_local(d, p)
    return arr


@dataclass
class Mesh:
    """A simplex mesh: ``coords`` (n_nodes x d, float64), ``conn``
    (n_elems x n_p, int32, local order of :func:`local_nodes`)."""
    d: int
    p: int
    coords: np.ndarray
    conn: np.ndarray
    name: str = ""

    @property
    def n_nodes(self) -> int:
        return int(self.coords.shape[0])

    @property
    def n_elems(self) -> int:
        return int(self.conn.shape[0])

    @property
    def n_p(self) -> int:
        return int(self.conn.shape[1])


def _seeds(seed: int, n: int):
    return [np.random.default_rng(s) for s in np.random.SeedSequence(seed).spawn(n)]


def _jitter_vertices(grid_shape, h, alpha, rng):
    """Jitter displacements for a vertex grid of shape (N+1,)*d indexed
    [.., y, x] (x fastest).  Boundary vertices move tangentially only."""
    d = len(grid_shape)
    disp = rng.uniform(-alpha * h, alpha * h, size=grid_shape + (d,))
    for axis_coord in range(d):
        # array axis holding coordinate `axis_coord` (x is the last array axis)
        arr_axis = d - 1 - axis_coord
        n = grid_shape[arr_axis]
        sl = [slice(None)] * d
        sl[arr_axis] = 0
        disp[tuple(sl) + (axis_coord,)] = 0.0
        sl[arr_axis] = n - 1
        disp[tuple(sl) + (axis_coord,)] = 0.0
    return disp


def _build_lagrange_mesh(d, p, N, vert_xyz, simplices_vidx, simplices_vlat, name):
    """Common P-p node placement.  ``simplices_vidx``: (E, d+1) vertex-grid
    flat indices; ``simplices_vlat``: (E, d+1, d) integer vertex-grid
    coordinates.  Returns a :class:`Mesh` on the p-refined lattice."""
    L = p * N + 1
    K = local_nodes(d, p)                      # (n_p, d+1)
    E = simplices_vidx.shape[0]
    n_p = K.shape[0]
    conn = np.empty((E, n_p), dtype=np.int64)
    coords = np.zeros((L ** d, d), dtype=np.float64)
    vx = vert_xyz[simplices_vidx]              # (E, d+1, d) jittered coords
    strides = np.array([L ** a for a in range(d)], dtype=np.int64)  # x fastest
    for loc in range(n_p):
        k = K[loc]                             # (d+1,)
        lat = np.einsum("t,etc->ec", k, simplices_vlat)  # lattice coords, integer
        idx = lat @ strides
        conn[:, loc] = idx
        x = np.einsum("t,etc->ec", k.astype(np.float64) / p, vx)
        coords[idx] = x
    used = np.zeros(L ** d, dtype=bool)
    used[conn.ravel()] = True
    if not used.all():
        raise AssertionError("lattice numbering left unused points")
    return Mesh(d=d, p=p, coords=coords, conn=conn.astype(np.int32), name=name)


def structured_tri(N: int, p: int = 1, alpha: float = 0.2, seed: int = 0) -> Mesh:
    """Unit square, N x N cells, each split into two triangles along the
    (0,0)-(1,1) diagonal: 2 N^2 elements, (pN+1)^2 dofs."""
    h = 1.0 / N
    (rng,) = _seeds(seed, 1)
    j, i = np.meshgrid(np.arange(N + 1), np.arange(N + 1), indexing="ij")
    xyz = np.stack([i * h, j * h], axis=-1).astype(np.float64)   # [y, x, 2]
    if alpha:
        xyz = xyz + _jitter_vertices((N + 1, N + 1), h, alpha, rng)
    vert_xyz = xyz.reshape(-1, 2)
    ci, cj = np.meshgrid(np.arange(N), np.arange(N), indexing="xy")
    ci = ci.ravel()
    cj = cj.ravel()                                # cell order: y-major, x fastest

    def vid(ii, jj):
        return jj * (N + 1) + ii

    v00 = np.stack([ci, cj], -1)
    v10 = v00 + [1, 0]
    v11 = v00 + [1, 1]
    v01 = v00 + [0, 1]
    t1 = np.stack([v00, v10, v11], 1)             # (cells, 3, 2)
    t2 = np.stack([v00, v11, v01], 1)
    lat = np.stack([t1, t2], 1).reshape(-1, 3, 2)  # element e = 2*cell + t
    vidx = vid(lat[..., 0], lat[..., 1])
    return _build_lagrange_mesh(2, p, N, vert_xyz, vidx, lat, f"tri_P{p}_N{N}")


_PERMS = list(itertools.permutations(range(3)))


def _perm_sign(pm):
    s = 1
    for a in range(3):
        for b in range(a + 1, 3):
            if pm[a] > pm[b]:
                s = -s
    return s


def structured_tet(N: int, p: int = 1, alpha: float = 0.15, seed: int = 0) -> Mesh:
    """Unit cube, N^3 cubes, each split into the six Kuhn tetrahedra (paths
    from corner (0,0,0) to (1,1,1) along the axis permutations), positively
    oriented: 6 N^3 elements, (pN+1)^3 dofs."""
    h = 1.0 / N
    (rng,) = _seeds(seed, 1)
    k, j, i = np.meshgrid(np.arange(N + 1), np.arange(N + 1), np.arange(N + 1), indexing="ij")
    xyz = np.stack([i * h, j * h, k * h], axis=-1).astype(np.float64)  # [z, y, x, 3]
    if alpha:
        xyz = xyz + _jitter_vertices((N + 1,) * 3, h, alpha, rng)
    vert_xyz = xyz.reshape(-1, 3)
    ck, cj, ci = np.meshgrid(np.arange(N), np.arange(N), np.arange(N), indexing="ij")
    c0 = np.stack([ci.ravel(), cj.ravel(), ck.ravel()], -1)  # cube order z, y, x fastest
    eye = np.eye(3, dtype=np.int64)
    tets = []
    for pm in _PERMS:
        v0 = c0
        v1 = v0 + eye[pm[0]]
        v2 = v1 + eye[pm[1]]
        v3 = v2 + eye[pm[2]]
        if _perm_sign(pm) > 0:
            tets.append(np.stack([v0, v1, v2, v3], 1))
        else:
            tets.append(np.stack([v0, v2, v1, v3], 1))
    lat = np.stack(tets, 1).reshape(-1, 4, 3)     # element e = 6*cube + t
    vidx = (lat[..., 2] * (N + 1) + lat[..., 1]) * (N + 1) + lat[..., 0]
    return _build_lagrange_mesh(3, p, N, vert_xyz, vidx, lat, f"tet_P{p}_N{N}")


def sliver_tri(N: int = 8, frac: float = 0.05, seed: int = 0, pull: float = 1e-5) -> Mesh:
    """A jitter-free structured P1 triangle mesh with near-degenerate
    (sliver) elements: for selected cells (i, j) the vertex (i+1, j) is moved
    to within ``pull*h`` of the cell's diagonal (i,j)-(i+1,j+1), which makes
    the cell's first triangle a sliver and keeps every other element valid.
    Selected vertices are two cells apart so their moves do not interact."""
    m = structured_tri(N, 1, alpha=0.0, seed=seed)
    rng = np.random.default_rng(seed)
    h = 1.0 / N
    coords = m.coords.copy()
    cand = [(i, j) for j in range(1, N - 1, 2) for i in range(0, N - 2, 2)]
    nsel = max(1, int(round(frac * len(cand))))
    sel = rng.choice(len(cand), size=min(nsel, len(cand)), replace=False)
    for s in sel:
        i, j = cand[s]
        v = j * (N + 1) + (i + 1)
        coords[v] = np.array([(i + 0.5) * h, (j + 0.5) * h]) + pull * h * np.array([1.0, -1.0]) / math.sqrt(2.0)
    return Mesh(d=2, p=1, coords=coords, conn=m.conn, name=f"sliver_N{N}")


def fan_tri(K: int = 300, seed: int = 0) -> Mesh:
    """P1 triangles (0, i, i+1) around a centre node 0, ring nodes 1..K on
    a circle of radius 1 with a small radial jitter: the centre's row has
    K+1 entries (long rows exercise the code paths for rows of more than 256
    entries)."""
    rng = np.random.default_rng(seed)
    th = 2.0 * math.pi * np.arange(K) / K
    r = 1.0 + rng.uniform(-0.05, 0.05, K)
    coords = np.vstack([[0.0, 0.0], np.stack([r * np.cos(th), r * np.sin(th)], 1)])
    i = np.arange(K)
    conn = np.stack([np.zeros(K, dtype=np.int64), 1 + i, 1 + (i + 1) % K], 1).astype(np.int32)
    return Mesh(d=2, p=1, coords=coords, conn=conn, name=f"fan_{K}")


def uniform_field(n: int, seed: int) -> np.ndarray:
    """Nodal values drawn independently from U[0,1]."""
    return np.random.default_rng(seed).uniform(0.0, 1.0, n)


def fourier_field(coords: np.ndarray, seed: int, modes: int = 8) -> np.ndarray:
    """Smooth random field with values in [0,1]:
    u(x) = 1/2 + 1/2 * sum_m a_m sin(2 pi k_m.x + theta_m) / sum_m |a_m|,
    a_m ~ U(0,1), k_m in {1..4}^d, theta_m ~ U(0, 2pi)."""
    rng = np.random.default_rng(seed)
    d = coords.shape[1]
    a = rng.uniform(0.0, 1.0, modes)
    kv = rng.integers(1, 5, size=(modes, d))
    th = rng.uniform(0.0, 2.0 * math.pi, modes)
    s = np.zeros(coords.shape[0])
    for m in range(modes):
        s += a[m] * np.sin(2.0 * math.pi * (coords @ kv[m]) + th[m])
    return 0.5 + 0.5 * s / np.sum(np.abs(a))


@dataclass
class Coeff:
    """Conductivity law k(u).  kind: 'poly' (params = c0..c4, k = sum c_i u^i),
    'sin' (params = alpha, beta, gamma: k = alpha + beta sin(gamma u)),
    'pwlin' (params = knots t_0..t_{m-1} followed by values k_0..k_{m-1};
    linear between knots, constant outside, a knot belongs to the branch on
    its left)."""
    kind: str
    params: tuple

    def numpy(self) -> np.ndarray:
        return np.asarray(self.params, dtype=np.float64)


@dataclass
class Workload:
    name: str
    mesh: Mesh
    u: np.ndarray
    coeff: Coeff
    mass_coeff: float = 1.0
    extra: dict = field(default_factory=dict)


def workload(name: str, scale: int | None = None) -> Workload:
    """The synthetic workloads, by name.  ``scale`` overrides the grid size N
    (for reduced-size parity runs with the same recipe).

    * ``tri_p1_64``: unit square 64x64 cells, 8 192 P1 triangles, jitter
      0.2h, u ~ U[0,1], k = 1 + 0.5u + 0.25u^2.  Seed 1.
    * ``tri_p2_1024``: 1024x1024 cells, 2 097 152 P2 triangles, jitter 0.2h,
      u = 8-mode Fourier field, k = 1 + u^2.  Seed 2.
    * ``tet_p1_128``: 128^3 cubes, 12 582 912 P1 tetrahedra, jitter 0.15h,
      u = Fourier field, k = 2 + sin(3u).  Seed 3.
    * ``tet_p2_64``: 64^3 cubes, 1 572 864 P2 tetrahedra, otherwise as
      tet_p1_128.  Seed 3.
    * ``tet_p3_32``: 32^3 cubes, 196 608 P3 tetrahedra (20 dofs, 24-point
      rule), otherwise as tet_p1_128.  Seed 3.
    """
    if name == "tri_p1_64":
        N = scale or 64
        s_mesh, s_u = np.random.SeedSequence(1).spawn(2)
        m = structured_tri(N, 1, 0.2, seed=int(s_mesh.generate_state(1)[0]))
        u = uniform_field(m.n_nodes, int(s_u.generate_state(1)[0]))
        return Workload(name, m, u, Coeff("poly", (1.0, 0.5, 0.25, 0.0, 0.0)))
    if name == "tri_p2_1024":
        N = scale or 1024
        s_mesh, s_u = np.random.SeedSequence(2).spawn(2)
        m = structured_tri(N, 2, 0.2, seed=int(s_mesh.generate_state(1)[0]))
        u = fourier_field(m.coords, int(s_u.generate_state(1)[0]))
        return Workload(name, m, u, Coeff("poly", (1.0, 0.0, 1.0, 0.0, 0.0)))
    if name in ("tet_p1_128", "tet_p2_64", "tet_p3_32"):
        p = {"tet_p1_128": 1, "tet_p2_64": 2, "tet_p3_32": 3}[name]
        N = scale or {1: 128, 2: 64, 3: 32}[p]
        s_mesh, s_u = np.random.SeedSequence(3).spawn(2)
        m = structured_tet(N, p, 0.15, seed=int(s_mesh.generate_state(1)[0]))
        u = fourier_field(m.coords, int(s_u.generate_state(1)[0]))
        return Workload(name, m, u, Coeff("sin", (2.0, 1.0, 3.0)))
    raise KeyError(name)


def sweep_field(wl: Workload, s: int) -> np.ndarray:
    """The s-th iterate of a Newton-style sweep on a workload: a fresh Fourier
    field with seed 3+s."""
    return fourier_field(wl.mesh.coords, 3 + s)


def batched_meshes(count: int = 64, seed: int = 4, e_min: float = 1e3, e_max: float = 2e5,
                   types=None):
    """Meshes of uneven size and type for a batched launch.  Each mesh draws a
    type (d, p) uniformly from ``types`` (default {2,3} x {1,2,3}) and a target
    element count log-uniform in [e_min, e_max]; the grid size is
    round(sqrt(E/2)) in 2D, round(cbrt(E/6)) in 3D (at least 1).  Each mesh
    gets its own Fourier field and k = 1 + a u + b u^2 with (a,b) ~ U[0,1]^2."""
    types = types or [(2, 1), (2, 2), (2, 3), (3, 1), (3, 2), (3, 3)]
    rng = np.random.default_rng(seed)
    out = []
    for idx in range(count):
        d, p = types[int(rng.integers(0, len(types)))]
        e_t = math.exp(rng.uniform(math.log(e_min), math.log(e_max)))
        N = max(1, int(round(math.sqrt(e_t / 2.0)))) if d == 2 else max(1, int(round((e_t / 6.0) ** (1 / 3))))
        ms = int(rng.integers(0, 2**31 - 1))
        mesh = structured_tri(N, p, 0.2, seed=ms) if d == 2 else structured_tet(N, p, 0.15, seed=ms)
        u = fourier_field(mesh.coords, ms + 1)
        a, b = rng.uniform(0.0, 1.0, 2)
        out.append(Workload(f"batch{idx}_{mesh.name}", mesh, u, Coeff("poly", (1.0, float(a), float(b), 0.0, 0.0))))
    return out


def curved(mesh: Mesh, amp: float = 0.1, seed: int = 0) -> Mesh:
    """A copy with curved elements for isoparametric mappings: every
    higher-order node (edge, face, interior) off the domain's boundary is
    moved by a smooth random field of size amp * h / p (h the mean edge
    length of the first element); vertices and nodes on the boundary stay, so
    neighbouring elements still share their curved sides and the elements
    still tile the unit square / cube."""
    d = mesh.d
    X = mesh.coords.copy()
    verts = np.unique(mesh.conn[:, : d + 1])
    ho = np.ones(mesh.n_nodes, dtype=bool)
    ho[verts] = False
    inner = np.all((X > 1e-12) & (X < 1 - 1e-12), axis=1)
    move = ho & inner
    v0 = mesh.coords[mesh.conn[0, : d + 1]]
    h = float(np.mean([np.linalg.norm(v0[a] - v0[b]) for a in range(d + 1) for b in range(a + 1, d + 1)]))
    rng = np.random.default_rng(seed)
    k = rng.integers(1, 3, size=(d, d))
    ph = rng.uniform(0, 2 * np.pi, size=d)
    disp = np.stack([np.sin(2 * np.pi * (X @ k[a]) + ph[a]) for a in range(d)], axis=1)
    X[move] += amp * h / mesh.p * disp[move]
    return Mesh(d=d, p=mesh.p, coords=X, conn=mesh.conn.copy(), name=mesh.name + "_curved")
