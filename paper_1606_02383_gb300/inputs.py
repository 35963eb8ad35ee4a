"""Seeded synthetic inputs shared by the oracle tests, the GPU tests and the bench.

This module holds no arithmetic of the boundary element method itself: it only
makes surface meshes (vertex coordinates + triangle connectivity) and random
complex densities, exactly as a user of the library would before calling it.
Both the CPU oracle and the CUDA path take these arrays as plain inputs.

Conventions (Section 2.1 of the paper, "n is the exterior normal of the elastic
region"): every triangle (a, b, c) is ordered so that (b - a) x (c - a) points
out of the scatterer, into the fluid.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "ball_tets",
    "voxel_body",
    "voxel_ball",
    "icosphere",
    "ellipsoid",
    "torus",
    "batch_bodies",
    "level_set_mesh",
    "translate_scale",
    "merge_meshes",
    "random_density",
    "plane_wave",
    "large_multibody",
]


def _icosahedron():
    t = (1.0 + 5.0 ** 0.5) / 2.0
    v = np.array(
        [[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
         [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
         [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], dtype=np.float64)
    f = np.array(
        [[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
         [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
         [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
         [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], dtype=np.int64)
    return v / np.linalg.norm(v, axis=1, keepdims=True), f


def _orient_outward(v, f, centre):
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    nrm = np.cross(b - a, c - a)
    flip = np.einsum("ij,ij->i", nrm, (a + b + c) / 3.0 - centre) < 0
    f = f.copy()
    f[flip, 1], f[flip, 2] = f[flip, 2], f[flip, 1].copy()
    return f


def icosphere(level: int, radius: float = 1.0, centre=(0.0, 0.0, 0.0)):
    """Icosahedron subdivided `level` times (20 * 4**level triangles), projected
    onto the sphere of the given radius. Returns (vertices float64 [nv,3],
    triangles int32 [nt,3]) with outward orientation."""
    v, f = _icosahedron()
    for _ in range(level):
        nv = v.shape[0]
        e = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]], axis=0)
        e = np.sort(e, axis=1)
        key = e[:, 0] * (nv + 1) + e[:, 1]
        ukey, inv = np.unique(key, return_inverse=True)
        ua, ub = ukey // (nv + 1), ukey % (nv + 1)
        mid = v[ua] + v[ub]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        nf = f.shape[0]
        m01 = nv + inv[0:nf]
        m12 = nv + inv[nf:2 * nf]
        m20 = nv + inv[2 * nf:3 * nf]
        v = np.concatenate([v, mid], axis=0)
        f = np.concatenate([
            np.stack([f[:, 0], m01, m20], axis=1),
            np.stack([m01, f[:, 1], m12], axis=1),
            np.stack([m20, m12, f[:, 2]], axis=1),
            np.stack([m01, m12, m20], axis=1)], axis=0)
    f = _orient_outward(v, f, np.zeros(3))
    v = v * float(radius) + np.asarray(centre, dtype=np.float64)[None, :]
    return np.ascontiguousarray(v), np.ascontiguousarray(f.astype(np.int32))


def _orient_by_direction(v, f, outward):
    a, b, c = v[f[:, 0]], v[f[:, 1]], v[f[:, 2]]
    nrm = np.cross(b - a, c - a)
    flip = np.einsum("ij,ij->i", nrm, outward) < 0
    f = f.copy()
    f[flip, 1], f[flip, 2] = f[flip, 2], f[flip, 1].copy()
    return f


def ellipsoid(n: int, axes=(1.0, 1.0, 1.0), centre=(0.0, 0.0, 0.0)):
    """Cube-sphere: each cube face split into n x n squares (two triangles
    each, 12 n^2 triangles), projected onto the unit sphere and scaled by the
    semi-axes."""
    g = np.linspace(-1.0, 1.0, n + 1)
    U, W = np.meshgrid(g, g, indexing="ij")
    verts, faces, off = [], [], 0
    for axis in range(3):
        for sign in (-1.0, 1.0):
            P = np.zeros((n + 1, n + 1, 3))
            P[..., axis] = sign
            P[..., (axis + 1) % 3] = U
            P[..., (axis + 2) % 3] = W
            verts.append(P.reshape(-1, 3))
            idx = np.arange((n + 1) * (n + 1)).reshape(n + 1, n + 1) + off
            a, b, c, d = idx[:-1, :-1], idx[1:, :-1], idx[1:, 1:], idx[:-1, 1:]
            faces.append(np.stack([a, b, c], -1).reshape(-1, 3))
            faces.append(np.stack([a, c, d], -1).reshape(-1, 3))
            off += (n + 1) * (n + 1)
    v = np.concatenate(verts)
    f = np.concatenate(faces)
    key = np.round(v * 1e9).astype(np.int64)
    _, first, inv = np.unique(key, axis=0, return_index=True, return_inverse=True)
    v = v[first]
    f = inv.reshape(-1)[f]
    v = v / np.linalg.norm(v, axis=1, keepdims=True)
    f = _orient_by_direction(v, f, (v[f[:, 0]] + v[f[:, 1]] + v[f[:, 2]]) / 3.0)
    v = v * np.asarray(axes, dtype=np.float64)[None, :] + np.asarray(centre, dtype=np.float64)[None, :]
    return np.ascontiguousarray(v), np.ascontiguousarray(f.astype(np.int32))


def torus(nu: int, nv: int, R: float = 1.0, r: float = 0.3, centre=(0.0, 0.0, 0.0)):
    """Torus of major radius R and minor radius r on an nu x nv (u, v) grid
    (2 nu nv triangles), oriented away from the tube's centre line."""
    u = 2 * np.pi * np.arange(nu) / nu
    w = 2 * np.pi * np.arange(nv) / nv
    Uu, Ww = np.meshgrid(u, w, indexing="ij")
    v = np.stack([(R + r * np.cos(Ww)) * np.cos(Uu), (R + r * np.cos(Ww)) * np.sin(Uu), r * np.sin(Ww)], -1)
    v = v.reshape(-1, 3)
    idx = np.arange(nu * nv).reshape(nu, nv)
    a = idx
    b = np.roll(idx, -1, axis=0)
    c = np.roll(np.roll(idx, -1, axis=0), -1, axis=1)
    d = np.roll(idx, -1, axis=1)
    f = np.concatenate([np.stack([a, b, c], -1).reshape(-1, 3), np.stack([a, c, d], -1).reshape(-1, 3)])
    cen = (v[f[:, 0]] + v[f[:, 1]] + v[f[:, 2]]) / 3.0
    ring = cen.copy()
    ring[:, 2] = 0.0
    ring = R * ring / np.linalg.norm(ring, axis=1, keepdims=True)
    f = _orient_by_direction(v, f, cen - ring)
    v = v + np.asarray(centre, dtype=np.float64)[None, :]
    return np.ascontiguousarray(v), np.ascontiguousarray(f.astype(np.int32))


def batch_bodies(count: int = 64, seed: int = 0, n_min: int = 2000, n_max: int = 50000):
    """The batching workload: `count` independent scatterers, half ellipsoids
    (semi-axes uniform in [0.5, 2]) and half tori (R = 1, r uniform in
    [0.2, 0.5]), triangle counts log-uniform in [n_min, n_max], wavenumbers
    uniform in [1, 8].  Returns a list of (vertices, triangles, k)."""
    rng = np.random.Generator(np.random.PCG64([int(seed), 3]))
    out = []
    for b in range(count):
        target = float(np.exp(rng.uniform(np.log(n_min), np.log(n_max))))
        k = float(rng.uniform(1.0, 8.0))
        if b % 2 == 0:
            axes = rng.uniform(0.5, 2.0, size=3)
            n = max(2, int(round(np.sqrt(target / 12.0))))
            V, T = ellipsoid(n, axes)
        else:
            r = float(rng.uniform(0.2, 0.5))
            nv = max(3, int(round(np.sqrt(target / 2.0 * r))))
            nu = max(3, int(round(target / (2.0 * nv))))
            V, T = torus(nu, nv, 1.0, r)
        out.append((V, T, k))
    return out


def _marching_tets(phi, lo, h, t):
    """Iso-surface phi = t of a grid function by marching tetrahedra.

    Every cube splits into the 6 tetrahedra that run from corner (0,0,0) to
    (1,1,1) along the 6 orders of the axes (a conforming split).  A tetrahedron
    with 1 or 3 corners inside (phi > t) contributes one triangle, with 2 a
    quadrilateral cut into two; cut points sit on the crossing edges at the
    linear-interpolation zero and are shared through their grid edge, so the
    surface is closed.  Triangles face from the inside corners to the outside
    ones, i.e. out of the region phi > t.  Cut points are kept 2% of an edge
    away from the grid vertices so that no triangle degenerates."""
    n0, n1, n2 = phi.shape
    I, J, K = np.meshgrid(np.arange(n0 - 1), np.arange(n1 - 1), np.arange(n2 - 1), indexing="ij")
    base = np.stack([I.ravel(), J.ravel(), K.ravel()], -1)
    unit = np.eye(3, dtype=np.int64)
    tets = []
    for perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
        c0 = np.zeros(3, np.int64)
        c1 = unit[perm[0]]
        c2 = c1 + unit[perm[1]]
        c3 = c2 + unit[perm[2]]
        tets.append(np.stack([base + c for c in (c0, c1, c2, c3)], 1))
    tet = np.concatenate(tets)                                        # [ntet, 4, 3]
    gid = (tet[..., 0] * n1 + tet[..., 1]) * n2 + tet[..., 2]        # [ntet, 4]
    val = phi.ravel()[gid]
    inside = val > t
    nin = inside.sum(1)
    keep = (nin > 0) & (nin < 4)
    tet, gid, val, inside, nin = tet[keep], gid[keep], val[keep], inside[keep], nin[keep]
    pos = lo + tet.astype(np.float64) * h
    verts_key, verts_xyz, faces = {}, [], []

    def cut(i, a, b):  # point on edge (a, b) of tetrahedron i
        ga, gb = gid[i, a], gid[i, b]
        key = (min(ga, gb), max(ga, gb))
        idx = verts_key.get(key)
        if idx is None:
            fa, fb = val[i, a], val[i, b]
            # kept away from the grid vertices so no cut edge degenerates
            s_ = min(max((t - fa) / (fb - fa), 0.02), 0.98)
            verts_xyz.append(pos[i, a] + s_ * (pos[i, b] - pos[i, a]))
            idx = len(verts_xyz) - 1
            verts_key[key] = idx
        return idx

    for i in range(tet.shape[0]):
        ins = [a for a in range(4) if inside[i, a]]
        out = [a for a in range(4) if not inside[i, a]]
        if len(ins) == 1 or len(ins) == 3:
            lone, rest = (ins[0], out) if len(ins) == 1 else (out[0], ins)
            tri = [cut(i, lone, r) for r in rest]
            faces.append((tri, ins, out, i))
        else:
            a, b = ins
            c, d = out
            q = [cut(i, a, c), cut(i, a, d), cut(i, b, d), cut(i, b, c)]
            faces.append(([q[0], q[1], q[2]], ins, out, i))
            faces.append(([q[0], q[2], q[3]], ins, out, i))
    V = np.asarray(verts_xyz)
    F = np.asarray([f[0] for f in faces], dtype=np.int64)
    a, b, c = V[F[:, 0]], V[F[:, 1]], V[F[:, 2]]
    nrm = np.cross(b - a, c - a)
    area2 = np.linalg.norm(nrm, axis=1)
    away = np.asarray([pos[f[3], f[2]].mean(0) - pos[f[3], f[1]].mean(0) for f in faces])
    flip = np.einsum("ij,ij->i", nrm, away) < 0
    F[flip, 1], F[flip, 2] = F[flip, 2], F[flip, 1].copy()
    del area2
    return V, F


def level_set_gaussians(seed: int = 0, n_gauss: int = 20):
    """Centres c_i (uniform in [-1,1]^3) and widths w_i (uniform in [0.2, 0.5])
    of the level-set function phi(x) = sum_i exp(-|x - c_i|^2 / (2 w_i^2))."""
    rng = np.random.Generator(np.random.PCG64([int(seed), 4]))
    c = rng.uniform(-1.0, 1.0, size=(n_gauss, 3))
    w = rng.uniform(0.2, 0.5, size=n_gauss)
    return c, w


def level_set_function(seed: int = 0, n_gauss: int = 20, grid: int = 64):
    """(phi [grid]^3, lo, h): the level-set function on a grid^3 lattice over [-2,2]^3."""
    c, w = level_set_gaussians(seed, n_gauss)
    x = np.linspace(-2.0, 2.0, grid)
    X, Y, Z = np.meshgrid(x, x, x, indexing="ij")
    P = np.stack([X, Y, Z], -1)
    phi = np.zeros(X.shape)
    for i in range(n_gauss):
        phi += np.exp(-np.sum((P - c[i]) ** 2, -1) / (2.0 * w[i] ** 2))
    return phi, np.array([-2.0, -2.0, -2.0]), x[1] - x[0]


def level_set_level(seed: int = 0, n_gauss: int = 20, grid: int = 64, target: int = 30000):
    """The iso-level (found by bisection) whose surface has about `target` triangles."""
    phi, _, _ = level_set_function(seed, n_gauss, grid)

    def count(t):  # triangles of the iso-surface at level t, without building it
        n0 = grid
        I, J, K = np.meshgrid(np.arange(n0 - 1), np.arange(n0 - 1), np.arange(n0 - 1), indexing="ij")
        base = np.stack([I.ravel(), J.ravel(), K.ravel()], -1)
        unit = np.eye(3, dtype=np.int64)
        tot = 0
        for perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
            cs = [np.zeros(3, np.int64), unit[perm[0]], unit[perm[0]] + unit[perm[1]], np.ones(3, np.int64)]
            nin = sum((phi[tuple((base + cc).T)] > t).astype(np.int64) for cc in cs)
            tot += int(np.sum((nin == 1) | (nin == 3)) + 2 * np.sum(nin == 2))
        return tot

    lo_t, hi_t = 1e-3, float(phi.max()) * 0.999
    for _ in range(40):
        mid = 0.5 * (lo_t + hi_t)
        if count(mid) > target:
            lo_t = mid
        else:
            hi_t = mid
    return 0.5 * (lo_t + hi_t)


def level_set_mesh(seed: int = 0, n_gauss: int = 20, grid: int = 64, target: int = 30000):
    """The differentiation workload's surface: the level set of
    phi(x) = sum_i exp(-|x - c_i|^2 / (2 w_i^2)) (c_i uniform in [-1,1]^3,
    w_i uniform in [0.2, 0.5]) on a grid^3 lattice over [-2,2]^3, at the
    iso-level (found by bisection) that gives about `target` triangles."""
    phi, lo, h = level_set_function(seed, n_gauss, grid)
    t = level_set_level(seed, n_gauss, grid, target)
    V, F = _marching_tets(phi, lo, h, t)
    return np.ascontiguousarray(V), np.ascontiguousarray(F.astype(np.int32))


def translate_scale(vertices, scale=1.0, shift=(0.0, 0.0, 0.0)):
    return np.ascontiguousarray(vertices * float(scale) + np.asarray(shift, dtype=np.float64)[None, :])


def merge_meshes(parts):
    """Concatenate several (vertices, triangles) meshes into one."""
    vs, fs, off = [], [], 0
    for v, f in parts:
        vs.append(v)
        fs.append(f.astype(np.int64) + off)
        off += v.shape[0]
    return (np.ascontiguousarray(np.concatenate(vs, axis=0)),
            np.ascontiguousarray(np.concatenate(fs, axis=0).astype(np.int32)))


def large_multibody(big_level: int = 7, small_level: int = 6):
    """Unit icosphere (level 7: 327,680 triangles) plus 8 icospheres of radius
    0.3 (level 6: 81,920 triangles each) centred at (+-1.5, +-1.5, +-1.5)."""
    parts = [icosphere(big_level, 1.0)]
    for sx in (-1.5, 1.5):
        for sy in (-1.5, 1.5):
            for sz in (-1.5, 1.5):
                parts.append(icosphere(small_level, 0.3, (sx, sy, sz)))
    return merge_meshes(parts)


def random_density(n: int, nrhs: int = 1, seed: int = 0, stream: int = 0, dtype=np.complex128):
    """Complex density with real and imaginary parts i.i.d. N(0,1), drawn from
    numpy's PCG64 seeded with (seed, stream). Shape [nrhs, n]."""
    rng = np.random.Generator(np.random.PCG64([int(seed), int(stream)]))
    re = rng.standard_normal((nrhs, n))
    im = rng.standard_normal((nrhs, n))
    return np.ascontiguousarray((re + 1j * im).astype(dtype))


def centroids(vertices, triangles):
    """Triangle centroids [nt, 3] (the collocation points), for building
    right-hand sides such as a plane wave sampled at the elements."""
    V = np.asarray(vertices, dtype=np.float64)
    T = np.asarray(triangles, dtype=np.int64)
    return V[T].mean(axis=1)


def plane_wave(points, k: float, direction=(0.0, 0.0, 1.0)):
    """exp(i k d.x) sampled at the given points (e.g. triangle centroids)."""
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    return np.exp(1j * float(k) * (np.asarray(points) @ d))


def voxel_body(mask, h: float = 1.0, origin=(0.0, 0.0, 0.0), jitter: float = 0.0, seed: int = 0):
    """Tetrahedra of the voxels where mask is true, for the elastic body of the
    coupled problem: every voxel is split into the six tetrahedra around its
    main diagonal (the same split in every voxel, so faces match), and the
    boundary faces (those of one tetrahedron only) form the surface mesh,
    normals out of the body.  Returns (nodes [n, 3] float64, tets [m, 4] int32
    with positive volume, tris [t, 3] int32); the surface uses the body's node
    numbering, so nodes and tris also make the BEM mesh.  jitter > 0 moves
    every node by up to jitter h per coordinate (seeded): on the exact lattice
    many centroid distances equal 2 or 4 longest edges, the thresholds of the
    near-singular rules, where two correct evaluations may pick different
    rules; moved nodes leave no such ties."""
    mask = np.asarray(mask, dtype=bool)
    n0, n1, n2 = mask.shape
    corner = np.zeros((n0 + 1, n1 + 1, n2 + 1), dtype=bool)
    for d0 in (0, 1):
        for d1 in (0, 1):
            for d2 in (0, 1):
                corner[d0:d0 + n0, d1:d1 + n1, d2:d2 + n2] |= mask
    ids = -np.ones(corner.shape, dtype=np.int64)
    pts = np.argwhere(corner)
    ids[tuple(pts.T)] = np.arange(pts.shape[0])
    nodes = np.asarray(origin, dtype=np.float64) + h * pts.astype(np.float64)
    if jitter > 0:
        nodes = nodes + jitter * h * np.random.default_rng(seed).uniform(-1.0, 1.0, nodes.shape)
    vox = np.argwhere(mask)
    unit = np.eye(3, dtype=np.int64)
    tets = []
    for perm in ((0, 1, 2), (0, 2, 1), (1, 0, 2), (1, 2, 0), (2, 0, 1), (2, 1, 0)):
        c0 = vox
        c1 = c0 + unit[perm[0]]
        c2 = c1 + unit[perm[1]]
        c3 = c2 + unit[perm[2]]
        tets.append(np.stack([ids[tuple(c.T)] for c in (c0, c1, c2, c3)], axis=1))
    tets = np.concatenate(tets)
    P = nodes[tets]
    vol = np.einsum("ij,ij->i", np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), P[:, 3] - P[:, 0])
    flip = vol < 0
    tets[flip, 2], tets[flip, 3] = tets[flip, 3].copy(), tets[flip, 2].copy()
    # the four faces of every tetrahedron with the opposite corner
    fidx = np.array([[1, 2, 3], [0, 2, 3], [0, 1, 3], [0, 1, 2]])
    faces = tets[:, fidx].reshape(-1, 3)
    opp = tets[:, [0, 1, 2, 3]].reshape(-1)
    key = np.sort(faces, axis=1)
    _, inv, cnt = np.unique(key, axis=0, return_inverse=True, return_counts=True)
    once = cnt[inv.ravel()] == 1
    faces, opp = faces[once], opp[once]
    a, b, c = nodes[faces[:, 0]], nodes[faces[:, 1]], nodes[faces[:, 2]]
    inward = np.einsum("ij,ij->i", np.cross(b - a, c - a), a - nodes[opp]) < 0
    faces[inward, 1], faces[inward, 2] = faces[inward, 2].copy(), faces[inward, 1].copy()
    return nodes, tets.astype(np.int32), faces.astype(np.int32)


def voxel_ball(n: int, radius: float, h: float = 1.0, jitter: float = 0.0, seed: int = 0):
    """The voxels of an n^3 lattice (spacing h, centred on the origin) whose
    centres lie within radius of the origin, as voxel_body's (nodes, tets, tris)."""
    g = (np.arange(n) - (n - 1) / 2.0) * h
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    mask = X ** 2 + Y ** 2 + Z ** 2 <= radius * radius
    return voxel_body(mask, h, origin=(-0.5 * n * h,) * 3, jitter=jitter, seed=seed)


def ball_tets(level: int, radius: float = 1.0, layers: int = 4):
    """Tetrahedra of a ball whose boundary is the level-`level` icosphere: the
    icosphere scaled to radii radius m / layers (m = 1 .. layers) and the
    centre; the centre and the innermost sphere's triangles make one
    tetrahedron each, and the prism between two spheres over a triangle with
    surface vertices a < b < c (a', b', c' one sphere out) is cut into
    (a, b, c, c'), (a, b, b', c'), (a, a', b', c'): every side face takes the
    diagonal from its lower-index inner vertex to its higher-index outer one,
    so neighbouring prisms match.  Returns (nodes, tets with positive volume,
    tris: the outer icosphere, normals out of the ball)."""
    Vs, Ts = icosphere(level, 1.0)
    nv = Vs.shape[0]
    nodes = [np.zeros((1, 3))]
    for m in range(1, layers + 1):
        nodes.append(Vs * (radius * m / layers))
    nodes = np.concatenate(nodes)

    def node(m, i):  # layer m (1-based) copy of surface vertex i
        return 1 + (m - 1) * nv + i

    tets = []
    for t in Ts:
        a, b, c = sorted(int(v) for v in t)
        tets.append([0, node(1, a), node(1, b), node(1, c)])
        for m in range(1, layers):
            A, B, C = node(m, a), node(m, b), node(m, c)
            A2, B2, C2 = node(m + 1, a), node(m + 1, b), node(m + 1, c)
            tets += [[A, B, C, C2], [A, B, B2, C2], [A, A2, B2, C2]]
    tets = np.asarray(tets, dtype=np.int64)
    P = nodes[tets]
    vol = np.einsum("ij,ij->i", np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]), P[:, 3] - P[:, 0])
    flip = vol < 0
    tets[flip, 2], tets[flip, 3] = tets[flip, 3].copy(), tets[flip, 2].copy()
    tris = (1 + (layers - 1) * nv + Ts).astype(np.int32)
    return nodes, tets.astype(np.int32), tris
