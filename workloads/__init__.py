"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds geometry and random-number generation only: closed
triangle meshes (geodesic spheres, concentric spheres, a closed box slab),
plane-wave directions and polarisations, and seeded complex vectors.  It
contains none of the boundary-element arithmetic (no basis functions, no
Green's functions, no quadrature), so both the CUDA path and the CPU oracle
may consume what it produces without sharing any of the method's code.

Every mesh is returned as ``(verts, tris)``: ``verts`` a float64 array of
shape (nv, 3) and ``tris`` an int32 array of shape (nt, 3) whose vertex order
is counter-clockwise seen from outside (outward normals).  The meshes are the
surface discretisations of the workloads in the paper's setting (a closed,
penetrable body in free space, Sec. III) lifted to three dimensions.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "icosahedron",
    "icosphere",
    "geodesic_sphere",
    "concentric_spheres",
    "coated_sphere",
    "box_mesh",
    "fibonacci_directions",
    "plane_wave_batch",
    "complex_normal",
    "uneven_sphere_batch",
    "circle_polygon",
    "ellipse_polygon",
    "airfoil_polygon",
]


def icosahedron():
    """Regular icosahedron with vertices on the unit sphere.

    Faces are found as the vertex triples that are pairwise at the minimum
    distance, then oriented so that their normal points away from the centre.
    """
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    v = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            v.append((0.0, s1, s2 * phi))
            v.append((s1, s2 * phi, 0.0))
            v.append((s2 * phi, 0.0, s1))
    v = np.array(v, dtype=np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    nv = len(v)
    d = np.linalg.norm(v[:, None, :] - v[None, :, :], axis=2)
    dmin = d[d > 1e-9].min()
    adj = np.abs(d - dmin) < 1e-9
    faces = []
    for a in range(nv):
        for b in range(a + 1, nv):
            if not adj[a, b]:
                continue
            for c in range(b + 1, nv):
                if adj[a, c] and adj[b, c]:
                    n = np.cross(v[b] - v[a], v[c] - v[a])
                    if np.dot(n, v[a] + v[b] + v[c]) > 0:
                        faces.append((a, b, c))
                    else:
                        faces.append((a, c, b))
    tris = np.array(faces, dtype=np.int32)
    assert tris.shape == (20, 3)
    return v, tris


def _subdivide(verts, tris):
    """Split every triangle into four through its edge midpoints."""
    verts = [tuple(p) for p in verts]
    cache = {}

    def mid(a, b):
        key = (a, b) if a < b else (b, a)
        idx = cache.get(key)
        if idx is None:
            pa = np.array(verts[a])
            pb = np.array(verts[b])
            verts.append(tuple(0.5 * (pa + pb)))
            idx = len(verts) - 1
            cache[key] = idx
        return idx

    out = []
    for a, b, c in tris:
        a, b, c = int(a), int(b), int(c)
        ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
        out += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
    return np.array(verts, dtype=np.float64), np.array(out, dtype=np.int32)


def icosphere(level: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)):
    """Icosahedron refined ``level`` times by 1-to-4 splits, vertices on the sphere.

    ``20 * 4**level`` triangles, ``30 * 4**level`` edges.  The circumscribed
    radius is ``radius`` (every vertex lies on the sphere).
    """
    v, t = icosahedron()
    for _ in range(level):
        v, t = _subdivide(v, t)
        v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v * radius + np.asarray(center, dtype=np.float64), t


def geodesic_sphere(freq: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)):
    """Class-I geodesic sphere of frequency ``freq``: ``20 * freq**2`` triangles.

    Each icosahedron face is split into ``freq**2`` triangles on a regular
    barycentric lattice, then the lattice points are projected on the sphere.
    """
    if freq < 1:
        raise ValueError("freq must be >= 1")
    v0, t0 = icosahedron()
    verts = []
    index = {}

    def vid(p):
        key = tuple(np.round(p * 1e12).astype(np.int64))
        i = index.get(key)
        if i is None:
            verts.append(p)
            i = len(verts) - 1
            index[key] = i
        return i

    tris = []
    for a, b, c in t0:
        A, B, C = v0[a], v0[b], v0[c]
        grid = {}
        for i in range(freq + 1):
            for j in range(freq + 1 - i):
                k = freq - i - j
                p = (i * A + j * B + k * C) / freq
                p = p / np.linalg.norm(p)
                grid[(i, j)] = vid(p)
        for i in range(freq):
            for j in range(freq - i):
                # upward triangle
                tris.append((grid[(i + 1, j)], grid[(i, j + 1)], grid[(i, j)]))
                if i + j < freq - 1:
                    tris.append((grid[(i + 1, j)], grid[(i + 1, j + 1)], grid[(i, j + 1)]))
    verts = np.array(verts, dtype=np.float64)
    tris = np.array(tris, dtype=np.int32)
    # orient every face outward
    e1 = verts[tris[:, 1]] - verts[tris[:, 0]]
    e2 = verts[tris[:, 2]] - verts[tris[:, 0]]
    cen = verts[tris].mean(axis=1)
    flip = np.einsum("ij,ij->i", np.cross(e1, e2), cen) < 0
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return verts * radius + np.asarray(center, dtype=np.float64), tris


def concentric_spheres(level_outer: int, radius_outer: float, level_inner: int, radius_inner: float):
    """Two nested icospheres; the inner one is returned as a separate mesh."""
    return icosphere(level_outer, radius_outer), icosphere(level_inner, radius_inner)


def coated_sphere(level_outer: int, radius_outer: float, level_inner: int, radius_inner: float):
    """A coated sphere as one mesh of two surfaces, with the regions each triangle separates.

    Returns (verts, tris, tri_regions): the outer icosphere's vertices and
    triangles first, then the inner one's (indices shifted), and tri_regions
    (nt, 2) int32 = (region on the normal side, region behind): (0, 1) on the
    outer surface (exterior / coating), (1, 2) on the inner one (coating / core).
    """
    (vo, to), (vi, ti) = concentric_spheres(level_outer, radius_outer, level_inner, radius_inner)
    verts = np.concatenate([vo, vi])
    tris = np.concatenate([to, ti + len(vo)]).astype(np.int32)
    regions = np.concatenate([np.tile([0, 1], (len(to), 1)), np.tile([1, 2], (len(ti), 1))]).astype(np.int32)
    return verts, tris, regions


def box_mesh(lx: float, ly: float, lz: float, nx: int, ny: int, nz: int):
    """Closed box [0,lx]x[0,ly]x[0,lz], structured faces, alternating diagonals.

    Face cells are split into two triangles along a diagonal whose direction
    alternates with the parity of the cell index.  ``4*(nx*ny+nx*nz+ny*nz)``
    triangles; vertices on the box edges are shared, so the surface is closed.
    """
    index = {}
    verts = []

    def vid(i, j, k):
        key = (i, j, k)
        v = index.get(key)
        if v is None:
            verts.append((lx * i / nx, ly * j / ny, lz * k / nz))
            v = len(verts) - 1
            index[key] = v
        return v

    tris = []

    def face(fixed_axis, fixed_val, a_axis, na, b_axis, nb, outward):
        for ia in range(na):
            for ib in range(nb):
                q = []
                for da, db in ((0, 0), (1, 0), (1, 1), (0, 1)):
                    c = [0, 0, 0]
                    c[fixed_axis] = fixed_val
                    c[a_axis] = ia + da
                    c[b_axis] = ib + db
                    q.append(vid(*c))
                if (ia + ib) % 2 == 0:
                    t1, t2 = (q[0], q[1], q[2]), (q[0], q[2], q[3])
                else:
                    t1, t2 = (q[0], q[1], q[3]), (q[1], q[2], q[3])
                tris.append(t1)
                tris.append(t2)

    n = (nx, ny, nz)
    for axis in range(3):
        a_axis, b_axis = [ax for ax in range(3) if ax != axis]
        face(axis, 0, a_axis, n[a_axis], b_axis, n[b_axis], False)
        face(axis, n[axis], a_axis, n[a_axis], b_axis, n[b_axis], True)
    verts = np.array(verts, dtype=np.float64)
    tris = np.array(tris, dtype=np.int32)
    e1 = verts[tris[:, 1]] - verts[tris[:, 0]]
    e2 = verts[tris[:, 2]] - verts[tris[:, 0]]
    cen = verts[tris].mean(axis=1) - np.array([lx, ly, lz]) / 2.0
    flip = np.einsum("ij,ij->i", np.cross(e1, e2), cen) < 0
    tris[flip] = tris[flip][:, [0, 2, 1]]
    return verts, tris


def fibonacci_directions(n: int):
    """Unit vectors on a Fibonacci sphere: z_i = 1-(2i+1)/n, phi_i = i*pi*(3-sqrt 5)."""
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - (2.0 * i + 1.0) / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    phi = i * math.pi * (3.0 - math.sqrt(5.0))
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def plane_wave_batch(n: int, seed: int = 0):
    """``n`` plane waves: Fibonacci directions, random polarisation angle.

    Returns ``(khat, e0)``: khat (n,3) float64 unit propagation directions and
    e0 (n,3) complex128 unit polarisation vectors orthogonal to khat, rotated
    by an angle psi ~ U[0, 2pi) drawn from ``numpy.random.default_rng(seed)``.
    """
    khat = fibonacci_directions(n)
    rng = np.random.default_rng(seed)
    psi = rng.uniform(0.0, 2.0 * math.pi, size=n)
    ref = np.where(np.abs(khat[:, 2:3]) < 0.9, np.array([[0.0, 0.0, 1.0]]), np.array([[1.0, 0.0, 0.0]]))
    u = np.cross(khat, ref)
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    w = np.cross(khat, u)
    e0 = np.cos(psi)[:, None] * u + np.sin(psi)[:, None] * w
    return khat, e0.astype(np.complex128)


def complex_normal(n: int, seed: int = 0, nrhs: int | None = None):
    """Seeded complex standard normal vector (or n x nrhs matrix), complex128."""
    rng = np.random.default_rng(seed)
    shape = (n,) if nrhs is None else (n, nrhs)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2.0)


def uneven_sphere_batch(count: int = 16, seed: int = 1):
    """Geodesic spheres of uneven size with random radius, k0 and permittivity.

    freq ~ U{8..32} (1280..20480 triangles), radius ~ U[0.5, 2],
    k0 = U[2, 10] / radius, eps_r = U[2, 5] + j U[-3, -1].
    Returns a list of dicts with keys freq, radius, k0, eps_r.
    """
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(count):
        freq = int(rng.integers(8, 33))
        radius = float(rng.uniform(0.5, 2.0))
        k0 = float(rng.uniform(2.0, 10.0)) / radius
        eps = complex(rng.uniform(2.0, 5.0), rng.uniform(-3.0, -1.0))
        out.append({"freq": freq, "radius": radius, "k0": k0, "eps_r": eps})
    return out


# ---------------------------------------------------------------------------
# closed curves of the two-dimensional (z-invariant) setting
# ---------------------------------------------------------------------------
def _equal_arc(points_of, n: int, samples: int = 1 << 18):
    """n points equally spaced in arc length along the closed parametric curve
    points_of(theta), theta in [0, 2 pi); returns (n, 2) float64, starting at theta = 0."""
    th = np.linspace(0.0, 2.0 * math.pi, samples + 1)
    p = points_of(th)
    seg = np.hypot(np.diff(p[:, 0]), np.diff(p[:, 1]))
    s = np.concatenate([[0.0], np.cumsum(seg)])
    target = np.arange(n) * (s[-1] / n)
    t = np.interp(target, s, th)
    return points_of(t)


def circle_polygon(n: int, radius: float = 1.0):
    """Regular n-gon inscribed in the circle of the given radius, counter-clockwise,
    first vertex on the +x axis."""
    th = 2.0 * math.pi * np.arange(n) / n
    return np.stack([radius * np.cos(th), radius * np.sin(th)], axis=1)


def ellipse_polygon(n: int, aspect: float = 1.5, perimeter: float = 2.0 * math.pi):
    """n vertices equally spaced in arc length on the ellipse with semi-axes
    (aspect * b, b) whose perimeter is ``perimeter``; counter-clockwise."""
    unit = lambda th: np.stack([aspect * np.cos(th), np.sin(th)], axis=-1)  # noqa: E731
    th = np.linspace(0.0, 2.0 * math.pi, (1 << 18) + 1)
    p = unit(th)
    per1 = float(np.sum(np.hypot(np.diff(p[:, 0]), np.diff(p[:, 1]))))
    b = perimeter / per1
    return _equal_arc(lambda t: b * unit(t), n)


def airfoil_polygon(n: int, perimeter: float = 2.0 * math.pi, center=(-0.08, 0.08), swell: float = 1.05):
    """Joukowsky airfoil: the image w = z + 1/z of the circle of centre ``center``
    and radius swell * |1 - center| (swell > 1 rounds the trailing edge), scaled
    to the given perimeter, n vertices equally spaced in arc length,
    counter-clockwise."""
    c = complex(*center)
    rho = swell * abs(1.0 - c)

    def raw(th):
        z = c + rho * np.exp(1j * th)
        w = z + 1.0 / z
        return np.stack([w.real, w.imag], axis=-1)

    th = np.linspace(0.0, 2.0 * math.pi, (1 << 18) + 1)
    p = raw(th)
    per1 = float(np.sum(np.hypot(np.diff(p[:, 0]), np.diff(p[:, 1]))))
    pts = _equal_arc(lambda t: raw(t) * (perimeter / per1), n)
    area2 = float(np.sum(pts[:, 0] * np.roll(pts[:, 1], -1) - np.roll(pts[:, 0], -1) * pts[:, 1]))
    return pts if area2 > 0 else pts[::-1].copy()
