"""Triangulated closed surfaces used as inputs.

Every mesh is returned as ``(vertices, triangles)``: ``vertices`` a float64
array of shape (nv, 3), ``triangles`` an int32 array of shape (nt, 3) whose
rows list vertex ids counter-clockwise when seen from outside (outward
normals).  The meshes are conforming: neighbouring triangles share vertex
ids, which is what the singular-quadrature case split of Sect. 8 relies on
(identical / common edge / common vertex / disjoint).

The paper's experiments use polygonal approximations of the unit sphere
(Sect. 2, Fig. 1 and Fig. 8).  The generators here are:

* ``icosphere(L)``: the icosahedron refined L times by edge midpoints,
  new vertices projected to the unit sphere; n = 20 * 4**L triangles
  (L=3: 1280, L=5: 20480, L=6: 81920, L=7: 327680).
* ``subdivided_icosahedron(s)``: each icosahedron face split into s*s
  triangles on a barycentric grid, projected to the sphere; n = 20 s^2.
  This gives meshes of any size between the icosphere levels.
* ``perturb_sphere``: radial perturbation r = 1 + a sin(3 theta) cos(2 phi).
* ``scale_axes``: ellipsoid with the given semi-axes.
"""

import numpy as np

_PHI = (1.0 + 5.0 ** 0.5) / 2.0


def icosahedron():
    """The regular icosahedron inscribed in the unit sphere, outward oriented."""
    raw = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            raw.append((0.0, s1, s2 * _PHI))
            raw.append((s1, s2 * _PHI, 0.0))
            raw.append((s2 * _PHI, 0.0, s1))
    v = np.array(raw, dtype=np.float64)
    v /= np.sqrt((v * v).sum(axis=1))[:, None]
    nv = v.shape[0]
    # edges of the icosahedron are the closest vertex pairs
    d2 = ((v[:, None, :] - v[None, :, :]) ** 2).sum(axis=2)
    edge = d2[d2 > 1e-12].min()
    adj = np.abs(d2 - edge) < 1e-9
    faces = []
    for a in range(nv):
        for b in range(a + 1, nv):
            if not adj[a, b]:
                continue
            for c in range(b + 1, nv):
                if adj[a, c] and adj[b, c]:
                    nrm = np.cross(v[b] - v[a], v[c] - v[a])
                    if np.dot(nrm, v[a] + v[b] + v[c]) > 0.0:
                        faces.append((a, b, c))
                    else:
                        faces.append((a, c, b))
    t = np.array(faces, dtype=np.int32)
    assert t.shape == (20, 3)
    return v, t


def _refine(v, t):
    """Split each triangle into four by its edge midpoints (projected)."""
    verts = [tuple(x) for x in v]
    mid = {}

    def midpoint(a, b):
        key = (a, b) if a < b else (b, a)
        idx = mid.get(key)
        if idx is None:
            m = np.asarray(verts[a]) + np.asarray(verts[b])
            m = m / np.sqrt(np.dot(m, m))
            idx = len(verts)
            verts.append(tuple(m))
            mid[key] = idx
        return idx

    out = []
    for a, b, c in t:
        a, b, c = int(a), int(b), int(c)
        ab = midpoint(a, b)
        bc = midpoint(b, c)
        ca = midpoint(c, a)
        out.append((a, ab, ca))
        out.append((ab, b, bc))
        out.append((ca, bc, c))
        out.append((ab, bc, ca))
    return np.array(verts, dtype=np.float64), np.array(out, dtype=np.int32)


def icosphere(level):
    """Icosahedron refined ``level`` times; 20 * 4**level triangles."""
    v, t = icosahedron()
    for _ in range(level):
        v, t = _refine(v, t)
    return v, t


def subdivided_icosahedron(s):
    """Each icosahedron face split into s*s triangles, projected to the sphere."""
    if s < 1:
        raise ValueError("s must be >= 1")
    v0, t0 = icosahedron()
    index = {}
    verts = []

    def vid(face, i, j):
        # grid point i*B + j*C + (s-i-j)*A over s, keyed by its exact
        # barycentric weights on the global icosahedron vertices
        a, b, c = (int(x) for x in face)
        w = {}
        for vert, wt in ((a, s - i - j), (b, i), (c, j)):
            if wt:
                w[vert] = w.get(vert, 0) + wt
        key = tuple(sorted(w.items()))
        idx = index.get(key)
        if idx is None:
            p = np.zeros(3)
            for vert, wt in key:
                p = p + wt * v0[vert]
            p = p / np.sqrt(np.dot(p, p))
            idx = len(verts)
            verts.append(p)
            index[key] = idx
        return idx

    tris = []
    for face in t0:
        for i in range(s):
            for j in range(s - i):
                p00 = vid(face, i, j)
                p10 = vid(face, i + 1, j)
                p01 = vid(face, i, j + 1)
                tris.append((p00, p10, p01))
                if i + j + 1 < s:
                    p11 = vid(face, i + 1, j + 1)
                    tris.append((p10, p11, p01))
    return np.array(verts, dtype=np.float64), np.array(tris, dtype=np.int32)


def perturb_sphere(v, amplitude=0.1):
    """Radially scale unit-sphere vertices by 1 + a sin(3 theta) cos(2 phi).

    theta = acos(z) is the polar angle, phi = atan2(y, x) the azimuth.
    """
    r = np.sqrt((v * v).sum(axis=1))
    u = v / r[:, None]
    theta = np.arccos(np.clip(u[:, 2], -1.0, 1.0))
    phi = np.arctan2(u[:, 1], u[:, 0])
    rad = 1.0 + amplitude * np.sin(3.0 * theta) * np.cos(2.0 * phi)
    return u * rad[:, None]


def scale_axes(v, axes):
    """Ellipsoid: scale the coordinates by the semi-axes (a, b, c)."""
    return v * np.asarray(axes, dtype=np.float64)[None, :]


def mesh_for_config(name):
    """The named single-mesh workloads.

    ``sphere1280``  icosphere level 3, ``sphere20480`` level 5,
    ``perturbed20480`` level 5 perturbed with amplitude 0.1,
    ``sphere81920`` level 6, ``ellipsoid327680`` level 7 with axes
    (1, 1.5, 2.5), ``ellipsoid1280`` level 3 with the same axes,
    ``sphere80`` / ``sphere320`` / ``sphere5120`` levels 1, 2, 4.
    """
    table = {
        "sphere80": (1, None, None),
        "sphere320": (2, None, None),
        "sphere1280": (3, None, None),
        "sphere5120": (4, None, None),
        "sphere20480": (5, None, None),
        "sphere81920": (6, None, None),
        "perturbed320": (2, 0.1, None),
        "perturbed1280": (3, 0.1, None),
        "perturbed20480": (5, 0.1, None),
        "ellipsoid1280": (3, None, (1.0, 1.5, 2.5)),
        "ellipsoid327680": (7, None, (1.0, 1.5, 2.5)),
    }
    level, amp, axes = table[name]
    v, t = icosphere(level)
    if amp is not None:
        v = perturb_sphere(v, amp)
    if axes is not None:
        v = scale_axes(v, axes)
    return v, t


def batch_meshes(count, seed=0, s_min=8, s_max=32):
    """A ragged batch of meshes of uneven size and shape.

    Shape is uniform over {sphere, ellipsoid with semi-axes U(0.5, 2)^3,
    perturbed sphere}; size is 20 s^2 triangles with s ~ U{s_min..s_max}
    (1280 to 20480 triangles for the defaults).
    """
    rng = np.random.default_rng(seed)
    out = []
    cache = {}
    for _ in range(count):
        kind = int(rng.integers(0, 3))
        s = int(rng.integers(s_min, s_max + 1))
        axes = rng.uniform(0.5, 2.0, size=3)
        if s not in cache:
            cache[s] = subdivided_icosahedron(s)
        v, t = cache[s]
        if kind == 1:
            v = scale_axes(v, axes)
        elif kind == 2:
            v = perturb_sphere(v, 0.1)
        out.append((np.ascontiguousarray(v), t.copy()))
    return out


def edge_midpoints_for_config(name):
    """Surface points at the edge midpoints of the mesh ``mesh_for_config(name)``
    (the quadratic nodes of curved triangles): for each triangle the points
    over its edges (0, 1), (1, 2), (2, 0), shape (nt, 3, 3).  The midpoint of
    the two unit-sphere vertices is projected onto the unit sphere and then
    perturbed and scaled like the vertices."""
    table = {"sphere80": (1, None, None), "sphere320": (2, None, None), "sphere1280": (3, None, None),
             "sphere5120": (4, None, None), "sphere20480": (5, None, None),
             "perturbed320": (2, 0.1, None), "perturbed1280": (3, 0.1, None),
             "perturbed20480": (5, 0.1, None), "ellipsoid1280": (3, None, (1.0, 1.5, 2.5))}
    level, amp, axes = table[name]
    v, t = icosphere(level)
    a = v[t]                                  # (nt, 3, 3) unit-sphere corners
    m = 0.5 * (a + a[:, [1, 2, 0], :])        # edges (0, 1), (1, 2), (2, 0)
    m = m / np.sqrt((m * m).sum(axis=2))[:, :, None]
    m = m.reshape(-1, 3)
    if amp is not None:
        m = perturb_sphere(m, amp)
    if axes is not None:
        m = scale_axes(m, axes)
    return m.reshape(-1, 3, 3)
