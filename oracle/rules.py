"""Quadrature rules (oracle).

* ``gauss_legendre_01``: Gauss-Legendre on [0, 1] (numpy's ``leggauss`` as
  a library primitive).  Pinned: exact for polynomials of degree 2q-1.
* ``RADON7`` / ``triangle_points``: the classical 7-point rule of degree 5
  on a triangle (centroid plus two symmetric orbits of three points whose
  coordinates and weights involve sqrt(15)).  The paper uses triangle
  quadrature for the piecewise-constant Galerkin entries (Sect. 2) without
  naming the rule; this 7-point rule is the reading used for every regular
  integral.  Pinned: exact for all monomials up to degree 5.
* ``box_rule``: the quadrature on the boundary of the axis-parallel box
  omega required by Eq. (2): an m x m Gauss-Legendre rule on each of the
  six faces, outward normals along the axes.  Pinned: weights sum to the
  surface area, flux of the fundamental solution (Gauss's law) and
  convergence of Green's representation formula (Sect. 2).
"""

import numpy as np


def gauss_legendre_01(q):
    """Nodes and weights of the q-point Gauss-Legendre rule on [0, 1]."""
    t, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * (t + 1.0), 0.5 * w


def _radon7():
    s = np.sqrt(15.0)
    a1 = (6.0 - s) / 21.0
    b1 = 1.0 - 2.0 * a1
    a2 = (6.0 + s) / 21.0
    b2 = 1.0 - 2.0 * a2
    w0 = 9.0 / 40.0
    w1 = (155.0 - s) / 1200.0
    w2 = (155.0 + s) / 1200.0
    bary = np.array([
        [1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0],
        [b1, a1, a1], [a1, b1, a1], [a1, a1, b1],
        [b2, a2, a2], [a2, b2, a2], [a2, a2, b2],
    ])
    wts = np.array([w0, w1, w1, w1, w2, w2, w2])
    return bary, wts


# barycentric coordinates (7 x 3) and weights (summing to 1, relative to area)
RADON7 = _radon7()


def triangle_areas(vertices, triangles):
    a = vertices[triangles[:, 0]]
    b = vertices[triangles[:, 1]]
    c = vertices[triangles[:, 2]]
    cr = np.cross(b - a, c - a)
    return 0.5 * np.sqrt((cr * cr).sum(axis=1))


def triangle_points(vertices, triangles, rule=RADON7):
    """Quadrature points (nt x 7 x 3) and weights * area (nt x 7) per triangle."""
    bary, wts = rule
    a = vertices[triangles[:, 0]]
    b = vertices[triangles[:, 1]]
    c = vertices[triangles[:, 2]]
    pts = (bary[None, :, 0, None] * a[:, None, :]
           + bary[None, :, 1, None] * b[:, None, :]
           + bary[None, :, 2, None] * c[:, None, :])
    area = triangle_areas(vertices, triangles)
    return pts, wts[None, :] * area[:, None]


def box_rule(lo, hi, m):
    """Tensor Gauss rule of order m on each face of the box [lo, hi].

    Returns points z (6 m^2 x 3), outward unit normals (6 m^2 x 3) and
    weights w (6 m^2).  Faces are ordered -x, +x, -y, +y, -z, +z; on each
    face the first remaining axis varies slowest.
    """
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    t, w = np.polynomial.legendre.leggauss(m)
    pts, nrm, wts = [], [], []
    for d in range(3):
        d1, d2 = [e for e in range(3) if e != d]
        mid1, half1 = 0.5 * (lo[d1] + hi[d1]), 0.5 * (hi[d1] - lo[d1])
        mid2, half2 = 0.5 * (lo[d2] + hi[d2]), 0.5 * (hi[d2] - lo[d2])
        for side in (-1.0, 1.0):
            for a in range(m):
                for b in range(m):
                    z = np.empty(3)
                    z[d] = lo[d] if side < 0 else hi[d]
                    z[d1] = mid1 + half1 * t[a]
                    z[d2] = mid2 + half2 * t[b]
                    n = np.zeros(3)
                    n[d] = side
                    pts.append(z)
                    nrm.append(n)
                    wts.append(w[a] * w[b] * half1 * half2)
    return np.array(pts), np.array(nrm), np.array(wts)
