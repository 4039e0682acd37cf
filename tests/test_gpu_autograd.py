"""Differentiation through the H^2 product.

``H2Matvec`` makes y = G_H2 u a torch operation whose backward is the
transposed H^2 product.  The test problem is the inverse problem of
recovering a boundary density from field values:

    L(u) = || P G_H2 u - f ||^2,

with P the exterior single-layer evaluation (P v)_k = sum_j v_j int_{T_j}
g(p_k, y) dy (7-point rule) at 4096 points p_k on the sphere of radius 3,
which encloses the ellipsoid with semi-axes (1, 1.5, 2.5), and
f = P G u* for u* = 1 + z/2 at the triangle centroids.  P and the loss are
plain torch; only G_H2 and its transpose run in the library.

On the 1280-triangle copy the gradient 2 G_H2^T P^T (P G_H2 u - f) is
checked against the oracle's H^2 (float64), against the dense Galerkin G
(within the compression error), against torch.autograd.gradcheck and
central finite differences; the float32 gradient against the float64
oracle.  On the full 327680-triangle ellipsoid the float32 gradient is held
to the float64 one, and the float64 gradient to a central finite difference
and the adjoint identity.
"""

import numpy as np
import pytest

import synth
from oracle import gca as ogca, h2 as oh2
from oracle.galerkin import Galerkin
from oracle.params import Params as OParams
from oracle.rules import triangle_points

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SMALL = dict(leaf_size=32, eta=2.0, box_gauss_m=3, aca_tol=1e-6, sauter_q=5)
LARGE = dict(leaf_size=64, eta=2.0, box_gauss_m=4, aca_tol=1e-8, sauter_q=5)
FOUR_PI = 4.0 * np.pi


@pytest.fixture(scope="module")
def lib():
    import paper_1810_08429_b300 as gca
    assert torch.cuda.is_available()
    return gca


def exterior_matrix(v, t, pts, chunk=2048):
    """P[k, j] = sum_q w_q(T_j) / (4 pi |p_k - x_q(T_j)|), float64 on the GPU."""
    xq, wq = triangle_points(v, t)
    X = torch.from_numpy(xq).cuda()
    W = torch.from_numpy(wq).cuda()
    Pp = torch.from_numpy(np.ascontiguousarray(pts)).cuda()
    n = len(t)
    out = torch.empty((len(pts), n), dtype=torch.float64, device="cuda")
    for j0 in range(0, n, chunk):
        j1 = min(n, j0 + chunk)
        d = Pp[:, None, None, :] - X[None, j0:j1]
        out[:, j0:j1] = (W[None, j0:j1] / d.norm(dim=-1)).sum(-1) / FOUR_PI
    return out


def target_density(v, t):
    c = v[t].mean(axis=1)
    return 1.0 + 0.5 * c[:, 2]


def loss_and_grad(lib, h, P, f, u0, prec):
    dt = torch.float64 if prec == "f64" else torch.float32
    u = u0.to(dt).clone().requires_grad_(True)
    y = lib.H2Matvec.apply(h, u, prec)
    r = P.to(dt) @ y - f.to(dt)
    L = (r * r).sum()
    L.backward()
    return L.detach(), u.grad.detach()


def rel(a, b):
    a = a.double() if torch.is_tensor(a) else torch.as_tensor(a)
    b = b.double() if torch.is_tensor(b) else torch.as_tensor(b)
    return float((a.cpu() - b.cpu()).norm() / b.cpu().norm())


@pytest.fixture(scope="module")
def small(lib):
    v, t = synth.mesh_for_config("ellipsoid1280")
    tree = lib.tree_build(v, t, SMALL["leaf_size"])
    h = lib.build(v, t, tree, lib.Params(**SMALL))
    Ho = ogca.build_h2(v, t, OParams(**SMALL))
    G = Galerkin(v, t, SMALL["sauter_q"]).dense_matrix()
    pts = synth.exterior_points(4096, radius=3.0, seed=0)
    P = exterior_matrix(v, t, pts)
    f = P @ torch.from_numpy(G @ target_density(v, t)).cuda()
    u0 = torch.from_numpy(synth.normal_rhs(len(t), 1, seed=0)[:, 0]).cuda()
    return h, Ho, G, P, f, u0


def test_gradient_matches_oracle_h2(lib, small):
    h, Ho, G, P, f, u0 = small
    _, g = loss_and_grad(lib, h, P, f, u0, "f64")
    Pn, fn, un = P.cpu().numpy(), f.cpu().numpy(), u0.cpu().numpy()
    r = Pn @ np.ravel(oh2.matvec(Ho, un)) - fn
    g_oracle = 2.0 * np.ravel(oh2.matvec_t(Ho, Pn.T @ r))
    assert rel(g, torch.from_numpy(g_oracle)) <= 1e-10
    # the dense Galerkin matrix: equal up to the compression error
    g_dense = 2.0 * G.T @ (Pn.T @ (Pn @ (G @ un) - fn))
    assert rel(g, torch.from_numpy(g_dense)) <= 1e-4


def test_gradient_float32(lib, small):
    h, Ho, G, P, f, u0 = small
    _, g32 = loss_and_grad(lib, h, P, f, u0, "f32")
    Pn, fn, un = P.cpu().numpy(), f.cpu().numpy(), u0.cpu().numpy()
    r = Pn @ np.ravel(oh2.matvec(Ho, un)) - fn
    g_oracle = 2.0 * np.ravel(oh2.matvec_t(Ho, Pn.T @ r))
    assert rel(g32, torch.from_numpy(g_oracle)) <= 1e-5


def test_finite_differences(lib, small):
    h, Ho, G, P, f, u0 = small
    L0, g = loss_and_grad(lib, h, P, f, u0, "f64")
    rng = np.random.default_rng(3)
    for _ in range(3):
        d = torch.from_numpy(rng.standard_normal(len(u0))).cuda()
        eps = 1e-6 * float(u0.norm() / d.norm())
        Lp, _ = loss_and_grad(lib, h, P, f, u0 + eps * d, "f64")
        Lm, _ = loss_and_grad(lib, h, P, f, u0 - eps * d, "f64")
        fd = float(Lp - Lm) / (2 * eps)
        an = float((g * d).sum())
        # relative to |g| |d|: a random direction is nearly orthogonal to g
        assert abs(fd - an) <= 1e-6 * float(g.norm() * d.norm()), (fd, an)


def test_gradcheck(lib, small):
    h = small[0]
    u = torch.from_numpy(synth.uniform_rhs(h.n, 1, seed=4)[:, 0]).cuda().requires_grad_(True)
    # the Jacobian is G_H2 itself: backward = transpose checked column by column
    assert torch.autograd.gradcheck(lambda x: lib.H2Matvec.apply(h, x, "f64"), (u,), eps=1e-6,
                                    atol=1e-9, rtol=1e-6, nondet_tol=1e-12, fast_mode=True)


def test_full_size_ellipsoid(lib):
    v, t = synth.mesh_for_config("ellipsoid327680")
    n = len(t)
    tree = lib.tree_build(v, t, LARGE["leaf_size"])
    h = lib.build(v, t, tree, lib.Params(**LARGE, flags=lib.DROP_BF16 | lib.DROP_EXPORT))
    pts = synth.exterior_points(4096, radius=3.0, seed=0)
    P = exterior_matrix(v, t, pts)
    ustar = torch.from_numpy(target_density(v, t)).cuda()
    f = P @ h.matvec(ustar, "f64")
    u0 = torch.from_numpy(synth.normal_rhs(n, 1, seed=0)[:, 0]).cuda()
    L64, g64 = loss_and_grad(lib, h, P, f, u0, "f64")
    L32, g32 = loss_and_grad(lib, h, P, f, u0, "f32")
    assert rel(g32, g64) <= 1e-5
    assert abs(float(L32) - float(L64)) <= 1e-5 * float(L64)
    # central difference along one random direction (float64)
    d = torch.from_numpy(synth.normal_rhs(n, 1, seed=7)[:, 0]).cuda()
    eps = 1e-6 * float(u0.norm() / d.norm())
    Lp, _ = loss_and_grad(lib, h, P, f, u0 + eps * d, "f64")
    Lm, _ = loss_and_grad(lib, h, P, f, u0 - eps * d, "f64")
    fd = float(Lp - Lm) / (2 * eps)
    an = float((g64 * d).sum())
    assert abs(fd - an) <= 1e-6 * float(g64.norm() * d.norm()), (fd, an)
    # adjoint identity <a, G_H2 b> = <G_H2^T a, b>
    a = torch.from_numpy(synth.normal_rhs(n, 1, seed=8)[:, 0]).cuda()
    lhs = float((a * h.matvec(d, "f64")).sum())
    rhs = float((h.matvec(a, "f64", transpose=True) * d).sum())
    assert abs(lhs - rhs) <= 1e-12 * (a.norm() * d.norm() * h.matvec(d, "f64").norm() / d.norm())
    assert h.status() == 0
