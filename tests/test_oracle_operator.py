"""Pins of the oracle's discrete x-ray transform (Sec. 2.1, Eq. 1-4) against
facts that do not come from the oracle itself: the closed-form projection of
a unit square (a trapezoid), brute-force line sampling, the analytic line
integral of an ellipse (Kak & Slaney, the paper's reference for Eq. 1), the
90-degree rotation symmetry of the Radon transform, and a dense SVD."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2410_06106_gb300 import synth


def trapezoid(c, s, tau):
    """projection of the unit square onto the ray normal: the convolution of
    boxes of widths |c| and |s|, normalised to unit area"""
    wp = 0.5 * (abs(c) + abs(s))
    wm = 0.5 * abs(abs(c) - abs(s))
    h = 1.0 / max(abs(c), abs(s))
    if wp == wm:  # axis-aligned: a box, half value exactly on the edge
        return h * (1.0 if abs(tau) < wp else 0.5 if abs(tau) == wp else 0.0)
    return h * min(max((wp - abs(tau)) / (wp - wm), 0.0), 1.0)


def test_chord_matches_trapezoid_closed_form():
    rng = np.random.default_rng(11)
    for _ in range(20000):
        th = rng.uniform(0.0, math.pi)
        c, s = math.cos(th), math.sin(th)
        tau = rng.uniform(-1.0, 1.0)
        xc, yc = rng.integers(-5, 6), rng.integers(-5, 6)
        t = tau + xc * c + yc * s
        assert abs(O.chord(c, s, t, xc, yc) - trapezoid(c, s, tau)) < 1e-12


def test_chord_matches_brute_force_line_sampling():
    rng = np.random.default_rng(12)
    L = 400000
    for _ in range(20):
        th = rng.uniform(0.0, math.pi)
        c, s = math.cos(th), math.sin(th)
        t = rng.uniform(-0.9, 0.9)
        lam = (np.arange(L) + 0.5) / L * 4.0 - 2.0  # the line segment |l| <= 2 covers the square
        x, y = t * c - lam * s, t * s + lam * c
        inside = (np.abs(x) <= 0.5) & (np.abs(y) <= 0.5)
        assert abs(inside.mean() * 4.0 - O.chord(c, s, t, 0.0, 0.0)) < 1e-4


def test_axis_aligned_rays_split_edges_and_conserve_length():
    N, B = 8, 13
    theta = np.array([0.0, math.pi / 2])
    g = O.Geometry(N, B, theta)
    c, s = g.c, g.s
    assert (c[0], s[0], c[1], s[1]) == (1.0, 0.0, 0.0, 1.0)  # snapped exactly
    for i in range(N):
        for j in range(N):
            img = np.zeros((N, N))
            img[i, j] = 1.0
            d = g.project(img)
            # N even, B odd: every ray lies on a pixel edge -> two bins of 1/2
            for a in range(2):
                nz = np.sort(d[a][d[a] != 0])
                assert np.array_equal(nz, [0.5, 0.5])
                assert d[a].sum() == 1.0


def test_single_pixel_projection_is_the_trapezoid():
    N, B, A = 6, 11, 24
    theta = synth.angles(A)
    g = O.Geometry(N, B, theta)
    for (i, j) in [(0, 0), (2, 3), (5, 1)]:
        img = np.zeros((N, N))
        img[i, j] = 1.0
        d = g.project(img)
        xc, yc = j - 0.5 * (N - 1), 0.5 * (N - 1) - i
        for a in range(A):
            for b in range(B):
                tau = (b - 0.5 * (B - 1)) - (xc * g.c[a] + yc * g.s[a])
                assert abs(d[a, b] - trapezoid(g.c[a], g.s[a], tau)) < 1e-12


def test_rays_missing_the_image_are_zero():
    N, B, A = 16, 41, 10
    g = O.Geometry(N, B, synth.angles(A))
    d = g.project(np.ones((N, N)))
    t = np.arange(B) - 0.5 * (B - 1)
    reach = 0.5 * N * (np.abs(g.c) + np.abs(g.s))  # half-width of the image's shadow
    outside = np.abs(t)[None, :] >= reach[:, None] + 1e-9
    assert outside.any() and np.all(d[outside] == 0.0)


@pytest.mark.parametrize("N", [32, 64, 128, 256])
def test_projection_converges_to_analytic_ellipse_integrals(N):
    """P (pixel-averaged ellipses) -> exact line integrals, first order in 1/N"""
    B = int(math.ceil(N * math.sqrt(2))) | 1
    theta = synth.angles(12) + 0.1
    g = O.Geometry(N, B, theta)
    f = N / 128.0
    ell = np.array([[25 * f, 10 * f, 20 * f, 8 * f, 0.3, 1.0],
                    [-20 * f, 30 * f, 25 * f, 10 * f, 1.2, 0.5],
                    [0.0, 0.0, 40 * f, 40 * f, 0.0, 0.2]])  # includes a disk
    img = synth.rasterize(ell, N, ss=8)
    rel = np.linalg.norm(g.project(img) - synth.ellipse_sinogram(ell, theta, B))
    rel /= np.linalg.norm(synth.ellipse_sinogram(ell, theta, B))
    assert rel < 2.6 / N  # measured ~2.3/N: error halves with each doubling of N
    if N == 256:
        assert rel < 0.02


def test_adjoint_dot_product_fp64():
    N, B, A = 24, 35, 17
    g = O.Geometry(N, B, synth.angles(A) + 0.05)
    rng = np.random.default_rng(3)
    x, y = rng.standard_normal((N, N)), rng.standard_normal((A, B))
    lhs = float(np.sum(g.project(x) * y))
    rhs = float(np.sum(x * g.backproject(y)))
    assert abs(lhs - rhs) <= 1e-12 * abs(rhs)


def test_quarter_turn_symmetry():
    """rotating the object by +90 degrees: P(u')(theta, t) = P(u)(theta - pi/2, t),
    and P(u)(theta - pi, t) = P(u)(theta, -t) below zero"""
    N, A = 16, 8
    B = 2 * N + 1
    g = O.Geometry(N, B, synth.angles(A))
    rng = np.random.default_rng(5)
    img = rng.random((N, N))
    d = g.project(img)
    d_rot = g.project(np.rot90(img))  # counter-clockwise quarter turn
    for a in range(A):
        ref = d[a - A // 2] if a >= A // 2 else d[a + A // 2][::-1]
        assert np.allclose(d_rot[a], ref, atol=1e-12)


def test_sampled_rays_and_pixels_match_full_operator():
    N, B, A = 20, 29, 9
    g = O.Geometry(N, B, synth.angles(A) + 0.2)
    rng = np.random.default_rng(8)
    img, sino = rng.random((N, N)), rng.random((A, B))
    d = g.project(img)
    ra, rb = rng.integers(0, A, 40), rng.integers(0, B, 40)
    assert np.allclose(g.project_rays(img, ra, rb), d[ra, rb], rtol=1e-13, atol=1e-13)
    bp = g.backproject(sino)
    pix = rng.integers(0, N * N, 40)
    assert np.allclose(g.backproject_pixels(sino, pix), bp.ravel()[pix], rtol=1e-13)


def test_operator_norm_matches_dense_svd():
    N, B, A = 8, 13, 7
    g = O.Geometry(N, B, synth.angles(A))
    P = np.stack([g.project(e.reshape(N, N)).ravel() for e in np.eye(N * N)], axis=1)
    sv = np.linalg.svd(P, compute_uv=False)[0]
    assert abs(g.opnorm_sq(iters=300) - sv * sv) < 1e-8 * sv * sv
    sel = np.array([1, 4, 6], np.int32)
    Ps = np.stack([g.project(e.reshape(N, N), sel).ravel() for e in np.eye(N * N)], axis=1)
    svs = np.linalg.svd(Ps, compute_uv=False)[0]
    assert abs(g.opnorm_sq(sel, iters=300) - svs * svs) < 1e-8 * svs * svs
