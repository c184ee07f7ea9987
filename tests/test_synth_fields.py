"""Checks of the synthetic field inputs beyond 3rd order: the degree-4 solid harmonics, the
tilted-slice readout and the second-order concomitant-field rows (Fig. S3d shows these rows
among the monitored field dynamics).  These arrays are inputs of the operator, so the checks
are on the input recipe, against closed forms."""

import math

import numpy as np

from paper_2211_07532_gb300 import synth


def _laplacian(f, x, y, z, h=1e-3):
    """Fourth-order central differences: exact (up to rounding) on polynomials of degree <= 5."""
    c = f(x, y, z)
    out = 0.0
    for e in np.eye(3):
        g = lambda s: f(x + s * e[0], y + s * e[1], z + s * e[2])
        out = out + (-g(2 * h) + 16 * g(h) - 30 * c + 16 * g(-h) - g(-2 * h)) / (12 * h * h)
    return out


def test_solid_harmonics_to_4th_order_are_harmonic_and_independent():
    rng = np.random.default_rng(0)
    x, y, z = rng.uniform(-0.1, 0.1, (3, 64))
    n = synth.n_terms(4)
    for l in range(n):
        f = lambda a, b, c: synth.sh_basis(a, b, c, 4)[l]
        scale = np.max(np.abs(f(x, y, z))) / 0.1 ** 2 + 1e-30   # |f| / r^2: size of second derivatives
        assert np.max(np.abs(_laplacian(f, x, y, z))) < 1e-6 * scale, l
        assert synth.term_degree(l) == int(math.isqrt(l))
    H = synth.sh_basis(x, y, z, 4)
    assert H.shape == (25, 64) and np.linalg.matrix_rank(H) == 25
    # homogeneous of its degree: h_l(2 r) = 2^deg h_l(r)
    H2 = synth.sh_basis(2 * x, 2 * y, 2 * z, 4)
    deg = np.array([synth.term_degree(l) for l in range(25)])
    assert np.allclose(H2, (2.0 ** deg)[:, None] * H, rtol=1e-12, atol=1e-15)


def test_tilted_slice_keeps_the_in_plane_encoding():
    """sum of the three linear terms = k_u u + k_v v + k_v sin(tilt) z0 for every tilt."""
    for tilt in (0.0, 0.35, 1.2):
        p = synth.make_problem(12, 10, nt=300, nc=2, order=1, eddy=False, tilt=tilt, z0=0.004, seed=3)
        U, V = synth.voxel_positions(12, 10, p["fov"], p["fov"] * 10 / 12)
        lin = p["k"][1:4].astype(np.float64).T @ p["h"][1:4].astype(np.float64)   # [nt][nr]
        kxy = synth.spiral_k(300, math.pi / (p["fov"] / 12), 12 / 8.0, 1.0)
        want = np.outer(kxy.real, U) + np.outer(kxy.imag, V) + np.outer(kxy.imag * math.sin(tilt) * 0.004,
                                                                        np.ones_like(U))
        assert np.allclose(lin, want, rtol=1e-5, atol=1e-5 * np.abs(want).max())


def test_gradients_integrate_back_to_k():
    rng = np.random.default_rng(1)
    k = np.cumsum(rng.standard_normal((3, 50)), axis=1)
    G = synth.gradients_from_k(k, 2e-6)
    assert np.allclose(synth.GAMMA * 2e-6 * np.cumsum(G, axis=1), k, rtol=1e-12, atol=1e-12)


def test_concomitant_rows_give_the_maxwell_phase():
    """sum_c k_c(t) h_c(r) = gamma dt sum_{n <= t} B_c(r, G[n]) with the Maxwell field written
    out point by point."""
    rng = np.random.default_rng(2)
    nt, dt, B0 = 40, 3e-6, 7.0
    G = rng.uniform(-0.08, 0.08, (3, nt))
    pts = rng.uniform(-0.1, 0.1, (3, 6))
    kc = synth.concomitant_coefficients(G, dt, B0)
    hc = synth.concomitant_basis(*pts)
    got = kc.T @ hc
    for j in range(6):
        x, y, z = pts[:, j]
        acc = 0.0
        for n in range(nt):
            gx, gy, gz = G[:, n]
            Bc = (gx * gx * z * z + gy * gy * z * z + gz * gz * (x * x + y * y) / 4.0
                  - gx * gz * x * z - gy * gz * y * z) / (2.0 * B0)
            acc += synth.GAMMA * dt * Bc
            assert abs(got[n, j] - acc) <= 1e-12 * max(1.0, abs(acc))


def test_concomitant_problem_layout():
    p = synth.make_problem(16, 16, nt=200, nc=2, order=4, tilt=0.3, concomitant=True, seed=4)
    assert p["nl"] == 25 + 4 and p["k"].shape == (29, 200) and p["h"].shape == (29, 256)
    q = synth.make_problem(16, 16, nt=200, nc=2, order=4, tilt=0.3, seed=4)
    assert np.array_equal(p["k"][:25], q["k"]) and np.array_equal(p["h"][:25], q["h"])
    assert np.array_equal(p["x_gt"], q["x_gt"]) and np.array_equal(p["noise"], q["noise"])
