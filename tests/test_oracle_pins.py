"""Pins of the FP64 oracle against what the mathematics and the literature fix.

None of these re-types the oracle's formulas: each compares it with an
independent result (numpy FFT, a dense least-squares solve, eigenvalues, a
published filter table, closed forms, brute force, optimality conditions).
"""

import math
import os

import numpy as np
import pytest

from paper_2211_07532_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _cart(n, fov=0.2):
    """Cartesian DFT set-up in FP64 (no storage rounding): terms (1, x, y)."""
    X, Y = synth.voxel_positions(n, n, fov, fov)
    m = (np.arange(n) - n // 2) * 2 * np.pi / fov
    KY, KX = np.meshgrid(m, m, indexing="ij")
    return X, Y, KX.reshape(-1), KY.reshape(-1)


def _prob(n, nl, k, h, nc=1, S=None, omega=None, t=None):
    nr = n * n
    return dict(nx=n, ny=n, nt=k.shape[1], nc=nc, nl=nl, k=k, h=h,
                S=np.ones((1, nr), complex) if S is None else S,
                omega=omega, t=t if t is not None else np.zeros(k.shape[1]))


def _dft2(img):
    return np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(img)))


def _rel(a, b):
    return np.linalg.norm(np.asarray(a) - np.asarray(b)) / np.linalg.norm(np.asarray(b))


# --------------------------------------------------------------------------
# Encoding operator (Eq. 1, Sec. 1): Cartesian special case -> FFT
# --------------------------------------------------------------------------

@pytest.mark.parametrize("n", [8, 16])
def test_cartesian_forward_is_centred_dft(oracle_lib, n):
    X, Y, KX, KY = _cart(n)
    k = np.stack([np.zeros_like(KX), KX, KY])
    h = np.stack([np.ones_like(X), X, Y])
    rng = np.random.default_rng(1)
    img = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    y = oracle_lib.forward(_prob(n, 3, k, h), img.reshape(-1))
    assert _rel(y.reshape(n, n), _dft2(img)) < 1e-12


@pytest.mark.parametrize("n", [8, 16])
def test_cartesian_adjoint_is_scaled_inverse_dft(oracle_lib, n):
    X, Y, KX, KY = _cart(n)
    k = np.stack([np.zeros_like(KX), KX, KY])
    h = np.stack([np.ones_like(X), X, Y])
    rng = np.random.default_rng(2)
    ksp = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    x = oracle_lib.adjoint(_prob(n, 3, k, h), ksp.reshape(1, -1))
    ref = n * n * np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(ksp)))
    assert _rel(x.reshape(n, n), ref) < 1e-12


@pytest.mark.parametrize("l", list(range(16)))
def test_every_field_term_enters_the_phase(oracle_lib, l):
    """Put the x-encoding in term l and the y-encoding in term (l+5) mod 16, all
    other terms zero: the result must still be the DFT.  Catches a dropped or
    misindexed term anywhere in the 3rd-order sum."""
    n = 8
    X, Y, KX, KY = _cart(n)
    L = 16
    l2 = (l + 5) % L
    k = np.zeros((L, n * n))
    h = np.zeros((L, n * n))
    rng = np.random.default_rng(10 + l)
    h[:] = rng.standard_normal((L, n * n))  # distractor basis values, zero coefficients
    k[l], h[l] = KX, X
    k[l2], h[l2] = KY, Y
    img = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    y = oracle_lib.forward(_prob(n, L, k, h), img.reshape(-1))
    assert _rel(y.reshape(n, n), _dft2(img)) < 1e-12


def test_b0_term_enters_as_omega_times_t(oracle_lib):
    """omega(r) = a x(r), t = k_x / a reproduces the x-encoding through the B0 term."""
    n = 8
    X, Y, KX, KY = _cart(n)
    a = 2 * np.pi * 37.0
    k = np.stack([np.zeros_like(KX), np.zeros_like(KX), KY])
    h = np.stack([np.ones_like(X), X, Y])
    prob = _prob(n, 3, k, h, omega=a * X, t=KX / a)
    rng = np.random.default_rng(3)
    img = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    y = oracle_lib.forward(prob, img.reshape(-1))
    assert _rel(y.reshape(n, n), _dft2(img)) < 1e-12


def test_constant_term_is_a_per_sample_phase(oracle_lib):
    """k_0(t) with h_0 = 1 multiplies sample t by exp(-i k_0(t)) (shift theorem)."""
    n = 8
    X, Y, KX, KY = _cart(n)
    rng = np.random.default_rng(4)
    k0 = rng.uniform(-50, 50, KX.size)
    k = np.stack([k0, KX, KY])
    h = np.stack([np.ones_like(X), X, Y])
    img = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    y = oracle_lib.forward(_prob(n, 3, k, h), img.reshape(-1))
    ref = _dft2(img).reshape(-1) * np.exp(-1j * k0)
    assert _rel(y[0], ref) < 1e-12


def test_coil_weighting_per_voxel(oracle_lib):
    """y_c = DFT(S_c x) for every coil c (Cartesian case)."""
    n, C = 8, 3
    X, Y, KX, KY = _cart(n)
    k = np.stack([np.zeros_like(KX), KX, KY])
    h = np.stack([np.ones_like(X), X, Y])
    rng = np.random.default_rng(5)
    S = rng.standard_normal((C, n * n)) + 1j * rng.standard_normal((C, n * n))
    img = rng.standard_normal(n * n) + 1j * rng.standard_normal(n * n)
    y = oracle_lib.forward(_prob(n, 3, k, h, nc=C, S=S), img)
    for c in range(C):
        assert _rel(y[c].reshape(n, n), _dft2((S[c] * img).reshape(n, n))) < 1e-12


@pytest.mark.parametrize("shape", [(5, 3, 7, 3, 3), (8, 8, 64, 4, 2), (6, 4, 33, 2, 1)])
def test_adjoint_identity(oracle_lib, shape):
    """<A x, y> = <x, A^H y> to 1e-12 on the synthetic expanded model (3rd order + B0)."""
    nx, ny, nt, nc, order = shape
    p = synth.make_problem(nx, ny, nt=nt, nc=nc, order=order, dwell=2e-5, turns=2.0, seed=99)
    rng = np.random.default_rng(6)
    x = rng.standard_normal(nx * ny) + 1j * rng.standard_normal(nx * ny)
    y = rng.standard_normal((nc, nt)) + 1j * rng.standard_normal((nc, nt))
    Ax = oracle_lib.forward(p, x)
    AHy = oracle_lib.adjoint(p, y)
    lhs = np.vdot(y, Ax)
    rhs = np.vdot(AHy, x)
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(Ax) * np.linalg.norm(y)


def test_row_forms_match_full_sums(oracle_lib):
    p = synth.make_problem(7, 5, nt=19, nc=3, order=3, dwell=1e-5, turns=2.0, seed=7)
    rng = np.random.default_rng(7)
    x = rng.standard_normal(35) + 1j * rng.standard_normal(35)
    y = rng.standard_normal((3, 19)) + 1j * rng.standard_normal((3, 19))
    ts = [0, 5, 18]
    rs = [0, 17, 34]
    np.testing.assert_allclose(oracle_lib.forward_rows(p, x, ts), oracle_lib.forward(p, x)[:, ts], rtol=0, atol=1e-12)
    np.testing.assert_allclose(oracle_lib.adjoint_rows(p, y, rs), oracle_lib.adjoint(p, y)[rs], rtol=0, atol=1e-12)


# --------------------------------------------------------------------------
# Complex soft-threshold (prox of tau*|.|, Eq. 1 penalty)
# --------------------------------------------------------------------------

def test_soft_threshold_closed_form():
    from oracle import wavelet as wv
    w = np.array([0, 1 + 0j, -2j, 3 + 4j, 0.3 - 0.4j])
    out = wv.soft(w, 1.0)
    np.testing.assert_allclose(out, [0, 0, -1j, (3 + 4j) * 0.8, 0], atol=1e-15)


def test_soft_threshold_is_the_prox_by_brute_force():
    """argmin_u 1/2|u - w|^2 + tau |u| on a fine complex grid matches soft(w, tau)."""
    from oracle import wavelet as wv
    rng = np.random.default_rng(8)
    tau = 0.7
    g = np.linspace(-3, 3, 1201)
    U = g[None, :] + 1j * g[:, None]
    for _ in range(6):
        w = complex(rng.uniform(-2.5, 2.5), rng.uniform(-2.5, 2.5))
        cost = 0.5 * np.abs(U - w) ** 2 + tau * np.abs(U)
        best = U.reshape(-1)[np.argmin(cost)]
        assert abs(best - wv.soft(np.array([w]), tau)[0]) < 2 * (g[1] - g[0])


# --------------------------------------------------------------------------
# Orthonormal wavelet W (Eq. 1, Sec. 2.1)
# --------------------------------------------------------------------------

def test_db4_taps_match_published_table():
    from oracle import wavelet as wv
    vals = [float(s) for s in open(os.path.join(GOLDEN, "db4_daubechies_table.txt"))
            if s.strip() and not s.startswith("#")]
    h, _ = wv.filters("db4")
    np.testing.assert_allclose(h, vals, rtol=0, atol=1e-12)


@pytest.mark.parametrize("name", ["haar", "db4"])
def test_filter_identities(name):
    from oracle import wavelet as wv
    h, g = wv.filters(name)
    m = h.size
    assert abs(h.sum() - math.sqrt(2)) < 1e-14
    assert abs(g.sum()) < 1e-14
    for s in range(0, m // 2):
        dot = sum(h[i] * h[i + 2 * s] for i in range(m - 2 * s))
        assert abs(dot - (1.0 if s == 0 else 0.0)) < 1e-14
    p = m // 2
    for q in range(p):  # vanishing moments of the highpass
        assert abs(sum(g[i] * i ** q for i in range(m))) < 1e-9 * (m ** q)


def test_haar_one_level_closed_form():
    from oracle import wavelet as wv
    a, b, c, d = 1.0, 2.0 + 1j, -3.0, 0.5j
    w = wv.dwt2(np.array([[a, b], [c, d]]), "haar", 1)
    ref = np.array([[(a + b + c + d) / 2, (a - b + c - d) / 2],
                    [(a + b - c - d) / 2, (a - b - c + d) / 2]])
    np.testing.assert_allclose(w, ref, atol=1e-15)


@pytest.mark.parametrize("name,n,levels", [("haar", 8, 3), ("db4", 8, 1), ("db4", 16, 2), ("haar", 16, 4)])
def test_wavelet_matrix_is_orthonormal(name, n, levels):
    from oracle import wavelet as wv
    W = np.zeros((n * n, n * n))
    for j in range(n * n):
        e = np.zeros(n * n)
        e[j] = 1.0
        W[:, j] = np.real(wv.dwt2(e.reshape(n, n), name, levels)).reshape(-1)
    np.testing.assert_allclose(W @ W.T, np.eye(n * n), atol=1e-13)
    # and idwt2 is its transpose
    rng = np.random.default_rng(9)
    c = rng.standard_normal((n, n))
    np.testing.assert_allclose(np.real(wv.idwt2(c, name, levels)).reshape(-1), W.T @ c.reshape(-1), atol=1e-13)


def test_perfect_reconstruction_208_db4_4_levels():
    from oracle import wavelet as wv
    rng = np.random.default_rng(10)
    img = rng.standard_normal((208, 208)) + 1j * rng.standard_normal((208, 208))
    back = wv.idwt2(wv.dwt2(img, "db4", 4), "db4", 4)
    assert _rel(back, img) < 1e-13


@pytest.mark.parametrize("name", ["haar", "db4"])
def test_constant_image_has_only_lowpass(name):
    from oracle import wavelet as wv
    J = 3
    w = wv.dwt2(np.full((16, 16), 1.5 - 0.5j), name, J)
    m = wv.detail_mask(w.shape, J)
    assert np.max(np.abs(w[m])) < 1e-13
    np.testing.assert_allclose(w[~m], (1.5 - 0.5j) * 2 ** J, atol=1e-13)


def test_db4_annihilates_cubic_ramp_away_from_the_wrap():
    """4 vanishing moments: first-level x-details of a cubic in x vanish except near the periodic seam."""
    from oracle import wavelet as wv
    n = 32
    xs = np.arange(n, dtype=float)
    img = np.tile(0.01 * xs ** 3 - 0.2 * xs ** 2 + xs, (n, 1))
    w = wv.dwt2(img, "db4", 1)
    hi_x = w[: n // 2, n // 2:]          # lo in y, hi in x
    assert np.max(np.abs(hi_x[:, : n // 2 - 3])) < 1e-10
    assert np.max(np.abs(hi_x[:, n // 2 - 3:])) > 1e-3


def test_prox_with_zero_threshold_is_identity_after_crop():
    from oracle import wavelet as wv
    rng = np.random.default_rng(11)
    v = rng.standard_normal(13 * 11) + 1j * rng.standard_normal(13 * 11)
    out = wv.prox(v, 11, 13, "db4", 2, 0.0)
    assert _rel(out, v) < 1e-13


# --------------------------------------------------------------------------
# Solvers (Sec. 2.1): power iteration, CGLS, FISTA
# --------------------------------------------------------------------------

def _tiny(seed=12, n=8, nt=128, nc=4, turns=3.0):
    p = synth.make_problem(n, nt=nt, nc=nc, order=2, dwell=2e-5, turns=turns, density_power=1.0,
                           seed=seed)
    nr = n * n
    A = np.zeros((nc * nt, nr), complex)
    import oracle
    for j in range(nr):
        e = np.zeros(nr, complex)
        e[j] = 1.0
        A[:, j] = oracle.forward(p, e).reshape(-1)
    rng = np.random.default_rng(seed)
    y = (A @ p["x_gt"].astype(complex)).reshape(nc, nt) + 0.05 * p["noise"]
    return p, A, y


def test_power_iteration_matches_dense_eigenvalue(oracle_lib):
    from oracle import recon
    p, A, y = _tiny()
    lam_max = np.linalg.eigvalsh(A.conj().T @ A).max()
    v0 = oracle_lib.adjoint(p, y)
    Lf = recon.power_lipschitz(p, v0, n_pow=300)
    assert abs(Lf - 2 * lam_max) < 1e-9 * lam_max


def test_cgls_reaches_least_squares(oracle_lib):
    from oracle import recon
    p, A, y = _tiny()
    x_ls = np.linalg.lstsq(A, y.reshape(-1), rcond=None)[0]
    x = recon.cgls(p, y, 200)
    assert _rel(x, x_ls) < 1e-9


def test_fista_lambda0_one_step_exact_when_normal_operator_is_scaled_identity(oracle_lib):
    """Cartesian full sampling: A^H A = n^2 I, L_f = 2 n^2, so one gradient step with
    step 1/L_f from x_0 = 0 lands on the least-squares solution A^H y / n^2."""
    from oracle import recon
    n = 8
    X, Y, KX, KY = _cart(n)
    prob = _prob(n, 3, np.stack([np.zeros_like(KX), KX, KY]), np.stack([np.ones_like(X), X, Y]))
    rng = np.random.default_rng(14)
    y = rng.standard_normal((1, n * n)) + 1j * rng.standard_normal((1, n * n))
    x1 = recon.fista(prob, y, 0.0, 1, 2.0 * n * n, "haar", 3)
    x_ls = n * n * np.fft.fftshift(np.fft.ifft2(np.fft.ifftshift(y.reshape(n, n)))).reshape(-1) / (n * n)
    assert _rel(x1, x_ls) < 1e-12


def test_fista_lambda0_converges_to_least_squares(oracle_lib):
    from oracle import recon
    p, A, y = _tiny(nt=256, turns=8.0)
    x_ls = np.linalg.lstsq(A, y.reshape(-1), rcond=None)[0]
    Lf = 2 * np.linalg.eigvalsh(A.conj().T @ A).max()
    errs = [_rel(recon.fista(p, y, 0.0, it, Lf, "haar", 3), x_ls) for it in (250, 2000)]
    assert errs[1] < 1e-4 and errs[1] < 0.05 * errs[0]


def test_fista_objective_decays_like_one_over_k_squared(oracle_lib):
    """Beck-Teboulle bound F(x_k) - F* <= 2 L_f ||x0 - x*||^2 / (k+1)^2."""
    from oracle import recon
    p, A, y = _tiny()
    Lf = 2 * np.linalg.eigvalsh(A.conj().T @ A).max()
    lam = 1e-3 * np.max(np.abs(oracle_lib.adjoint(p, y))) * 50
    x_star = recon.fista(p, y, lam, 4000, Lf, "haar", 3)
    F_star = recon.objective(p, x_star, y, lam, "haar", 3)
    _, hist = recon.fista(p, y, lam, 40, Lf, "haar", 3, history=True)
    for k, xk in enumerate(hist, start=1):
        gap = recon.objective(p, xk, y, lam, "haar", 3) - F_star
        assert gap <= 2 * Lf * np.linalg.norm(x_star) ** 2 / (k + 1) ** 2 * (1 + 1e-9) + 1e-9


@pytest.mark.parametrize("name,levels", [("haar", 3), ("db4", 1)])
def test_fista_fixed_point_satisfies_kkt(oracle_lib, name, levels):
    """At convergence (lam > 0, W orthonormal since 8 = 2^3): with g = 2 W A^H (A x - y)
    and w = W x, every detail coefficient has g_j = -lam w_j/|w_j| (w_j != 0) or
    |g_j| <= lam (w_j = 0), and every low-pass coefficient has g_j = 0."""
    from oracle import recon
    from oracle import wavelet as wv
    p, A, y = _tiny(seed=13)
    Lf = 2 * np.linalg.eigvalsh(A.conj().T @ A).max()
    lam = 0.2 * np.max(np.abs(oracle_lib.adjoint(p, y)))
    x = recon.fista(p, y, lam, 20000, Lf, name, levels)
    n = p["nx"]
    g = wv.dwt2((2 * oracle_lib.adjoint(p, oracle_lib.forward(p, x) - y)).reshape(n, n), name, levels)
    w = wv.dwt2(x.reshape(n, n), name, levels)
    mask = wv.detail_mask(w.shape, levels)
    tol = 1e-6 * lam
    assert np.max(np.abs(g[~mask])) < tol
    nz = mask & (np.abs(w) > 1e-9 * np.max(np.abs(w)))
    z = mask & ~nz
    assert nz.sum() > 0 and z.sum() > 0
    assert np.max(np.abs(g[nz] + lam * w[nz] / np.abs(w[nz]))) < tol
    assert np.max(np.abs(g[z])) <= lam + tol
