"""Pins for the oracle's undecimated wavelet, its prox step and the sigma / 2 rule
(Sec. 2.1; Supporting Information S1, Method 2)."""

import math

import numpy as np
import pytest

from oracle import swt
from oracle import wavelet as wv


def _dense_W(n, name):
    cols = []
    for j in range(n * n):
        e = np.zeros(n * n, np.complex128)
        e[j] = 1.0
        cols.append(swt.swt2(e.reshape(n, n), name).reshape(-1))
    return np.stack(cols, axis=1)  # [4 n^2][n^2]


@pytest.mark.parametrize("name", ["haar", "db4"])
def test_tight_frame_and_projection(name):
    W = _dense_W(8, name)
    assert np.allclose(W.conj().T @ W, np.eye(64), atol=1e-13)          # W^H W = I
    P = W @ W.conj().T                                                     # W W^H: orthogonal projection
    assert np.allclose(P @ P, P, atol=1e-13) and np.allclose(P, P.conj().T, atol=1e-13)
    assert round(float(np.real(np.trace(P)))) == 64


@pytest.mark.parametrize("name", ["haar", "db4"])
def test_inverse_is_the_adjoint(name):
    rng = np.random.default_rng(3)
    x = rng.standard_normal((12, 10)) + 1j * rng.standard_normal((12, 10))
    c = rng.standard_normal((4, 12, 10)) + 1j * rng.standard_normal((4, 12, 10))
    lhs = np.vdot(swt.swt2(x, name), c)
    rhs = np.vdot(x, swt.iswt2(c, name))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)
    assert np.allclose(swt.iswt2(swt.swt2(x, name), name), x, atol=1e-12)


@pytest.mark.parametrize("name", ["haar", "db4"])
def test_even_samples_are_the_decimated_transform(name):
    """At even positions the undecimated coefficients are the 1-level DWT's, / 2."""
    rng = np.random.default_rng(4)
    x = rng.standard_normal((16, 16)) + 1j * rng.standard_normal((16, 16))
    c = swt.swt2(x, name)
    d = wv.dwt2(x, name, 1)
    for fy in range(2):
        for fx in range(2):
            blk = d[fy * 8:(fy + 1) * 8, fx * 8:(fx + 1) * 8]
            assert np.allclose(c[fx + 2 * fy][::2, ::2], blk / 2, atol=1e-12)


def test_shift_equivariance():
    rng = np.random.default_rng(5)
    x = rng.standard_normal((16, 12)) + 1j * rng.standard_normal((16, 12))
    a = swt.swt2(np.roll(x, (3, 5), axis=(0, 1)), "db4")
    b = np.roll(swt.swt2(x, "db4"), (3, 5), axis=(1, 2))
    assert np.allclose(a, b, atol=1e-12)


def test_haar_closed_form():
    rng = np.random.default_rng(6)
    a = rng.standard_normal((6, 7)) + 1j * rng.standard_normal((6, 7))
    A = lambda dy, dx: np.roll(a, (-dy, -dx), axis=(0, 1))  # a[y + dy, x + dx] (periodic)
    c = swt.swt2(a, "haar")
    assert np.allclose(c[0], (A(0, 0) + A(0, 1) + A(1, 0) + A(1, 1)) / 4)
    assert np.allclose(c[1], (A(0, 0) - A(0, 1) + A(1, 0) - A(1, 1)) / 4)
    assert np.allclose(c[2], (A(0, 0) + A(0, 1) - A(1, 0) - A(1, 1)) / 4)
    assert np.allclose(c[3], (A(0, 0) - A(0, 1) - A(1, 0) + A(1, 1)) / 4)


def test_prox_limits_and_nonexpansive():
    rng = np.random.default_rng(7)
    v = rng.standard_normal(200) + 1j * rng.standard_normal(200)
    assert np.allclose(swt.prox(v, 10, 20, "db4", 0.0), v, atol=1e-12)      # tau = 0: identity
    c = swt.swt2(v.reshape(10, 20), "db4")
    c[1:] = 0
    assert np.allclose(swt.prox(v, 10, 20, "db4", 1e9), swt.iswt2(c, "db4").reshape(-1), atol=1e-12)
    w = rng.standard_normal(200) + 1j * rng.standard_normal(200)
    d = np.linalg.norm(swt.prox(v, 10, 20, "db4", 0.7) - swt.prox(w, 10, 20, "db4", 0.7))
    assert d <= np.linalg.norm(v - w) * (1 + 1e-12)


def test_histogram_mode_of_a_rayleigh_sample():
    """The histogram rule recovers the mode sigma of a Rayleigh law (+-10 % at n = 2e5),
    with or without a heavy tail of large 'signal' values beyond the noise."""
    rng = np.random.default_rng(8)
    for sigma in (0.3, 7.0):
        m = rng.rayleigh(sigma, 200_000)
        assert abs(swt.rayleigh_sigma(m) - sigma) < 0.1 * sigma
        tail = np.concatenate([m, rng.uniform(10 * sigma, 1000 * sigma, 20_000)])
        assert abs(swt.rayleigh_sigma(tail) - sigma) < 0.1 * sigma
    assert swt.rayleigh_sigma(np.zeros(10)) == 0.0


def test_noise_sigma_through_the_transform():
    """White complex noise with per-component std s: every detail coefficient of the tight
    frame is complex Gaussian with per-component std s / 2, so sigma = s / 2."""
    rng = np.random.default_rng(9)
    s = 1.7
    x = s * (rng.standard_normal((256, 256)) + 1j * rng.standard_normal((256, 256)))
    for name in ("haar", "db4"):
        est = swt.rayleigh_sigma(swt.swt2(x, name)[1:])
        assert abs(est - s / 2) < 0.1 * s / 2


def test_fista_with_lambda_zero_is_plain_fista():
    """lambda = 0: the tight-frame step is the identity, so the iterates are plain FISTA's."""
    import oracle
    from oracle import recon
    from paper_2211_07532_gb300 import synth
    oracle.build()
    p = synth.make_problem(12, 10, nt=400, nc=2, order=1, dwell=4e-6, turns=3.0, seed=11)
    y = synth.random_kspace(np.random.default_rng(12), 2, 400)
    L = recon.power_lipschitz(p, oracle.adjoint(p, y), 20)
    a = swt.fista(p, y, 0.0, 6, L, "db4")
    b = recon.fista(p, y, 0.0, 6, L, "haar", 1)
    assert np.allclose(a, b, atol=1e-10 * np.linalg.norm(b))
