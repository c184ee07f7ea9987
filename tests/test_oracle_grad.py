"""Pins of the oracle's reverse-mode gradient through unrolled FISTA: central finite
differences of the FP64 forward unroll along random directions (x_0, lambda, k_l(t))."""

import numpy as np
import pytest

from paper_2211_07532_gb300 import synth


def _setup(seed=21, n=8, nt=96, nc=2, order=1, iters=4):
    import oracle
    from oracle import recon
    p = synth.make_problem(n, nt=nt, nc=nc, order=order, dwell=2e-5, turns=3.0, seed=seed)
    p = {k: (np.asarray(v, np.float64) if isinstance(v, np.ndarray) and v.dtype == np.float32 else v)
         for k, v in p.items()}
    y = oracle.forward(p, p["x_gt"]) + 0.05 * p["noise"]
    lam = 0.05 * float(np.max(np.abs(oracle.adjoint(p, y))))
    L = recon.power_lipschitz(p, oracle.adjoint(p, y), 50)
    rng = np.random.default_rng(seed)
    x0 = 0.1 * (rng.standard_normal(n * n) + 1j * rng.standard_normal(n * n))
    return p, y, lam, L, x0, iters


def _loss(p, y, lam, L, iters, x0):
    from oracle import recon
    x = recon.fista(p, y, lam, iters, L, "haar", 2, x0=x0)
    return float(np.mean(np.abs(x - p["x_gt"]) ** 2)), x


def test_soft_threshold_vjp_by_finite_differences():
    from oracle import recon
    rng = np.random.default_rng(3)
    w = rng.standard_normal(50) + 1j * rng.standard_normal(50)
    g = rng.standard_normal(50) + 1j * rng.standard_normal(50)
    tau = 0.8
    wbar, taubar = recon.soft_vjp(w, g, tau)
    from oracle import wavelet as wv
    f = lambda ww, tt: float(np.sum(np.real(np.conj(g) * wv.soft(ww, tt))))
    d = rng.standard_normal(50) + 1j * rng.standard_normal(50)
    eps = 1e-6
    fd = (f(w + eps * d, tau) - f(w - eps * d, tau)) / (2 * eps)
    assert abs(fd - np.real(np.vdot(wbar, d))) < 1e-7 * (1 + abs(fd))
    fd_tau = (f(w, tau + eps) - f(w, tau - eps)) / (2 * eps)
    assert abs(fd_tau - taubar) < 1e-7 * (1 + abs(fd_tau))


@pytest.mark.parametrize("which", ["x0", "lam", "k"])
def test_unrolled_fista_gradient_by_finite_differences(oracle_lib, which):
    from oracle import recon
    p, y, lam, L, x0, iters = _setup()
    _, xK = _loss(p, y, lam, L, iters, x0)
    nr = p["nx"] * p["ny"]
    gK = 2.0 * (xK - p["x_gt"]) / nr     # d mean|x - x_gt|^2 / d(Re, Im) as a complex cotangent
    x0bar, lambar, kbar = recon.fista_unrolled_grad(p, y, lam, L, iters, "haar", 2, x0, gK)
    rng = np.random.default_rng(7)
    eps = 1e-6
    if which == "x0":
        d = rng.standard_normal(nr) + 1j * rng.standard_normal(nr)
        f = lambda e: _loss(p, y, lam, L, iters, x0 + e * d)[0]
        pred = float(np.real(np.vdot(x0bar, d)))
    elif which == "lam":
        f = lambda e: _loss(p, y, lam + e * lam, L, iters, x0)[0]
        pred = lambar * lam
    else:
        d = rng.standard_normal(p["k"].shape) * np.abs(p["k"]).max(axis=1, keepdims=True) * 1e-3
        def f(e):
            q = dict(p)
            q["k"] = p["k"] + e * d
            return _loss(q, y, lam, L, iters, x0)[0]
        pred = float(np.sum(kbar * d))
    fd = (f(eps) - f(-eps)) / (2 * eps)
    print(which, fd, pred)
    assert abs(fd - pred) <= 1e-5 * abs(fd) + 1e-12
