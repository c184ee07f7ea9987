"""FP64 solvers around A_exp: Lipschitz estimate, FISTA, CGLS (Eq. 1; Sec. 2.1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Readings of the paper fixed here (each also listed in the design notes):
* objective F(x) = ||A x - y||_2^2 + lam * sum_detail |(W x)_j|, Eq. (1) as printed
  (no 1/2), low-pass weight 0 (Supporting Information S1);
* gradient of the data term 2 A^H (A x - y), Lipschitz constant L_f = 2 lambda_max(A^H A),
  step 1/L_f, threshold lam/L_f;
* FISTA in the Beck-Teboulle form, x_0 = 0 (or a given start), fixed iteration
  count; with an orthonormal W the "balanced" variant of Sec. 2.1 has the same prox;
* power iteration: v_0 = given vector normalised, mu_i = Re<v_{i-1}, A^H A v_{i-1}>,
  v_i = A^H A v_{i-1} / ||A^H A v_{i-1}||, L_f = 2 mu_n;
* CGLS: conjugate gradient on the normal equations with a fixed count (Sec. 2.1, 20 iterations).
"""

from __future__ import annotations

import math

import numpy as np

from . import adjoint, forward
from . import wavelet as wv


def normal_op(prob, v):
    return adjoint(prob, forward(prob, v))


def power_lipschitz(prob, v0, n_pow: int = 30):
    """L_f = 2 mu_n after n_pow power iterations on A^H A from v0."""
    v = np.asarray(v0, np.complex128).reshape(-1)
    v = v / np.linalg.norm(v)
    mu = 0.0
    for _ in range(n_pow):
        w = normal_op(prob, v)
        mu = float(np.real(np.vdot(v, w)))
        v = w / np.linalg.norm(w)
    return 2.0 * mu


def objective(prob, x, y, lam, name, levels):
    r = forward(prob, x) - np.asarray(y)
    return float(np.sum(np.abs(r) ** 2)) + lam * wv.l1_detail(x, prob["ny"], prob["nx"], name, levels)


def fista(prob, y, lam, iters, lipschitz, name, levels, x0=None, history=False):
    """FISTA on Eq. (1): returns x_iters (and the list of iterates if ``history``)."""
    nr = prob["nx"] * prob["ny"]
    y = np.asarray(y, np.complex128)
    x_prev = np.zeros(nr, np.complex128) if x0 is None else np.asarray(x0, np.complex128).reshape(nr)
    z = x_prev.copy()
    t = 1.0
    tau = lam / lipschitz
    hist = []
    for _ in range(iters):
        grad = 2.0 * adjoint(prob, forward(prob, z) - y)
        v = z - grad / lipschitz
        x = wv.prox(v, prob["ny"], prob["nx"], name, levels, tau)
        t_next = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        z = x + ((t - 1.0) / t_next) * (x - x_prev)
        x_prev = x
        t = t_next
        if history:
            hist.append(x.copy())
    return (x_prev, hist) if history else x_prev


def fista_step(prob, y, lam, lipschitz, name, levels, z, x_prev, t):
    """One FISTA iteration from (z_k, x_{k-1}, t_k): returns (x_k, z_{k+1}, t_{k+1})."""
    grad = 2.0 * adjoint(prob, forward(prob, z) - y)
    v = z - grad / lipschitz
    x = wv.prox(v, prob["ny"], prob["nx"], name, levels, lam / lipschitz)
    t_next = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
    return x, x + ((t - 1.0) / t_next) * (x - x_prev), t_next


def cgls(prob, y, iters):
    """Conjugate gradient least squares on A^H A x = A^H y from x = 0."""
    nr = prob["nx"] * prob["ny"]
    y = np.asarray(y, np.complex128)
    x = np.zeros(nr, np.complex128)
    r = y.copy()
    s = adjoint(prob, r)
    p = s.copy()
    gamma = float(np.real(np.vdot(s, s)))
    for _ in range(iters):
        if gamma == 0.0:
            break
        q = forward(prob, p)
        alpha = gamma / float(np.real(np.vdot(q, q)))
        x = x + alpha * p
        r = r - alpha * q
        s = adjoint(prob, r)
        gamma_new = float(np.real(np.vdot(s, s)))
        p = s + (gamma_new / gamma) * p
        gamma = gamma_new
    return x


def nrmse(x, x_ref) -> float:
    """||x - x_ref||_2 / ||x_ref||_2 (the normalisation Sec. 2.2.2 leaves unstated)."""
    x = np.asarray(x).reshape(-1)
    x_ref = np.asarray(x_ref).reshape(-1)
    return float(np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref))


def default_lambda(prob, y, rel: float = 1e-3) -> float:
    """lam = rel * ||A^H y||_inf (the workload's fixed-lambda rule)."""
    return rel * float(np.max(np.abs(adjoint(prob, y))))
