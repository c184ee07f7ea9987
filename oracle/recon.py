"""FP64 solvers around A_exp: Lipschitz estimate, FISTA, CGLS (Eq. 1; Sec. 2.1).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Readings of the paper fixed here:
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


def _operators(prob, ops):
    """(A, A^H) as callables: the exact FP64 double sums, or the pair ``ops`` (e.g. the
    rounding emulation of ``oracle.precision``) when given."""
    if ops is not None:
        return ops
    return (lambda v: forward(prob, v)), (lambda r: adjoint(prob, r))


def power_lipschitz(prob, v0, n_pow: int = 30, ops=None):
    """L_f = 2 mu_n after n_pow power iterations on A^H A from v0."""
    fwd, adj = _operators(prob, ops)
    v = np.asarray(v0, np.complex128).reshape(-1)
    v = v / np.linalg.norm(v)
    mu = 0.0
    for _ in range(n_pow):
        w = adj(fwd(v))
        mu = float(np.real(np.vdot(v, w)))
        v = w / np.linalg.norm(w)
    return 2.0 * mu


def objective(prob, x, y, lam, name, levels):
    r = forward(prob, x) - np.asarray(y)
    return float(np.sum(np.abs(r) ** 2)) + lam * wv.l1_detail(x, prob["ny"], prob["nx"], name, levels)


def fista(prob, y, lam, iters, lipschitz, name, levels, x0=None, history=False, ops=None):
    """FISTA on Eq. (1): returns x_iters (and the list of iterates if ``history``)."""
    fwd, adj = _operators(prob, ops)
    nr = prob["nx"] * prob["ny"]
    y = np.asarray(y, np.complex128)
    x_prev = np.zeros(nr, np.complex128) if x0 is None else np.asarray(x0, np.complex128).reshape(nr)
    z = x_prev.copy()
    t = 1.0
    tau = lam / lipschitz
    hist = []
    for _ in range(iters):
        grad = 2.0 * adj(fwd(z) - y)
        v = z - grad / lipschitz
        x = wv.prox(v, prob["ny"], prob["nx"], name, levels, tau)
        t_next = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        z = x + ((t - 1.0) / t_next) * (x - x_prev)
        x_prev = x
        t = t_next
        if history:
            hist.append(x.copy())
    return (x_prev, hist) if history else x_prev


def cgls(prob, y, iters, ops=None):
    """Conjugate gradient least squares on A^H A x = A^H y from x = 0."""
    fwd, adj = _operators(prob, ops)
    nr = prob["nx"] * prob["ny"]
    y = np.asarray(y, np.complex128)
    x = np.zeros(nr, np.complex128)
    r = y.copy()
    s = adj(r)
    p = s.copy()
    gamma = float(np.real(np.vdot(s, s)))
    for _ in range(iters):
        if gamma == 0.0:
            break
        q = fwd(p)
        alpha = gamma / float(np.real(np.vdot(q, q)))
        x = x + alpha * p
        r = r - alpha * q
        s = adj(r)
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


def soft_vjp(w, gbar, tau):
    """VJP of the complex soft-threshold S(w) = w max(0, 1 - tau/|w|) at w for cotangent gbar.

    For |w| > tau the real Jacobian is (1 - tau/r) I + (tau/r^3) [a b]^T [a b] (w = a + ib,
    r = |w|), symmetric, so wbar = (1 - tau/r) gbar + (tau/r^3) w Re(conj(w) gbar); dS/dtau =
    -w/r gives taubar = -Re(conj(gbar) w)/r.  For |w| <= tau both are zero.
    Returns (wbar, taubar summed over all entries)."""
    w = np.asarray(w, np.complex128)
    g = np.asarray(gbar, np.complex128)
    r = np.abs(w)
    act = r > tau
    rs = np.where(act, r, 1.0)
    wbar = np.where(act, (1.0 - tau / rs) * g + (tau / rs ** 3) * w * np.real(np.conj(w) * g), 0.0)
    taubar = float(np.sum(np.where(act, -np.real(np.conj(g) * w) / rs, 0.0)))
    return wbar, taubar


def fista_unrolled_grad(prob, y, lam, lipschitz, iters, name, levels, x0, xbar_K):
    """Reverse-mode gradient through `iters` FISTA steps (x_0 -> x_iters), FP64.

    Cotangent convention: for a real loss, gbar = dLoss/dRe + i dLoss/dIm.  Given the
    cotangent xbar_K of x_iters (an array, or a function of x_iters that returns it),
    returns (x0bar complex [nr], lambar float, kbar [nl][nt]) with L_f held fixed.  Recursion (z_{k+1} = (1+b_k) x_k - b_k x_{k-1}, x_k = P(v_k),
    v_k = z_k - (2/L) A^H (A z_k - y)):
        xbar_k = (1+b_k) zbar_{k+1} - b_{k+1} zbar_{k+2}  (+ xbar_K at k = iters)
        vbar_k = crop W^H S'^T W pad xbar_k,   lambar += taubar / L
        zbar_k = vbar_k - (2/L) A^H A vbar_k
        kbar  += -(2/L) Re[ d/dk <A vbar_k, A z_k> + d/dk <vbar_k, A^H r_k> ]   (r_k = A z_k - y)
        x0bar  = zbar_1 - b_1 zbar_2
    """
    from . import adjoint_dk, forward_dk
    ny, nx = prob["ny"], prob["nx"]
    nr = nx * ny
    y = np.asarray(y, np.complex128)
    L = float(lipschitz)
    tau = lam / L
    shp = wv.padded_shape(ny, nx, levels)
    mask = wv.detail_mask(shp, levels)
    # forward pass with checkpoints z_k, x_k and the momentum weights b_k
    x = [np.asarray(x0, np.complex128).reshape(nr)]
    z = [None, x[0].copy()]
    b = [0.0] * (iters + 3)
    t = 1.0
    for k in range(1, iters + 1):
        v = z[k] - 2.0 * adjoint(prob, forward(prob, z[k]) - y) / L
        x.append(wv.prox(v, ny, nx, name, levels, tau))
        t_next = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        b[k] = (t - 1.0) / t_next
        t = t_next
        z.append(x[k] + b[k] * (x[k] - x[k - 1]))
    # backward pass
    zbar = [None] * (iters + 3)
    zbar[iters + 1] = np.zeros(nr, np.complex128)
    zbar[iters + 2] = np.zeros(nr, np.complex128)
    kbar = np.zeros(np.shape(prob["k"]))
    lambar = 0.0
    for k in range(iters, 0, -1):
        xbar = (1.0 + b[k]) * zbar[k + 1] - b[k + 1] * zbar[k + 2]
        if k == iters:
            xK_bar = xbar_K(x[iters]) if callable(xbar_K) else xbar_K
            xbar = xbar + np.asarray(xK_bar, np.complex128).reshape(nr)
        r = forward(prob, z[k]) - y
        v = z[k] - 2.0 * adjoint(prob, r) / L
        w = wv.dwt2(wv.pad(v.reshape(ny, nx), shp), name, levels)
        gw = wv.dwt2(wv.pad(xbar.reshape(ny, nx), shp), name, levels)
        wbar_d, taubar = soft_vjp(w[mask], gw[mask], tau)
        gw[mask] = wbar_d
        lambar += taubar / L
        vbar = wv.idwt2(gw, name, levels)[:ny, :nx].reshape(nr)
        u = forward(prob, vbar)
        zbar[k] = vbar - 2.0 * adjoint(prob, u) / L
        kbar += -(2.0 / L) * np.real(forward_dk(prob, z[k], u) + adjoint_dk(prob, r, vbar))
    x0bar = zbar[1] - b[1] * zbar[2]
    return x0bar, lambar, kbar
