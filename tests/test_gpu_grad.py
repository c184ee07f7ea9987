"""Gradients through unrolled FISTA on the GPU (FP32) with respect to the start image, lambda
and every k_l(t):
* against the FP64 oracle's reverse mode (``oracle.recon.fista_unrolled_grad``) on small
  problems and on one slice of the 170x170 / 16-coil / 12k-sample / 2nd-order + B0 workload
  (3 unrolled iterations; the oracle's own data, lambda, L_f and loss cotangent), bar 1e-3;
* against central finite differences of the GPU forward unroll on the full workload (batch of
  8 slices, 10 iterations), with the bars the piecewise-smooth loss admits (see that test)."""

import numpy as np
import pytest

from paper_2211_07532_gb300 import synth
from tests._data import rel

pytestmark = pytest.mark.gpu
TOL = 1e-3


@pytest.fixture(scope="module")
def ax():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2211_07532_gb300 import build
    build.build()
    import paper_2211_07532_gb300 as ax
    ax.lib()
    return ax


def _small(nx=24, ny=20, seed=31):
    import oracle
    from oracle import recon
    p = synth.make_problem(nx, ny, nt=400, nc=4, order=2, dwell=4e-6, turns=4.0, seed=seed)
    y = (oracle.forward(p, p["x_gt"]) + 0.05 * p["noise"]).astype(np.complex64)
    lam = float(np.float32(0.05 * np.max(np.abs(oracle.adjoint(p, y)))))
    L = recon.power_lipschitz(p, oracle.adjoint(p, y), 40)
    rng = np.random.default_rng(seed)
    x0 = (0.1 * (rng.standard_normal(nx * ny) + 1j * rng.standard_normal(nx * ny))).astype(np.complex64)
    return p, y, lam, L, x0


def test_unrolled_forward_matches_cs_recon(ax):
    import torch
    from paper_2211_07532_gb300.autograd import unrolled_fista
    p, y, lam, L, x0 = _small()
    yg = torch.as_tensor(y, device="cuda")
    x0g = torch.as_tensor(x0, device="cuda")
    k = torch.as_tensor(p["k"], device="cuda")
    xK = unrolled_fista(p, yg, x0g, torch.tensor(lam, dtype=torch.float64), k, 5, L, wavelet="haar", levels=2)
    prob = ax.Problem.from_arrays(p)
    xr, _ = ax.cs_recon(prob, yg, lam, 5, wavelet="haar", levels=2, lipschitz=L, x0=x0g)
    assert rel(xK.detach().cpu().numpy(), xr.cpu().numpy()) < 1e-6


@pytest.mark.parametrize("nx,ny,wavelet,levels", [(24, 20, "haar", 2), (22, 17, "db4", 3)])
def test_gradients_match_oracle_reverse_mode(ax, nx, ny, wavelet, levels):
    """Second case: zero padding 22x17 -> 24x24 and the 8-tap wavelet (crop/pad in the VJP)."""
    import torch
    from oracle import recon
    from paper_2211_07532_gb300.autograd import unrolled_fista
    p, y, lam, L, x0 = _small(nx, ny)
    iters = 5
    yg = torch.as_tensor(y, device="cuda")
    x0g = torch.as_tensor(x0, device="cuda").requires_grad_(True)
    lam_t = torch.tensor(lam, dtype=torch.float64, requires_grad=True)
    k = torch.as_tensor(p["k"], device="cuda").requires_grad_(True)
    xgt = torch.as_tensor(p["x_gt"], device="cuda")
    xK = unrolled_fista(p, yg, x0g, lam_t, k, iters, L, wavelet=wavelet, levels=levels)
    loss = torch.mean(torch.abs(xK - xgt) ** 2)
    loss.backward()
    xK_o = recon.fista(p, y, lam, iters, L, wavelet, levels, x0=x0)
    gK = 2.0 * (xK_o - p["x_gt"]) / (nx * ny)          # the oracle's own loss cotangent
    x0bar, lambar, kbar = recon.fista_unrolled_grad(p, y, lam, L, iters, wavelet, levels, x0, gK)
    ex = rel(x0g.grad.cpu().numpy(), x0bar)
    el = abs(float(lam_t.grad) - lambar) / abs(lambar)
    ek = rel(k.grad.cpu().numpy(), kbar)
    print(f"grad vs oracle: x0 {ex:.2e} lambda {el:.2e} k {ek:.2e}")
    assert ex < TOL and el < TOL and ek < TOL


def test_gradients_match_oracle_diff170(ax):
    """One slice of the differentiation workload at full size (170^2, 16 coils, 12 000 samples,
    2nd order + B0, db4 J=4), 3 unrolled iterations from x0 = 0: the GPU's gradients of
    mean |x_K - x_gt|^2 against the FP64 oracle's reverse mode.  Everything the oracle uses is
    its own: the data (oracle forward + seeded noise), lambda = 1e-3 ||A^H y||_inf, L_f (1.05 x a
    4-step power iteration; any fixed value serves, both sides use it) and the loss cotangent.
    This runs the k-gradient kernel in its full-size configuration (16 coils, split sample runs)."""
    import torch
    import oracle
    from oracle import recon
    from paper_2211_07532_gb300.autograd import unrolled_fista
    p = synth.diff_170(index=0)
    nr = 170 * 170
    y0 = oracle.forward(p, p["x_gt"])
    y = (y0 + np.sqrt(np.mean(np.abs(y0) ** 2)) / p["snr"] * p["noise"]).astype(np.complex64)
    aty = oracle.adjoint(p, y)
    lam = float(np.float32(1e-3 * np.max(np.abs(aty))))
    L = 1.05 * recon.power_lipschitz(p, aty, 4)
    iters = 3
    x0 = np.zeros(nr, np.complex64)
    xK_o = []

    def loss_cotangent(xK):                               # the oracle's own x_K
        xK_o.append(xK)
        return 2.0 * (xK - p["x_gt"]) / nr

    x0bar, lambar, kbar = recon.fista_unrolled_grad(p, y, lam, L, iters, "db4", 4, x0, loss_cotangent)
    xK_o = xK_o[0]

    x0g = torch.as_tensor(x0, device="cuda").requires_grad_(True)
    lam_t = torch.tensor(lam, dtype=torch.float64, requires_grad=True)
    k = torch.as_tensor(p["k"], device="cuda").requires_grad_(True)
    xgt = torch.as_tensor(p["x_gt"], device="cuda")
    xK = unrolled_fista(p, torch.as_tensor(y, device="cuda"), x0g, lam_t, k, iters, L, wavelet="db4", levels=4)
    torch.mean(torch.abs(xK - xgt) ** 2).backward()
    ef = rel(xK.detach().cpu().numpy(), xK_o)
    ex = rel(x0g.grad.cpu().numpy(), x0bar)
    el = abs(float(lam_t.grad) - lambar) / abs(lambar)
    ek = rel(k.grad.cpu().numpy(), kbar)
    print(f"diff170 vs oracle: x_K {ef:.2e}; gradients x0 {ex:.2e} lambda {el:.2e} k {ek:.2e}")
    assert ef < 1e-5
    assert ex < TOL and el < TOL and ek < TOL


def test_gradients_match_finite_differences_diff170(ax):
    """170^2, 16 coils, 12k samples, 2nd order + B0, 10 unrolled iterations, batch of 8 slices;
    loss = mean over slices of mean |x_K - x_gt|^2 (accumulated in FP64); central differences
    with step h = 1e-3 along the normalised gradient of each parameter group.

    The loss is only piecewise smooth: every soft-threshold |w| = tau is a kink, and a
    difference quotient over [p - h, p + h] straddles the kinks it crosses, so its error is
    O(h) rather than O(h^2); and the FP32 rounding of x_K puts noise of ~7e-9 on the loss
    (measured as the scatter of the quotient at small h).  The bars at h = 1e-3 follow:
    * k: the quotient is smooth enough (few kinks move per unit of field change): < 1e-3;
    * x0: kink-limited, O(h): < 5e-3 at h = 1e-3 (measured 2.0e-3), and the error must shrink
      with h (8.7e-4 at 5e-4, 3.7e-4 at 2.5e-4 measured);
    * lambda: every change of lambda moves all thresholds and its derivative is the smallest
      (1.6e-4), so the loss's rounding noise (~1e-8) divided by 2h dominates the quotient at
      h = 1e-3 (measured 6e-3 to 6e-2 between builds).  The test measures that noise itself --
      the loss at lambda (1 +- 1e-6) and (1 +- 2e-6), where the true change (~2e-10) is far below
      it -- and
      holds the quotient to 3 x noise / h plus 1 % of the derivative.
    The analytic gradients themselves are held to 1e-3 against the FP64 oracle's reverse mode
    at this size (test above), and the oracle's against FP64 finite differences to ~1e-7
    (tests/test_oracle_grad.py)."""
    import torch
    import paper_2211_07532_gb300 as axm
    from paper_2211_07532_gb300.autograd import unrolled_fista
    iters, B = 10, 8
    slices = []
    for i in range(B):
        p = synth.diff_170(index=i)
        prob = axm.Problem.from_arrays(p)
        ws = axm.workspace(prob)
        axm.prepare(prob, ws)
        xg = torch.as_tensor(p["x_gt"], device="cuda")
        y0 = axm.a_exp_forward(prob, xg, ws)
        y = (y0 + float(torch.sqrt(torch.mean(y0.abs() ** 2))) / p["snr"]
             * torch.as_tensor(p["noise"], device="cuda")).contiguous()
        _, L = axm.cs_recon(prob, y, 0.0, 0, n_power=30)
        lam = 1e-3 * float(axm.a_exp_adjoint(prob, y, ws).abs().max())
        slices.append((p, y, xg, float(L.cpu()[0]), lam))

    def total_loss(x0s, lam_scale, ks):
        out = 0.0
        for (p, y, xg, L, lam), x0, k in zip(slices, x0s, ks):
            xK = unrolled_fista(p, y, x0, lam_scale * lam, k, iters, L, wavelet="db4", levels=4)
            out = out + torch.mean(torch.abs(xK.to(torch.complex128) - xg.to(torch.complex128)) ** 2)
        return out / B

    x0s = [torch.zeros(170 * 170, dtype=torch.complex64, device="cuda").requires_grad_(True) for _ in slices]
    lam_s = torch.tensor(1.0, dtype=torch.float64, requires_grad=True)
    ks = [torch.as_tensor(s[0]["k"], device="cuda").requires_grad_(True) for s in slices]
    loss = total_loss(x0s, lam_s, ks)
    loss.backward()
    # directions: x0 with unit RMS per voxel, k with at most 1 rad of phase change per unit
    # step at the FOV edge, lambda relative (lam_s = 1)
    gx = torch.cat([g.grad for g in x0s])
    dx = [g.grad / torch.linalg.vector_norm(gx) * (170.0 * np.sqrt(B)) for g in x0s]
    hmax = [torch.as_tensor(np.abs(s[0]["h"]).max(axis=1), device="cuda") for s in slices]
    gk = [k.grad * hm[:, None] for k, hm in zip(ks, hmax)]
    nk = float(max(torch.max(torch.abs(g)) for g in gk))
    dk = [g / nk / hm.clamp_min(1e-6)[:, None] for g, hm in zip(gk, hmax)]
    with torch.no_grad():
        pred = {"x0": sum(float(torch.sum((g.grad.conj() * d).real)) for g, d in zip(x0s, dx)),
                "lambda": float(lam_s.grad),
                "k": sum(float(torch.sum(k.grad * d)) for k, d in zip(ks, dk))}
        shift = {"x0": lambda h: (total_loss([x + h * d for x, d in zip(x0s, dx)], lam_s, ks),
                                  total_loss([x - h * d for x, d in zip(x0s, dx)], lam_s, ks)),
                 "lambda": lambda h: (total_loss(x0s, lam_s + h, ks), total_loss(x0s, lam_s - h, ks)),
                 "k": lambda h: (total_loss(x0s, lam_s, [k + h * d for k, d in zip(ks, dk)]),
                                 total_loss(x0s, lam_s, [k - h * d for k, d in zip(ks, dk)]))}
        base = float(total_loss(x0s, lam_s, ks))
        noise = max(abs(float(total_loss(x0s, lam_s + e, ks)) - base - e * pred["lambda"]) for e in (1e-6, -1e-6, 2e-6, -2e-6))
        err = {}
        steps = {"x0": (1e-3, 5e-4, 2.5e-4), "k": (1e-3,), "lambda": (1e-3,)}
        for name in pred:
            for h in steps[name]:
                lp, lm = shift[name](h)
                fd = (float(lp) - float(lm)) / (2 * h)
                err[(name, h)] = abs(fd - pred[name]) / abs(pred[name])
                print(f"FD {name} h={h:.2e}: analytic {pred[name]:.6e} fd {fd:.6e} rel {err[(name, h)]:.2e}")
    assert err[("k", 1e-3)] < TOL
    assert err[("x0", 1e-3)] < 5 * TOL
    assert err[("x0", 2.5e-4)] < err[("x0", 5e-4)] < err[("x0", 1e-3)]   # the O(h) kink error shrinks
    lam_bar = (3.0 * noise / 1e-3 + 0.01 * abs(pred["lambda"])) / abs(pred["lambda"])
    print(f"FD lambda: loss noise {noise:.2e}, bar {lam_bar:.2e}")
    assert err[("lambda", 1e-3)] < lam_bar
