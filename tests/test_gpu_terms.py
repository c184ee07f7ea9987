"""Field models beyond 3rd order on the GPU: 4th-order solid harmonics and the second-order
concomitant-field rows (Fig. S3d) as extra terms of the same operator, 21 to 30 terms with
B0 (the 32-wide term padding).  Every form against the FP64 oracle, plus the k-gradient of
the unrolled FISTA step.  Bars: FP32 and FP16 hi+lo 1e-5, BF16 5e-3 (the operator bars),
gradients 1e-3."""

import math

import numpy as np
import pytest

from paper_2211_07532_gb300 import synth
from tests._data import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ax():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2211_07532_gb300 import build
    build.build()
    import paper_2211_07532_gb300 as ax
    ax.lib()
    return ax


CASES = [  # nx, ny, nt, nc, order, concomitant, b0 -> terms
    (37, 29, 1500, 8, 4, True, True),      # 25 + 4 + B0 = 30
    (21, 26, 777, 20, 4, False, False),    # 25
    (16, 16, 1024, 32, 3, True, True),     # 16 + 4 + B0 = 21 (smallest count on the 32 padding)
    (9, 5, 129, 3, 4, True, False),        # 29, ragged everything
]
FORMS = [("fp32", 1e-5), ("bf16", 5e-3), ("fp16x2", 1e-5)]


def _problem(case):
    nx, ny, nt, nc, order, conc, b0 = case
    p = synth.make_problem(nx, ny, nt=nt, nc=nc, order=order, dwell=4e-6, turns=max(nx, ny) / 8.0 + 1,
                           tilt=math.radians(25), concomitant=conc, z0=0.01, seed=777 + nx * 3 + nt,
                           with_b0=b0)
    q = dict(p)
    if not b0:
        q["omega"] = None
    return p, q, b0


@pytest.mark.parametrize("form,tol", FORMS)
@pytest.mark.parametrize("case", CASES)
def test_operator_with_extended_field_terms(ax, case, form, tol):
    import oracle
    import torch
    prec = {"fp32": ax.FP32, "bf16": ax.BF16_TC, "fp16x2": ax.FP16X2_TC}[form]
    p, q, b0 = _problem(case)
    nt, nc = case[2], case[3]
    assert 21 <= p["nl"] + b0 <= 32
    rng = np.random.default_rng(nt + nc)
    x = synth.random_image(rng, case[0] * case[1])
    y = synth.random_kspace(rng, nc, nt)
    prob = ax.Problem.from_arrays(p, with_b0=b0)
    ws = ax.workspace(prob, prec)
    ax.prepare(prob, ws, prec)
    f = ax.a_exp_forward(prob, torch.as_tensor(x, device="cuda"), ws, precision=prec)
    a = ax.a_exp_adjoint(prob, torch.as_tensor(y, device="cuda"), ws, precision=prec)
    torch.cuda.synchronize()
    assert ax.read_status(ws) == 0
    ef, ea = rel(f.cpu().numpy(), oracle.forward(q, x)), rel(a.cpu().numpy(), oracle.adjoint(q, y))
    print(f"{form} {case} terms {p['nl'] + b0}: forward rel {ef:.2e} adjoint rel {ea:.2e}")
    assert ef < tol and ea < tol


def test_k_gradient_with_extended_field_terms(ax):
    """Reverse mode through 4 unrolled FISTA steps with 30 field terms, against the oracle."""
    import oracle
    import torch
    from oracle import recon
    from paper_2211_07532_gb300.autograd import unrolled_fista
    nx, ny = 20, 18
    p = synth.make_problem(nx, ny, nt=400, nc=4, order=4, dwell=4e-6, turns=4.0, tilt=math.radians(25),
                           concomitant=True, z0=0.01, seed=91)
    y = (oracle.forward(p, p["x_gt"]) + 0.05 * p["noise"]).astype(np.complex64)
    lam = float(np.float32(0.05 * np.max(np.abs(oracle.adjoint(p, y)))))
    L = recon.power_lipschitz(p, oracle.adjoint(p, y), 40)
    rng = np.random.default_rng(92)
    x0 = (0.1 * (rng.standard_normal(nx * ny) + 1j * rng.standard_normal(nx * ny))).astype(np.complex64)
    iters = 4
    x0g = torch.as_tensor(x0, device="cuda").requires_grad_(True)
    lam_t = torch.tensor(lam, dtype=torch.float64, requires_grad=True)
    k = torch.as_tensor(p["k"], device="cuda").requires_grad_(True)
    xK = unrolled_fista(p, torch.as_tensor(y, device="cuda"), x0g, lam_t, k, iters, L, wavelet="haar", levels=2)
    loss = torch.mean(torch.abs(xK - torch.as_tensor(p["x_gt"], device="cuda")) ** 2)
    loss.backward()
    gK = 2.0 * (xK.detach().cpu().numpy().astype(np.complex128) - p["x_gt"]) / (nx * ny)
    x0bar, lambar, kbar = recon.fista_unrolled_grad(p, y, lam, L, iters, "haar", 2, x0, gK)
    ex, ek = rel(x0g.grad.cpu().numpy(), x0bar), rel(k.grad.cpu().numpy(), kbar)
    el = abs(float(lam_t.grad) - lambar) / abs(lambar)
    print(f"30 terms, grad vs oracle: x0 {ex:.2e} lambda {el:.2e} k {ek:.2e}")
    assert ex < 1e-3 and el < 1e-3 and ek < 1e-3


def test_too_many_terms_is_rejected(ax):
    """33 terms (4th order + concomitant rows + 3 more + B0) exceed the 32-wide padding."""
    import torch
    p = synth.make_problem(8, 8, nt=64, nc=2, order=4, concomitant=True, seed=5)
    k = np.concatenate([p["k"], p["k"][:3]], axis=0)
    h = np.concatenate([p["h"], p["h"][:3]], axis=0)
    q = dict(p, k=np.ascontiguousarray(k), h=np.ascontiguousarray(h), nl=32)
    prob = ax.Problem.from_arrays(q)
    with pytest.raises(Exception):
        ax.workspace(prob)
    torch.cuda.synchronize()
