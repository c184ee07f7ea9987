"""Parity of the BF16 tensor-core form (tcgen05) with the FP64 oracle.

Operator bound (BF16, round to nearest): every real component of the encoding elements and of
the contraction operand is rounded once to 8 significant bits.  The rounding error is uniform in
+-ulp/2 and ulp/|v| lies between 2^-8 and 2^-7, so for mantissas spread over an octave the rms
relative error of one rounding is 2^-8/sqrt(6) = 1.6e-3; a product of two rounded factors has
sqrt(2) times that, 2.3e-3, and the independent errors of a sum add in quadrature, so the
relative L2 error of A x or A^H y for white inputs is ~2.3e-3.  The test bound is 5e-3.

Reconstruction bound: the oracle runs the same FISTA on its BF16 emulation
(``oracle.precision``: the same two roundings written out, everything else exact); the
emulated image's distance to the exact FP64 image is what the rounding alone does after this
many iterations, and the GPU image must stay within 3x that distance."""

import numpy as np
import pytest

from paper_2211_07532_gb300 import synth
from tests._data import rel, simulated

pytestmark = pytest.mark.gpu
TOL_OP = 5e-3
RECON_MARGIN = 3.0   # GPU image error / emulated BF16 image error


@pytest.fixture(scope="module")
def ax():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2211_07532_gb300 import build
    build.build()
    import paper_2211_07532_gb300 as ax
    ax.lib()
    return ax


def _apply(ax, p, x, y, with_b0=True):
    import torch
    prob = ax.Problem.from_arrays(p, with_b0=with_b0)
    ws = ax.workspace(prob, ax.BF16_TC)
    ax.prepare(prob, ws, ax.BF16_TC)
    f = ax.a_exp_forward(prob, torch.as_tensor(x, device="cuda"), ws, precision=ax.BF16_TC)
    a = ax.a_exp_adjoint(prob, torch.as_tensor(y, device="cuda"), ws, precision=ax.BF16_TC)
    torch.cuda.synchronize()
    assert ax.read_status(ws) == 0
    return f.cpu().numpy(), a.cpu().numpy()


SHAPES = [  # nx, ny, nt, nc, order, b0
    (64, 64, 2048, 8, 2, True),     # the 64^2 / 8-coil / 2nd-order workload's shapes
    (13, 11, 777, 3, 3, True),      # ragged tiles and samples, 3 coils -> 8-wide
    (17, 9, 1025, 20, 3, True),     # 20 coils -> 32-wide
    (24, 16, 300, 12, 1, False),    # 12 coils -> 16-wide, no B0
    (40, 40, 1500, 32, 3, True),
    (1, 1, 1, 1, 0, False),
]


@pytest.mark.parametrize("shape", SHAPES)
def test_bf16_operator_matches_oracle(ax, shape):
    import oracle
    nx, ny, nt, nc, order, b0 = shape
    p = synth.make_problem(nx, ny, nt=nt, nc=nc, order=order, dwell=4e-6, turns=max(nx, ny) / 8.0 + 1,
                           seed=4321 + nx + nt, with_b0=b0)
    rng = np.random.default_rng(nt + 1)
    x = synth.random_image(rng, nx * ny)
    y = synth.random_kspace(rng, nc, nt)
    f, a = _apply(ax, p, x, y, with_b0=b0)
    q = dict(p)
    if not b0:
        q["omega"] = None
    ef, ea = rel(f, oracle.forward(q, x)), rel(a, oracle.adjoint(q, y))
    print(f"bf16 {shape}: forward rel {ef:.2e} adjoint rel {ea:.2e}")
    assert ef < TOL_OP and ea < TOL_OP


def test_bf16_tiny64_error_table(ax):
    """The 64^2 precision workload: relative L2 error against the FP64 oracle for A x,
    A^H y and the final FISTA image (20 iterations, Haar J=3, same L_f on both sides)."""
    import torch
    import oracle
    from oracle import recon
    p, y, lam = simulated("tiny_64")
    f, a = _apply(ax, p, p["x_gt"], y)
    ef = rel(f, oracle.forward(p, p["x_gt"]))
    ea = rel(a, oracle.adjoint(p, y))
    Lf = recon.power_lipschitz(p, oracle.adjoint(p, y), 30)
    prob = ax.Problem.from_arrays(p)
    x, L = ax.cs_recon(prob, torch.as_tensor(y, device="cuda"), lam, p["iters"], precision=ax.BF16_TC,
                       wavelet="haar", levels=3, lipschitz=Lf)
    from oracle import precision
    ref = recon.fista(p, y, lam, p["iters"], Lf, "haar", 3)
    emul = recon.fista(p, y, lam, p["iters"], Lf, "haar", 3, ops=precision.bf16_operators(p))
    ex, ee = rel(x.cpu().numpy(), ref), rel(emul, ref)
    print(f"bf16 tiny64: A x rel {ef:.2e}, A^H y rel {ea:.2e}, FISTA image rel {ex:.2e} "
          f"(BF16 emulation {ee:.2e}); nrmse vs phantom {rel(x.cpu().numpy(), p['x_gt']):.4f} "
          f"(oracle {rel(ref, p['x_gt']):.4f})")
    assert ef < TOL_OP and ea < TOL_OP and ex < RECON_MARGIN * ee


def test_bf16_power_iteration(ax):
    import torch
    import oracle
    from oracle import recon
    p, y, lam = simulated("tiny_64")
    Lf = recon.power_lipschitz(p, oracle.adjoint(p, y), 30)
    prob = ax.Problem.from_arrays(p)
    _, L = ax.cs_recon(prob, torch.as_tensor(y, device="cuda"), lam, 0, precision=ax.BF16_TC, n_power=30)
    Lg = float(L.cpu().numpy()[0])
    print(f"bf16 L_f {Lg:.6e} oracle {Lf:.6e} rel {abs(Lg - Lf) / Lf:.2e}")
    assert abs(Lg - Lf) < TOL_OP * Lf


def test_bf16_slice200_sampled(ax):
    """Full 200^2 / 32-coil / 24k-sample / 3rd-order + B0 size, sampled outputs."""
    import torch
    import oracle
    p = synth.slice_200()
    rng = np.random.default_rng(9)
    y = synth.random_kspace(rng, p["nc"], p["nt"])
    f, a = _apply(ax, p, p["x_gt"], y)
    ts = np.unique(np.concatenate([[0, p["nt"] - 1], rng.choice(p["nt"], 40, replace=False)]))
    rs = np.unique(np.concatenate([[0, 39999], rng.choice(40000, 40, replace=False)]))
    ef = rel(f[:, ts], oracle.forward_rows(p, p["x_gt"], ts))
    ea = rel(a[rs], oracle.adjoint_rows(p, y, rs))
    print(f"bf16 slice200 sampled: forward rel {ef:.2e} adjoint rel {ea:.2e}")
    assert ef < TOL_OP and ea < TOL_OP


@pytest.mark.parametrize("precision", ["bf16", "fp16x2"])
def test_tensor_core_operators_are_repeatable(ax, precision):
    """The persistent tensor-core kernels hand stages between warp roles through mbarriers;
    a missing or misplaced wait shows up as results that change from run to run.  Full
    200^2 / 32-coil / 24k-sample size, 12 applications each way: bitwise identical."""
    import torch
    prec = {"bf16": ax.BF16_TC, "fp16x2": ax.FP16X2_TC}[precision]
    p = synth.slice_200()
    prob = ax.Problem.from_arrays(p)
    ws = ax.workspace(prob, prec)
    ax.prepare(prob, ws, prec)
    x = torch.as_tensor(p["x_gt"], device="cuda")
    y = torch.as_tensor(p["noise"], device="cuda")
    f0 = ax.a_exp_forward(prob, x, ws, precision=prec).clone()
    a0 = ax.a_exp_adjoint(prob, y, ws, precision=prec).clone()
    for _ in range(12):
        assert torch.equal(ax.a_exp_forward(prob, x, ws, precision=prec), f0)
        assert torch.equal(ax.a_exp_adjoint(prob, y, ws, precision=prec), a0)
    torch.cuda.synchronize()
    assert ax.read_status(ws) == 0
