"""Parity of the FP16 hi+lo tensor-core form (tcgen05) with the FP64 oracle.

Bound.  Each operand value v is carried as v_hi + 2^-11 v_lo' with v_hi = fp16(v) (11
significant bits) and v_lo' = fp16(2^11 (v - v_hi)): the representation error is at most
half an FP16 ulp of the residual, 2^-22 |v| (2.4e-7).  The dropped lo x lo product is of
the same order, so a product of two split factors carries ~2^-21 relative error, below the
FP32 phase arithmetic that both the CUDA-core and the tensor-core forms share (2.8e-7 in
the tile-centred form).  The FP32 requirement, relative L2 error below 1e-5, therefore
applies to this form unchanged: the tests use the FP32 bounds.

The B operand is scaled by a power of two taken from its largest component; the scale
cases below (1e-30 and 1e25 times a unit-scale image, an all-zero image) check that the
scaling neither loses precision nor overflows FP16."""

import numpy as np
import pytest

from paper_2211_07532_gb300 import synth
from tests._data import rel, simulated

pytestmark = pytest.mark.gpu
TOL = 1e-5


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
    ws = ax.workspace(prob, ax.FP16X2_TC)
    ax.prepare(prob, ws, ax.FP16X2_TC)
    f = ax.a_exp_forward(prob, torch.as_tensor(x, device="cuda"), ws, precision=ax.FP16X2_TC)
    a = ax.a_exp_adjoint(prob, torch.as_tensor(y, device="cuda"), ws, precision=ax.FP16X2_TC)
    torch.cuda.synchronize()
    assert ax.read_status(ws) == 0
    return f.cpu().numpy(), a.cpu().numpy()


SHAPES = [  # nx, ny, nt, nc, order, b0
    (64, 64, 2048, 8, 2, True),
    (13, 11, 777, 3, 3, True),
    (17, 9, 1025, 20, 3, True),
    (24, 16, 300, 12, 1, False),
    (40, 40, 1500, 32, 3, True),
    (1, 1, 1, 1, 0, False),
]


@pytest.mark.parametrize("shape", SHAPES)
def test_fp16x2_operator_matches_oracle(ax, shape):
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
    print(f"fp16x2 {shape}: forward rel {ef:.2e} adjoint rel {ea:.2e}")
    assert ef < TOL and ea < TOL


@pytest.mark.parametrize("scale", [1e-30, 1e25])
def test_fp16x2_scaling_extremes(ax, scale):
    """Inputs far outside FP16's range: the power-of-two scaling keeps the relative error."""
    import oracle
    p = synth.make_problem(24, 20, nt=700, nc=8, order=2, dwell=4e-6, turns=4.0, seed=91)
    rng = np.random.default_rng(92)
    x = (synth.random_image(rng, 24 * 20) * np.float32(scale)).astype(np.complex64)
    y = (synth.random_kspace(rng, 8, 700) * np.float32(scale)).astype(np.complex64)
    f, a = _apply(ax, p, x, y)
    ef, ea = rel(f, oracle.forward(p, x)), rel(a, oracle.adjoint(p, y))
    print(f"fp16x2 scale {scale:.0e}: forward rel {ef:.2e} adjoint rel {ea:.2e}")
    assert ef < TOL and ea < TOL


def test_fp16x2_zero_input_gives_zero(ax):
    p = synth.make_problem(16, 16, nt=300, nc=4, order=2, seed=93)
    f, a = _apply(ax, p, np.zeros(256, np.complex64), np.zeros((4, 300), np.complex64))
    assert np.all(f == 0) and np.all(a == 0)


def test_fp16x2_tiny64_error_table(ax):
    """The 64^2 precision workload: A x, A^H y and the final FISTA image (20 iterations,
    Haar J=3, same L_f on both sides) against the FP64 oracle."""
    import torch
    import oracle
    from oracle import recon
    p, y, lam = simulated("tiny_64")
    f, a = _apply(ax, p, p["x_gt"], y)
    ef = rel(f, oracle.forward(p, p["x_gt"]))
    ea = rel(a, oracle.adjoint(p, y))
    Lf = recon.power_lipschitz(p, oracle.adjoint(p, y), 30)
    prob = ax.Problem.from_arrays(p)
    x, L = ax.cs_recon(prob, torch.as_tensor(y, device="cuda"), lam, p["iters"], precision=ax.FP16X2_TC,
                       wavelet="haar", levels=3, lipschitz=Lf)
    ref = recon.fista(p, y, lam, p["iters"], Lf, "haar", 3)
    ex = rel(x.cpu().numpy(), ref)
    print(f"fp16x2 tiny64: A x rel {ef:.2e}, A^H y rel {ea:.2e}, FISTA image rel {ex:.2e}")
    assert ef < TOL and ea < TOL and ex < TOL


def test_fp16x2_power_iteration(ax):
    import torch
    import oracle
    from oracle import recon
    p, y, lam = simulated("tiny_64")
    Lf = recon.power_lipschitz(p, oracle.adjoint(p, y), 30)
    prob = ax.Problem.from_arrays(p)
    _, L = ax.cs_recon(prob, torch.as_tensor(y, device="cuda"), lam, 0, precision=ax.FP16X2_TC, n_power=30)
    Lg = float(L.cpu().numpy()[0])
    print(f"fp16x2 L_f {Lg:.6e} oracle {Lf:.6e} rel {abs(Lg - Lf) / Lf:.2e}")
    assert abs(Lg - Lf) < TOL * Lf


def test_fp16x2_slice200_sampled(ax):
    """Full 200^2 / 32-coil / 24k-sample / 3rd-order + B0 size, sampled outputs."""
    import oracle
    p = synth.slice_200()
    rng = np.random.default_rng(9)
    y = synth.random_kspace(rng, p["nc"], p["nt"])
    f, a = _apply(ax, p, p["x_gt"], y)
    ts = np.unique(np.concatenate([[0, p["nt"] - 1], rng.choice(p["nt"], 40, replace=False)]))
    rs = np.unique(np.concatenate([[0, 39999], rng.choice(40000, 40, replace=False)]))
    ef = rel(f[:, ts], oracle.forward_rows(p, p["x_gt"], ts))
    ea = rel(a[rs], oracle.adjoint_rows(p, y, rs))
    print(f"fp16x2 slice200 sampled: forward rel {ef:.2e} adjoint rel {ea:.2e}")
    assert ef < TOL and ea < TOL


def test_fp16x2_batch_matches_oracle(ax):
    """A small ragged batch through the persistent batched solver in the FP16 hi+lo form."""
    import torch
    import oracle
    from oracle import recon
    shapes = [(24, 24, 700), (17, 13, 333), (32, 32, 1200)]
    probs, ys, lams = [], [], []
    for i, (nx, ny, nt) in enumerate(shapes):
        p = synth.make_problem(nx, ny, nt=nt, nc=8, order=3, dwell=4e-6, turns=max(nx, ny) / 8.0 + 1,
                               seed=777 + i)
        y0 = oracle.forward(p, p["x_gt"])
        ys.append((y0 + 0.05 * np.sqrt(np.mean(np.abs(y0) ** 2)) * p["noise"]).astype(np.complex64))
        lams.append(float(np.float32(2e-2 * np.max(np.abs(oracle.adjoint(p, ys[-1]))))))
        probs.append(p)
    P = [ax.Problem.from_arrays(p) for p in probs]
    Y = [torch.as_tensor(y, device="cuda") for y in ys]
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        xs, L = ax.cs_recon_batched(P, Y, lams, 8, precision=ax.FP16X2_TC, wavelet="db4", levels=2, n_power=20)
        torch.cuda.synchronize()
    Ls = L.cpu().numpy()
    for q, (p, y, lam) in enumerate(zip(probs, ys, lams)):
        Lo = recon.power_lipschitz(p, oracle.adjoint(p, y), 20)
        ref = recon.fista(p, y, lam, 8, Lo, "db4", 2)  # the oracle's own L_f
        e = rel(xs[q].cpu().numpy(), ref)
        print(f"fp16x2 batch problem {q}: vs oracle {e:.2e}, L_f rel {abs(Ls[q] - Lo) / Lo:.2e}")
        assert abs(Ls[q] - Lo) < TOL * Lo
        assert e < TOL
