"""The paper's own regulariser on the GPU (Sec. 2.1; Supporting Information S1): the one-level
undecimated wavelet, its prox step, the lambda = sigma / 2 rule and the FISTA reconstruction
with it, against the FP64 oracle.

The lambda rule picks histogram bins.  On the forward/prox and rule tests below the GPU's
FP32 magnitudes can fall on the other side of a bin edge from the oracle's FP64 ones, so there
lambda is held to one coarse bin (U / 64 / 2, ~4 % of lambda).  In the FP32 reconstruction the
GPU's decision must equal the oracle's (lambda to FP32 rounding) and the image is compared with
the oracle's own run; the BF16 reconstruction takes the oracle's lambda as a given value (its
rounding can move a coefficient across a bin edge) and is held to 3x the image error of the
oracle's BF16 rounding emulation (``oracle.precision``)."""

import numpy as np
import pytest

from paper_2211_07532_gb300 import synth
from tests._data import rel, simulated

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


@pytest.mark.parametrize("name", ["haar", "db4"])
@pytest.mark.parametrize("shape", [(13, 11), (64, 64), (200, 200)])
def test_swt_forward_and_prox(ax, name, shape):
    import torch
    from oracle import swt
    ny, nx = shape
    rng = np.random.default_rng(nx * ny)
    x = (rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))).astype(np.complex64)
    xd = torch.as_tensor(x, device="cuda")
    c = ax.swt_forward(xd, name).cpu().numpy()
    ref = swt.swt2(x, name)
    e = rel(c, ref)
    tau = 0.3
    p = ax.swt_prox(xd, tau, name).cpu().numpy()
    ep = rel(p, swt.prox(x, ny, nx, name, tau))
    print(f"swt {name} {shape}: coefficients rel {e:.2e}, prox rel {ep:.2e}")
    assert e < 1e-6 and ep < 1e-6


def test_swt_lambda_rule(ax):
    import torch
    import oracle
    from oracle import swt
    p, y, lam = simulated("tiny_64")
    z = oracle.adjoint(p, y).reshape(64, 64).astype(np.complex64)
    zd = torch.as_tensor(z, device="cuda")
    for name in ("haar", "db4"):
        lg = float(ax.swt_lambda(zd, name).cpu()[0])
        c = ax.swt_forward(zd, name).cpu().numpy()
        lo = 0.5 * swt.rayleigh_sigma(c[1:])               # the rule on the GPU's own coefficients
        lo64 = 0.5 * swt.rayleigh_sigma(swt.swt2(z, name)[1:])
        m = np.abs(c[1:]).reshape(-1)
        m = m[m > 0]
        bin_w = 0.5 * 4 * np.median(m) / 64                 # one coarse bin of lambda, roughly
        print(f"lambda {name}: gpu {lg:.6e}, rule on gpu coefficients {lo:.6e}, FP64 {lo64:.6e}")
        assert abs(lg - lo) <= 1.01 * bin_w and abs(lg - lo64) <= 2.01 * bin_w


def test_recon_with_the_paper_regulariser(ax):
    """FP32: lambda = sigma / 2 decided on the GPU equals the oracle's decision; the image
    matches the oracle's run at its own lambda."""
    import torch
    import oracle
    from oracle import recon, swt
    p, y, lam = simulated("tiny_64")
    yd = torch.as_tensor(y, device="cuda")
    prob = ax.Problem.from_arrays(p)
    Lf = recon.power_lipschitz(p, oracle.adjoint(p, y), 30)
    lam_out = torch.zeros(1, dtype=torch.float64, device="cuda")
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        x, _ = ax.cs_recon(prob, yd, 0.0, p["iters"], precision=ax.FP32, wavelet="db4", undecimated=True,
                           lambda_rule=ax.LAMBDA_RAYLEIGH, lambda_out=lam_out, lipschitz=Lf)
        torch.cuda.synchronize()
    lg = float(lam_out.cpu()[0])
    lo = swt.rayleigh_lambda(p, y, "db4")
    ref = swt.fista(p, y, lo, p["iters"], Lf, "db4")
    e = rel(x.cpu().numpy(), ref)
    print(f"FP32 undecimated db4: lambda gpu {lg:.7e} oracle {lo:.7e}; image rel {e:.2e}; "
          f"nrmse vs phantom {rel(x.cpu().numpy(), p['x_gt']):.4f} (oracle {rel(ref, p['x_gt']):.4f})")
    assert abs(lg - lo) <= 1e-5 * lo
    assert e < 1e-5


def test_bf16_recon_with_the_paper_regulariser(ax):
    """BF16 tensor cores, undecimated db4, the oracle's lambda = sigma / 2 given."""
    import torch
    import oracle
    from oracle import precision, recon, swt
    p, y, lam = simulated("tiny_64")
    prob = ax.Problem.from_arrays(p)
    Lf = recon.power_lipschitz(p, oracle.adjoint(p, y), 30)
    lo = swt.rayleigh_lambda(p, y, "db4")
    x, _ = ax.cs_recon(prob, torch.as_tensor(y, device="cuda"), lo, p["iters"], precision=ax.BF16_TC,
                       wavelet="db4", undecimated=True, lipschitz=Lf)
    ref = swt.fista(p, y, lo, p["iters"], Lf, "db4")
    emul = swt.fista(p, y, lo, p["iters"], Lf, "db4", ops=precision.bf16_operators(p))
    e, ee = rel(x.cpu().numpy(), ref), rel(emul, ref)
    print(f"BF16 undecimated db4: image rel {e:.2e} (BF16 emulation {ee:.2e})")
    assert e < 3.0 * ee


def test_given_lambda_matches_oracle(ax):
    import torch
    import oracle
    from oracle import recon, swt
    p, y, lam = simulated("tiny_64")
    prob = ax.Problem.from_arrays(p)
    Lf = recon.power_lipschitz(p, oracle.adjoint(p, y), 30)
    x, _ = ax.cs_recon(prob, torch.as_tensor(y, device="cuda"), lam, 15, wavelet="haar", undecimated=True,
                       lipschitz=Lf, use_graph=False)
    e = rel(x.cpu().numpy(), swt.fista(p, y, lam, 15, Lf, "haar"))
    print(f"given lambda, haar: rel {e:.2e}")
    assert e < 1e-5


def test_rule_without_undecimated_is_refused(ax):
    import torch
    p, y, lam = simulated("tiny_64")
    prob = ax.Problem.from_arrays(p)
    with pytest.raises(ax.AexpError, match="UNSUPPORTED"):
        ax.cs_recon(prob, torch.as_tensor(y, device="cuda"), 0.0, 2, lambda_rule=ax.LAMBDA_RAYLEIGH)
