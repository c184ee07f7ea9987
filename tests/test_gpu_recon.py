"""Parity of the reconstruction (power iteration + FISTA on Eq. 1) with the FP64 oracle.

Bars: Lipschitz estimate relative error <= 1e-5; FISTA image relative L2 <= 1e-5
(FP32 form) after the workload's iteration count, both sides given the same L_f."""

import numpy as np
import pytest

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
    return ax


@pytest.fixture(scope="module")
def tiny(ax):
    import oracle
    from oracle import recon
    p, y, lam = simulated("tiny_64")
    v0 = oracle.adjoint(p, y)
    Lf = recon.power_lipschitz(p, v0, n_pow=30)
    return p, y, lam, Lf


def test_power_iteration_matches_oracle(ax, tiny):
    import torch
    p, y, lam, Lf = tiny
    prob = ax.Problem.from_arrays(p)
    x, L = ax.cs_recon(prob, torch.as_tensor(y, device="cuda"), lam, 0, wavelet="haar", levels=3, n_power=30)
    Lg = float(L.cpu().numpy()[0])
    print(f"L_f gpu {Lg:.9e} oracle {Lf:.9e} rel {abs(Lg - Lf) / Lf:.2e}")
    assert abs(Lg - Lf) <= TOL * Lf


@pytest.mark.parametrize("use_graph", [True, False])
def test_tiny64_fista_matches_oracle(ax, tiny, use_graph):
    """64^2, 8 coils, 2nd order + B0, Haar J=3, 20 iterations, lam = 1e-3 ||A^H y||_inf."""
    import torch
    from oracle import recon
    p, y, lam, Lf = tiny
    ref = recon.fista(p, y, lam, p["iters"], Lf, "haar", 3)
    prob = ax.Problem.from_arrays(p)
    side = torch.cuda.Stream()  # graph capture needs a non-default stream
    with torch.cuda.stream(side):
        x, L = ax.cs_recon(prob, torch.as_tensor(y, device="cuda"), lam, p["iters"], wavelet="haar", levels=3,
                           lipschitz=Lf, use_graph=use_graph)
        xg = x.cpu().numpy()
    e = rel(xg, ref)
    print(f"tiny64 fista rel {e:.2e}; nrmse vs phantom gpu {rel(xg, p['x_gt']):.4f} oracle {rel(ref, p['x_gt']):.4f}")
    assert e < TOL


def test_tiny64_graph_replay_is_identical(ax, tiny):
    import torch
    p, y, lam, Lf = tiny
    prob = ax.Problem.from_arrays(p)
    yg = torch.as_tensor(y, device="cuda")
    opts = ax.recon_opts(wavelet="haar", levels=3, lipschitz=Lf)
    ws = ax.recon_workspace(prob, opts)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        x1, _ = ax.cs_recon(prob, yg, lam, 5, opts=opts, ws=ws)      # captured
        a = x1.clone()
        x2, _ = ax.cs_recon(prob, yg, lam, 5, opts=opts, ws=ws, x_out=x1)  # replayed
        torch.cuda.synchronize()
        assert torch.equal(a, x2)
        assert ax.read_status(ws) == 0


def test_fista_with_start_image(ax, tiny):
    import torch
    from oracle import recon
    p, y, lam, Lf = tiny
    rng = np.random.default_rng(3)
    x0 = (0.1 * (rng.standard_normal(64 * 64) + 1j * rng.standard_normal(64 * 64))).astype(np.complex64)
    ref = recon.fista(p, y, lam, 4, Lf, "db4", 2, x0=x0)
    prob = ax.Problem.from_arrays(p)
    x, _ = ax.cs_recon(prob, torch.as_tensor(y, device="cuda"), lam, 4, wavelet="db4", levels=2, lipschitz=Lf,
                       x0=torch.as_tensor(x0, device="cuda"))
    assert rel(x.cpu().numpy(), ref) < TOL


@pytest.mark.slow
def test_slice200_two_iterations_match_oracle(ax):
    """Full 200^2 / 32-coil / 24k-sample / 3rd-order+B0 workload, db4 J=4, two FISTA
    iterations (4 oracle applications) with the same L_f on both sides."""
    import torch
    from oracle import recon
    p, y, lam = simulated("slice_200")
    prob = ax.Problem.from_arrays(p)
    yg = torch.as_tensor(y, device="cuda")
    _, L = ax.cs_recon(prob, yg, lam, 0, wavelet="db4", levels=4, n_power=30)
    Lf = float(L.cpu().numpy()[0])
    x, _ = ax.cs_recon(prob, yg, lam, 2, wavelet="db4", levels=4, lipschitz=Lf)
    ref = recon.fista(p, y, lam, 2, Lf, "db4", 4)
    e = rel(x.cpu().numpy(), ref)
    print(f"slice200 2-iteration fista rel {e:.2e}")
    assert e < TOL
