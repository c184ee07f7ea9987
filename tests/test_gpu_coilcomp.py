"""Coil compression on the GPU against the oracle (principal components of the data;
Sec. 2.2.1 / 2.2.2): eigenvalues, the compressed data and maps element by element (the
eigenvector phases are fixed by the same normalisation on both sides), and the compressed
problem's adjoint and reconstruction."""

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


@pytest.mark.parametrize("nc,nv", [(8, 8), (8, 4), (5, 3), (32, 16), (32, 20), (1, 1)])
def test_compression_matches_oracle(ax, nc, nv):
    import torch
    import oracle
    from oracle import coilcomp
    p = synth.make_problem(24, 20, nt=900, nc=nc, order=2, dwell=4e-6, turns=4.0, seed=300 + nc)
    rng = np.random.default_rng(nc)
    y = (oracle.forward(p, p["x_gt"]) + 0.05 * synth.random_kspace(rng, nc, 900)).astype(np.complex64)
    prob = ax.Problem.from_arrays(p)
    pv, yv, eig = ax.coil_compress(prob, torch.as_tensor(y, device="cuda"), nv)
    q, yv_o, e_o = coilcomp.compress(p, y, nv)
    ee = np.max(np.abs(eig.cpu().numpy() - e_o)) / e_o[0]
    ey = rel(yv.cpu().numpy(), yv_o)
    es = rel(pv.S.cpu().numpy(), q["S"])
    print(f"nc {nc} -> {nv}: eigenvalues {ee:.1e}, data rel {ey:.1e}, maps rel {es:.1e}")
    assert ee < 1e-12 and ey < 1e-6 and es < 1e-6


def test_compressed_reconstruction(ax):
    """32 -> 16 virtual coils on the 64^2 workload's shapes (8 coils -> 4 here) through cs_recon,
    against the oracle's FISTA on the oracle-compressed problem."""
    import torch
    import oracle
    from oracle import coilcomp, recon
    p, y, lam = simulated("tiny_64")
    prob = ax.Problem.from_arrays(p)
    pv, yv, _ = ax.coil_compress(prob, torch.as_tensor(y, device="cuda"), 4)
    q, yv_o, _ = coilcomp.compress(p, y, 4)
    Lf = recon.power_lipschitz(q, oracle.adjoint(q, yv_o), 30)
    x, _ = ax.cs_recon(pv, yv, lam, p["iters"], wavelet="haar", levels=3, lipschitz=Lf, use_graph=False)
    ref = recon.fista(q, yv_o, lam, p["iters"], Lf, "haar", 3)
    e = rel(x.cpu().numpy(), ref)
    print(f"compressed recon rel {e:.2e}; nrmse vs phantom {rel(x.cpu().numpy(), p['x_gt']):.4f} "
          f"(8 coils: oracle {rel(recon.fista(p, y, lam, p['iters'], Lf, 'haar', 3), p['x_gt']):.4f})")
    assert e < 1e-5
