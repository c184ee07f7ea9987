"""Ragged batches in one persistent launch per operator application (BF16 tensor cores).

Each problem of a small ragged batch (different image sizes, sample counts, field
coefficients) must reproduce (a) the single-problem reconstruction of the same problem and
(b) the FP64 oracle's FISTA iterate (its own power-iteration L_f), within 3x the image error
of the oracle's BF16 rounding emulation run the same way (power iteration and FISTA on the
emulated operator; ``oracle.precision``)."""

import numpy as np
import pytest

from paper_2211_07532_gb300 import synth
from tests._data import rel

pytestmark = pytest.mark.gpu
RECON_MARGIN = 3.0
TOL_OP = 5e-3

SHAPES = [(24, 24, 700), (17, 13, 333), (32, 32, 1200), (9, 21, 512), (40, 28, 901)]


@pytest.fixture(scope="module")
def ax():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2211_07532_gb300 import build
    build.build()
    import paper_2211_07532_gb300 as ax
    ax.lib()
    return ax


@pytest.fixture(scope="module")
def batch(ax):
    import oracle
    probs, ys, lams = [], [], []
    for i, (nx, ny, nt) in enumerate(SHAPES):
        p = synth.make_problem(nx, ny, nt=nt, nc=8, order=3, dwell=4e-6, turns=max(nx, ny) / 8.0 + 1,
                               seed=777 + i)
        y0 = oracle.forward(p, p["x_gt"])
        y = (y0 + 0.05 * np.sqrt(np.mean(np.abs(y0) ** 2)) * p["noise"]).astype(np.complex64)
        lam = float(np.float32(2e-2 * np.max(np.abs(oracle.adjoint(p, y)))))
        probs.append(p)
        ys.append(y)
        lams.append(lam)
    return probs, ys, lams


def test_batch_matches_single_problem_and_oracle(ax, batch):
    import torch
    import oracle
    from oracle import precision, recon
    probs, ys, lams = batch
    P = [ax.Problem.from_arrays(p) for p in probs]
    Y = [torch.as_tensor(y, device="cuda") for y in ys]
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        xs, L = ax.cs_recon_batched(P, Y, lams, 8, precision=ax.BF16_TC, wavelet="db4", levels=2, n_power=20)
        torch.cuda.synchronize()
        Ls = L.cpu().numpy()
        for q, (p, y, lam) in enumerate(zip(probs, ys, lams)):
            xs1, L1 = ax.cs_recon(P[q], Y[q], lam, 8, precision=ax.BF16_TC, wavelet="db4", levels=2, n_power=20)
            e_single = rel(xs[q].cpu().numpy(), xs1.cpu().numpy())
            assert abs(Ls[q] - float(L1.cpu().numpy()[0])) <= 1e-4 * Ls[q]
            Lo = recon.power_lipschitz(p, oracle.adjoint(p, y), 20)
            ref = recon.fista(p, y, lam, 8, Lo, "db4", 2)
            ops = precision.bf16_operators(p)
            Le = recon.power_lipschitz(p, ops[1](y), 20, ops=ops)
            emul = recon.fista(p, y, lam, 8, Le, "db4", 2, ops=ops)
            e_oracle, e_emul = rel(xs[q].cpu().numpy(), ref), rel(emul, ref)
            print(f"batch problem {q} {SHAPES[q]}: vs single {e_single:.2e}, vs oracle {e_oracle:.2e} "
                  f"(BF16 emulation {e_emul:.2e}), L_f {Ls[q]:.4e} (oracle {Lo:.4e})")
            assert e_single < 1e-4
            assert e_oracle < RECON_MARGIN * e_emul


def test_batch_lipschitz_matches_oracle(ax, batch):
    import torch
    import oracle
    from oracle import recon
    probs, ys, lams = batch
    P = [ax.Problem.from_arrays(p) for p in probs]
    Y = [torch.as_tensor(y, device="cuda") for y in ys]
    _, L = ax.cs_recon_batched(P, Y, lams, 0, precision=ax.BF16_TC, n_power=30)
    Ls = L.cpu().numpy()
    for q, (p, y) in enumerate(zip(probs, ys)):
        Lo = recon.power_lipschitz(p, oracle.adjoint(p, y), 30)
        assert abs(Ls[q] - Lo) <= TOL_OP * Lo


def test_batch_rejects_mixed_paddings(ax, batch):
    import torch
    probs, ys, lams = batch
    p2 = synth.make_problem(16, nt=256, nc=20, order=3, seed=5)   # 20 coils -> 32-wide padding
    P = [ax.Problem.from_arrays(probs[0]), ax.Problem.from_arrays(p2)]
    Y = [torch.as_tensor(ys[0], device="cuda"), torch.zeros((20, 256), dtype=torch.complex64, device="cuda")]
    with pytest.raises(ax.AexpError, match="UNSUPPORTED"):
        ax.cs_recon_batched(P, Y, [1.0, 1.0], 2, precision=ax.BF16_TC)


def test_batch_reconstruction_is_repeatable(ax, batch):
    """The ragged batch runs the persistent tensor-core kernels over all problems at once;
    three runs of the whole batched solve must agree bit for bit."""
    import torch
    probs, ys, lams = batch
    P = [ax.Problem.from_arrays(p) for p in probs]
    Y = [torch.as_tensor(y, device="cuda") for y in ys]
    runs = []
    for _ in range(3):
        xs, L = ax.cs_recon_batched(P, Y, lams, 8, precision=ax.BF16_TC, wavelet="db4", levels=2, n_power=20)
        torch.cuda.synchronize()
        runs.append(([x.clone() for x in xs], L.clone()))
    for xs, L in runs[1:]:
        assert torch.equal(L, runs[0][1])
        assert all(torch.equal(a, b) for a, b in zip(xs, runs[0][0]))
