"""The work-item autotuner: it returns one of its candidates, and reconstructions laid out
with the chosen granularity still match the FP64 oracle (the granularity changes only the
split of the sample and voxel reductions, i.e. the FP32 summation order)."""

import numpy as np
import pytest

from paper_2211_07532_gb300 import synth
from tests._data import rel, simulated

pytestmark = pytest.mark.gpu
CANDIDATES = {2, 4, 8, 16, 32}


@pytest.fixture(scope="module")
def ax():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2211_07532_gb300 import build
    build.build()
    import paper_2211_07532_gb300 as ax
    ax.lib()
    return ax


@pytest.mark.parametrize("precision", ["FP32", "FP16X2_TC"])
def test_autotune_single_problem(ax, precision):
    import torch
    from oracle import recon
    import oracle
    prec = getattr(ax, precision)
    p, y, lam = simulated("tiny_64")
    prob = ax.Problem.from_arrays(p)
    opts = ax.recon_opts(precision=prec, wavelet="haar", levels=3)
    best, variant, ms = ax.autotune(prob, opts)
    print(f"{precision}: items_per_sm {best}, tiling {variant}, {ms:.3f} ms per A^H A")
    assert best in CANDIDATES and variant in (0, 1) and ms > 0
    assert ax.autotune(prob, opts)[:2] == (best, variant)  # remembered for the shape
    Lf = recon.power_lipschitz(p, oracle.adjoint(p, y), 30)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        x, _ = ax.cs_recon(prob, torch.as_tensor(y, device="cuda"), lam, p["iters"], precision=prec,
                           wavelet="haar", levels=3, lipschitz=Lf, items_per_sm=best, tile_variant=variant)
        torch.cuda.synchronize()
    ref = recon.fista(p, y, lam, p["iters"], Lf, "haar", 3)
    assert rel(x.cpu().numpy(), ref) < 1e-5


def test_autotune_batch(ax):
    import torch
    import oracle
    from oracle import recon
    shapes = [(24, 24, 700), (17, 13, 333), (32, 32, 1200), (40, 28, 901)]
    probs, ys, lams = [], [], []
    for i, (nx, ny, nt) in enumerate(shapes):
        p = synth.make_problem(nx, ny, nt=nt, nc=8, order=3, dwell=4e-6, turns=max(nx, ny) / 8.0 + 1, seed=900 + i)
        y0 = oracle.forward(p, p["x_gt"])
        ys.append((y0 + 0.05 * np.sqrt(np.mean(np.abs(y0) ** 2)) * p["noise"]).astype(np.complex64))
        lams.append(float(np.float32(2e-2 * np.max(np.abs(oracle.adjoint(p, ys[-1]))))))
        probs.append(p)
    P = [ax.Problem.from_arrays(p) for p in probs]
    Y = [torch.as_tensor(y, device="cuda") for y in ys]
    opts = ax.recon_opts(precision=ax.FP16X2_TC, wavelet="db4", levels=2, n_power=20)
    best, variant, ms = ax.autotune(P, opts)
    print(f"batch: items_per_sm {best}, tiling {variant}, {ms:.3f} ms per A^H A of the batch")
    assert best in CANDIDATES and variant == 0   # the FP16 hi+lo form has one tiling
    opts.items_per_sm = best
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        xs, L = ax.cs_recon_batched(P, Y, lams, 6, opts=opts)
        torch.cuda.synchronize()
    for q, (p, y, lam) in enumerate(zip(probs, ys, lams)):
        Lo = recon.power_lipschitz(p, oracle.adjoint(p, y), 20)   # the oracle's own L_f
        ref = recon.fista(p, y, lam, 6, Lo, "db4", 2)
        assert rel(xs[q].cpu().numpy(), ref) < 1e-5


def test_autotune_refuses_capture(ax):
    import torch
    p, y, lam = simulated("tiny_64")
    prob = ax.Problem.from_arrays(p)
    opts = ax.recon_opts(precision=ax.FP32)
    side = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    ws = torch.empty(1 << 26, dtype=torch.uint8, device="cuda")
    with torch.cuda.stream(side):
        with pytest.raises(ax.AexpError, match="INVALID_ARG"):
            with torch.cuda.graph(g, stream=side):
                ax.autotune(prob, opts, ws=ws)


@pytest.mark.parametrize("precision", ["FP32", "BF16_TC", "FP16X2_TC"])
def test_tiling_variant_matches_oracle(ax, precision):
    """The alternative tiling (FP32 at 32 coils: two samples / voxels per thread; BF16: deeper
    rings; FP16 hi+lo: phases on the CUDA cores) computes the same reconstruction: FP32 and FP16
    hi+lo within the FP32 bar, BF16 within 3x the oracle's BF16 rounding emulation, as the
    default tiling."""
    import torch
    import oracle
    from oracle import precision as prec_emul
    from oracle import recon
    p = synth.make_problem(32, 24, nt=1000, nc=32, order=3, dwell=4e-6, turns=5.0, seed=4242)
    y0 = oracle.forward(p, p["x_gt"])
    y = (y0 + 0.05 * np.sqrt(np.mean(np.abs(y0) ** 2)) * p["noise"]).astype(np.complex64)
    lam = float(np.float32(1e-2 * np.max(np.abs(oracle.adjoint(p, y)))))
    Lf = recon.power_lipschitz(p, oracle.adjoint(p, y), 20)
    prob = ax.Problem.from_arrays(p)
    prec = getattr(ax, precision)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        x, _ = ax.cs_recon(prob, torch.as_tensor(y, device="cuda"), lam, 10, precision=prec, wavelet="db4",
                           levels=2, lipschitz=Lf, tile_variant=1)
        torch.cuda.synchronize()
    ref = recon.fista(p, y, lam, 10, Lf, "db4", 2)
    e = rel(x.cpu().numpy(), ref)
    if precision in ("FP32", "FP16X2_TC"):
        bar = 1e-5
    else:
        bar = 3.0 * rel(recon.fista(p, y, lam, 10, Lf, "db4", 2, ops=prec_emul.bf16_operators(p)), ref)
    print(f"{precision} tiling 1: image rel {e:.2e} (bar {bar:.2e})")
    assert e < bar
