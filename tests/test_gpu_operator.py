"""Parity of A_exp / A_exp^H (FP32 CUDA cores) with the FP64 oracle.

Bar: relative L2 error <= 1e-5 (FP32 form), on the same seeded inputs.  The 32-coil cases run
in the default tiling and, through aexp_prepare_tiled, in tiling 1 (two samples / voxels per
thread), whose summation order differs but whose bar is the same."""

import numpy as np
import pytest

from paper_2211_07532_gb300 import synth
from tests._data import rel

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


def _run(ax, p, x, y, with_b0=True, tile_variant=0):
    import torch
    prob = ax.Problem.from_arrays(p, with_b0=with_b0)
    ws = ax.workspace(prob, tile_variant=tile_variant)
    ax.prepare(prob, ws, tile_variant=tile_variant)
    xg = torch.as_tensor(x, dtype=torch.complex64, device="cuda")
    yg = torch.as_tensor(y, dtype=torch.complex64, device="cuda")
    fwd = ax.a_exp_forward(prob, xg, ws)
    adj = ax.a_exp_adjoint(prob, yg, ws)
    torch.cuda.synchronize()
    assert ax.read_status(ws) == 0
    return fwd.cpu().numpy(), adj.cpu().numpy()


def _oracle_problem(p, with_b0):
    q = dict(p)
    if not with_b0:
        q["omega"] = None
    return q


SHAPES = [  # nx, ny, nt, nc, order, b0
    (13, 11, 777, 3, 3, True),      # partial tiles both ways, ragged nt
    (8, 8, 512, 8, 2, False),       # exactly one tile, exactly one sample block
    (1, 1, 1, 1, 0, False),         # degenerate: one voxel, one sample, one coil, one term
    (17, 9, 1025, 20, 3, True),     # 20 coils (paper's in-vivo count), 17 terms
    (24, 16, 300, 32, 1, True),     # 32 coils
    (5, 7, 64, 16, 2, True),
    (9, 9, 2000, 17, 3, False),     # 17 coils -> 20-wide padding
    (40, 3, 129, 5, 3, True),
]


@pytest.mark.parametrize("shape", SHAPES)
def test_ragged_shapes_match_oracle(ax, shape):
    import oracle
    nx, ny, nt, nc, order, b0 = shape
    p = synth.make_problem(nx, ny, nt=nt, nc=nc, order=order, dwell=4e-6, turns=max(nx, ny) / 8.0 + 1,
                           seed=1234 + nx * 7 + nt, with_b0=b0)
    rng = np.random.default_rng(nt)
    x = synth.random_image(rng, nx * ny)
    y = synth.random_kspace(rng, nc, nt)
    f, a = _run(ax, p, x, y, with_b0=b0)
    q = _oracle_problem(p, b0)
    assert rel(f, oracle.forward(q, x)) < TOL
    assert rel(a, oracle.adjoint(q, y)) < TOL


SHAPES_32 = [  # nx, ny, nt, nc, order, b0: coil counts padded to 32 (where tiling 1 applies)
    (24, 16, 300, 32, 1, True),
    (13, 11, 777, 29, 3, True),     # partial tiles both ways, ragged nt, 3 padded coils
    (1, 1, 1, 21, 0, False),        # degenerate: one voxel, one sample, one term
    (40, 3, 129, 32, 3, True),
    (19, 23, 2100, 32, 2, False),   # several sample stages and voxel blocks
]


@pytest.mark.parametrize("shape", SHAPES_32)
def test_alternative_tiling_matches_oracle(ax, shape):
    import oracle
    nx, ny, nt, nc, order, b0 = shape
    p = synth.make_problem(nx, ny, nt=nt, nc=nc, order=order, dwell=4e-6, turns=max(nx, ny) / 8.0 + 1,
                           seed=4321 + nx * 7 + nt, with_b0=b0)
    rng = np.random.default_rng(nt + 1)
    x = synth.random_image(rng, nx * ny)
    y = synth.random_kspace(rng, nc, nt)
    f, a = _run(ax, p, x, y, with_b0=b0, tile_variant=1)
    q = _oracle_problem(p, b0)
    ef, ea = rel(f, oracle.forward(q, x)), rel(a, oracle.adjoint(q, y))
    print(f"{shape} tiling 1: forward rel {ef:.2e} adjoint rel {ea:.2e}")
    assert ef < TOL and ea < TOL


def test_cartesian_case_matches_oracle(ax):
    import oracle
    p = synth.cartesian_problem(32)
    rng = np.random.default_rng(3)
    x = synth.random_image(rng, 32 * 32)
    y = synth.random_kspace(rng, 1, 32 * 32)
    q = dict(p)
    q["omega"] = None
    f, a = _run(ax, q, x, y, with_b0=False)
    assert rel(f, oracle.forward(q, x)) < TOL
    assert rel(a, oracle.adjoint(q, y)) < TOL


@pytest.mark.parametrize("kind", ["phantom", "white"])
def test_tiny64_matches_oracle(ax, kind):
    import oracle
    p = synth.tiny_64()
    rng = np.random.default_rng(11)
    x = p["x_gt"] if kind == "phantom" else synth.random_image(rng, 64 * 64)
    y = oracle.forward(p, p["x_gt"]).astype(np.complex64) if kind == "phantom" else synth.random_kspace(rng, 8, 2048)
    f, a = _run(ax, p, x, y)
    ef, ea = rel(f, oracle.forward(p, x)), rel(a, oracle.adjoint(p, y))
    print(f"tiny64 {kind}: forward rel {ef:.2e} adjoint rel {ea:.2e}")
    assert ef < TOL and ea < TOL


@pytest.fixture(scope="module", params=[0, 1], ids=["tiling0", "tiling1"])
def slice200(ax, request):
    """The 200^2 workload in the default tiling and in tiling 1."""
    import torch
    p = synth.slice_200()
    rng = np.random.default_rng(200)
    x_white = synth.random_image(rng, p["nx"] * p["ny"])
    y_white = synth.random_kspace(rng, p["nc"], p["nt"])
    prob = ax.Problem.from_arrays(p)
    ws = ax.workspace(prob, tile_variant=request.param)
    ax.prepare(prob, ws, tile_variant=request.param)
    out = {}
    for name, x in (("phantom", p["x_gt"]), ("white", x_white)):
        out["fwd_" + name] = ax.a_exp_forward(prob, torch.as_tensor(x, device="cuda"), ws).cpu().numpy()
    out["adj_white"] = ax.a_exp_adjoint(prob, torch.as_tensor(y_white, device="cuda"), ws).cpu().numpy()
    assert ax.read_status(ws) == 0
    return p, x_white, y_white, out, request.param


@pytest.mark.parametrize("kind", ["phantom", "white"])
def test_slice200_forward_sampled_rows(slice200, kind):
    """200^2, 32 coils, 24k samples, 3rd order + B0: 64 sample rows (incl. first and
    last) recomputed one by one by the oracle."""
    import oracle
    p, x_white, _, out, _ = slice200
    x = p["x_gt"] if kind == "phantom" else x_white
    rng = np.random.default_rng(5)
    ts = np.unique(np.concatenate([[0, 1, p["nt"] - 1], rng.choice(p["nt"], 61, replace=False)]))
    ref = oracle.forward_rows(p, x, ts)
    e = rel(out["fwd_" + kind][:, ts], ref)
    print(f"slice200 forward {kind}: sampled rel {e:.2e}")
    assert e < TOL


def test_slice200_adjoint_sampled_voxels(slice200):
    import oracle
    p, _, y_white, out, _ = slice200
    rng = np.random.default_rng(6)
    nr = p["nx"] * p["ny"]
    rs = np.unique(np.concatenate([[0, nr - 1, 199, 200 * 199], rng.choice(nr, 60, replace=False)]))
    ref = oracle.adjoint_rows(p, y_white, rs)
    e = rel(out["adj_white"][rs], ref)
    print(f"slice200 adjoint white: sampled rel {e:.2e}")
    assert e < TOL


def test_slice200_adjoint_identity(ax, slice200):
    """<A x, y> = <x, A^H y> holds at full size (computed in FP64 from the GPU outputs)."""
    p, x_white, y_white, out, _ = slice200
    Ax = out["fwd_white"].astype(np.complex128)
    AHy = out["adj_white"].astype(np.complex128)
    lhs = np.vdot(y_white.astype(np.complex128), Ax)
    rhs = np.vdot(AHy, x_white.astype(np.complex128))
    assert abs(lhs - rhs) <= TOL * np.linalg.norm(Ax) * np.linalg.norm(y_white)


def test_unprepared_workspace_is_rejected(ax):
    import torch
    p = synth.make_problem(8, nt=64, nc=2, order=1)
    prob = ax.Problem.from_arrays(p)
    ws = ax.workspace(prob)
    x = torch.zeros(64, dtype=torch.complex64, device="cuda")
    with pytest.raises(ax.AexpError, match="NOT_PREPARED"):
        ax.a_exp_forward(prob, x, ws)


def test_slice200_operator_is_repeatable(ax, slice200):
    """Partial sums are reduced in a fixed order: repeated applications agree bit for bit."""
    import torch
    p, variant = slice200[0], slice200[4]
    prob = ax.Problem.from_arrays(p)
    ws = ax.workspace(prob, tile_variant=variant)
    ax.prepare(prob, ws, tile_variant=variant)
    x = torch.as_tensor(p["x_gt"], device="cuda")
    y = torch.as_tensor(p["noise"], device="cuda")
    f0, a0 = ax.a_exp_forward(prob, x, ws).clone(), ax.a_exp_adjoint(prob, y, ws).clone()
    for _ in range(4):
        assert torch.equal(ax.a_exp_forward(prob, x, ws), f0)
        assert torch.equal(ax.a_exp_adjoint(prob, y, ws), a0)
