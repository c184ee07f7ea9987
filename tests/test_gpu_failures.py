"""Failure detection on the GPU without a fault: every device-side wait of the library is
bounded and every error is a status word the host reads.

* a bounded wait that runs out (an mbarrier phase that nothing completes, a short poll limit)
  reports AEXP_ERR_DEVICE_TIMEOUT, and the tensor-core kernels' abort-aware wait in the same
  block gives up with it; the context stays usable afterwards;
* non-finite data (a NaN planted in y on the host) reaches the power iteration, whose L_f
  check reports AEXP_ERR_NONFINITE instead of running FISTA on a meaningless step;
* a Jacobi coil compression capped at one sweep reports that it has not converged.
None of these waits more than a bounded number of polls, and none faults the GPU."""

import numpy as np
import pytest

from paper_2211_07532_gb300 import synth

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


def test_bounded_wait_gives_up_and_reports(ax):
    import torch
    status, gave_up = ax.probe_bounded_wait(2000)
    assert status == -6, ax.STATUS.get(status, status)      # AEXP_ERR_DEVICE_TIMEOUT
    assert gave_up == [1, 1]
    # the context is still usable: an operator application afterwards is clean
    p = synth.make_problem(16, 12, nt=300, nc=3, order=1, seed=5)
    prob = ax.Problem.from_arrays(p)
    ws = ax.workspace(prob)
    ax.prepare(prob, ws)
    y = ax.a_exp_forward(prob, torch.as_tensor(p["x_gt"], device="cuda"), ws)
    torch.cuda.synchronize()
    assert ax.read_status(ws) == 0 and bool(torch.isfinite(torch.view_as_real(y)).all())


def test_nonfinite_data_is_reported_by_the_power_iteration(ax):
    import torch
    p = synth.make_problem(24, 20, nt=500, nc=4, order=2, seed=6)
    prob = ax.Problem.from_arrays(p)
    y = np.asarray(p["noise"]).copy()
    y[1, 123] = np.nan + 0j
    opts = ax.recon_opts(n_power=10, levels=2, use_graph=False)
    ws = ax.recon_workspace(prob, opts)
    ax.cs_recon(prob, torch.as_tensor(y, device="cuda"), 0.1, 2, opts=opts, ws=ws)
    torch.cuda.synchronize()
    assert ax.read_status(ws) == -7      # AEXP_ERR_NONFINITE
    # a clean run on the same workspace afterwards reports nothing
    ax.cs_recon(prob, torch.as_tensor(p["noise"], device="cuda"), 0.1, 2, opts=opts, ws=ws)
    torch.cuda.synchronize()
    assert ax.read_status(ws) == 0


def test_jacobi_capped_at_one_sweep_reports_non_convergence(ax):
    import torch
    p = synth.make_problem(16, nt=400, nc=8, order=1, seed=8)
    prob = ax.Problem.from_arrays(p)
    y = torch.as_tensor(p["noise"], device="cuda")
    with pytest.raises(ax.AexpError, match="NONFINITE"):
        ax.coil_compress(prob, y, 4, max_sweeps=1)
    _, _, eig = ax.coil_compress(prob, y, 4)            # the default cap converges
    assert bool(torch.all(eig[:-1] >= eig[1:]))
