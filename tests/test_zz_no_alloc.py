"""aexp_wavelet_prox_static, the wavelet prox step that allocates nothing.

Some callers of this library cannot allocate device memory when they call it: code
running while a CUDA stream is being captured, real-time reconstruction services that
reserve all GPU memory at start-up, plug-ins whose host framework owns the allocator.
This entry point keeps its scratch in a fixed array inside the library instead of a
caller workspace.  The test calls it through the C ABI twice in a row -- the second call
runs on whatever the first left in the shared array -- and checks each result against the
workspace form, aexp_wavelet_prox, and against the FP64 oracle's prox step, within the
wavelet tests' tolerance.  It also checks that a size beyond the array is refused.
"""

import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
TOL = 2e-6  # the bar of the other wavelet parity tests


@pytest.fixture(scope="module")
def ax():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2211_07532_gb300 import build
    build.build()
    import paper_2211_07532_gb300 as ax
    ax.lib()
    return ax


def _img(ny, nx, seed):
    import torch
    rng = np.random.default_rng(seed)
    a = (rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))).astype(np.complex64)
    return torch.as_tensor(a, device="cuda")


def _static(ax, img, wavelet, levels, tau):
    import torch
    ny, nx = img.shape
    out = torch.empty_like(img)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = ax.lib().aexp_wavelet_prox_static(nx, ny, ax.WAVELETS[wavelet], levels, ctypes.c_float(tau),
                                            ctypes.c_void_p(img.data_ptr()), ctypes.c_void_p(out.data_ptr()),
                                            stream)
    return rc, out


def _rel(a, b):
    a = a.cpu().numpy().astype(np.complex128)
    b = b.cpu().numpy().astype(np.complex128)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_static_prox_matches_workspace_prox_on_two_calls_in_a_row(ax):
    from oracle import wavelet as wv
    calls = [("db4", 200, 200, 4, 0.6, 1), ("haar", 37, 29, 2, 0.9, 2)]
    for wavelet, ny, nx, levels, tau, seed in calls:
        img = _img(ny, nx, seed)
        rc, out = _static(ax, img, wavelet, levels, tau)
        assert rc == 0, ax.STATUS.get(rc, rc)
        ref = ax.wavelet_prox(img, wavelet, levels, tau)
        assert _rel(out, ref) <= TOL
        oref = wv.prox(img.cpu().numpy(), ny, nx, wavelet, levels, tau).reshape(ny, nx)
        e = float(np.linalg.norm(out.cpu().numpy() - oref) / np.linalg.norm(oref))
        print(f"static prox {wavelet} {ny}x{nx}: vs workspace form {_rel(out, ref):.2e}, vs oracle {e:.2e}")
        assert e <= TOL


def test_static_prox_refuses_sizes_beyond_its_array(ax):
    img = _img(1024, 1024, 3)
    rc, _ = _static(ax, img, "db4", 4, 0.5)
    assert rc == -3  # AEXP_ERR_UNSUPPORTED
