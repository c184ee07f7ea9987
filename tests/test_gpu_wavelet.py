"""Parity of the wavelet step (W, soft-threshold, W^H) with the FP64 oracle.

Bar: relative L2 <= 2e-6.  Derivation: each output is a J-level cascade of
2*taps-term FP32 dot products per level (rows and columns); with unit-norm
orthonormal filters the rounding error grows like eps * sqrt(2 * taps * J)
per coefficient, i.e. <= 6e-8 * sqrt(2*8*4) ~ 5e-7 for db4 at J = 4, with margin."""

import numpy as np
import pytest

from tests._data import rel

pytestmark = pytest.mark.gpu
TOL = 2e-6

# The prox step's levels 2..J run in one cluster of CTAs where its shared memory plan fits (the
# square cases), in one CTA for wide strips whose band scratch does not fit beside two copies of
# the level-1 approximation (db4 32 x 1600), and one launch per level beyond that (256 x 240).
CASES = [("haar", 64, 64, 3), ("db4", 200, 200, 4), ("db4", 13, 11, 2), ("haar", 11, 13, 1),
         ("db4", 170, 170, 4), ("haar", 1, 1, 1), ("db4", 16, 16, 4), ("db4", 32, 1600, 4),
         ("haar", 32, 1600, 4), ("db4", 256, 240, 3)]


@pytest.fixture(scope="module")
def ax():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_2211_07532_gb300 import build
    build.build()
    import paper_2211_07532_gb300 as ax
    return ax


def _img(ny, nx, seed):
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((ny, nx)) + 1j * rng.standard_normal((ny, nx))).astype(np.complex64)


@pytest.mark.parametrize("name,ny,nx,J", CASES)
def test_forward_transform_matches_oracle(ax, name, ny, nx, J):
    import torch
    from oracle import wavelet as wv
    img = _img(ny, nx, ny * 100 + nx)
    coef = ax.wavelet_forward(torch.as_tensor(img, device="cuda"), name, J).cpu().numpy()
    ref = wv.dwt2(wv.pad(img.astype(np.complex128), wv.padded_shape(ny, nx, J)), name, J)
    assert coef.shape == ref.shape
    assert rel(coef, ref) < TOL


@pytest.mark.parametrize("name,ny,nx,J", CASES)
def test_prox_matches_oracle(ax, name, ny, nx, J):
    import torch
    from oracle import wavelet as wv
    img = _img(ny, nx, ny * 7 + nx)
    shp = wv.padded_shape(ny, nx, J)
    w = wv.dwt2(wv.pad(img.astype(np.complex128), shp), name, J)
    tau = float(np.median(np.abs(w[wv.detail_mask(shp, J)])))  # about half the details shrink to 0
    out = ax.wavelet_prox(torch.as_tensor(img, device="cuda"), name, J, tau).cpu().numpy()
    ref = wv.prox(img.astype(np.complex128), ny, nx, name, J, np.float32(tau)).reshape(ny, nx)
    assert rel(out, ref) < TOL


def test_prox_zero_threshold_is_identity(ax):
    import torch
    img = _img(37, 29, 1)
    out = ax.wavelet_prox(torch.as_tensor(img, device="cuda"), "db4", 3, 0.0).cpu().numpy()
    assert rel(out, img) < TOL
