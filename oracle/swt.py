"""The paper's own regulariser: undecimated 2-D wavelet, one level, lambda = sigma / 2 (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 2.1 regularises with the undecimated wavelet transform W at one level and sets the
weighting from W A^H y (the zero-filled reconstruction); Supporting Information S1 (Method 2)
takes the magnitudes of the high-pass coefficients of the level as Rayleigh distributed, reads
sigma off the maximum of their histogram, and uses lambda = sigma / 2 (low-pass weight 0).

Readings fixed here:
* W: the 1-level stationary transform with the orthonormal filters of ``oracle.wavelet``
  (Haar or Daubechies-4), periodic, no downsampling, separable (rows x, then columns y),
  every filter scaled by 1/sqrt(2) per dimension so that W^H W = I (a tight frame):
      c_s[y, x] = 1/2 sum_{my, mx} f_{s,y}[my] f_{s,x}[mx] v[(y + my) mod ny, (x + mx) mod nx]
  for the four subbands s = fx + 2 fy (f = h for 0, g for 1): 0 LL, 1 HL, 2 LH, 3 HH;
* prox step of "balanced FISTA" (Sec. 2.1) with the tight frame: x = W^H soft_detail(W v, tau),
  tau = lambda / L_f, detail subbands s = 1, 2, 3 only;
* histogram: the magnitudes m = |c_s| of all detail coefficients of the level, exact zeros
  discarded; m_max = max m; a 4096-bin histogram over [0, m_max] gives the median bin
  (smallest bin whose cumulative count reaches ceil(n / 2)), med = its centre; then a 64-bin
  histogram over [0, 4 med) (for a Rayleigh law the median is 1.18 sigma, so the range covers
  the noise peak and cuts the signal tail); sigma = the centre of its fullest bin (lowest on a
  tie); lambda = sigma / 2.  Bin of m in n_b bins over [0, u): floor(m * (n_b / u)), with
  m = u falling in the last bin of the fine histogram.
"""

from __future__ import annotations

import math

import numpy as np

from . import wavelet as wv

FINE_BINS = 4096
COARSE_BINS = 64


def _filter_axis(a: np.ndarray, taps: np.ndarray, axis: int) -> np.ndarray:
    """out[j] = (1/sqrt 2) sum_m taps[m] a[(j + m) mod n] along `axis`."""
    out = np.zeros_like(a, dtype=np.complex128)
    for m, c in enumerate(taps):
        out += c * np.roll(a, -m, axis=axis)
    return out / math.sqrt(2.0)


def _filter_axis_adjoint(c: np.ndarray, taps: np.ndarray, axis: int) -> np.ndarray:
    """Transpose of ``_filter_axis``: out[(j + m) mod n] += (1/sqrt 2) taps[m] c[j]."""
    out = np.zeros_like(c, dtype=np.complex128)
    for m, t in enumerate(taps):
        out += t * np.roll(c, m, axis=axis)
    return out / math.sqrt(2.0)


def swt2(img: np.ndarray, name: str) -> np.ndarray:
    """One-level undecimated 2-D transform: [4][ny][nx], subband s = fx + 2 fy."""
    h, g = wv.filters(name)
    a = np.asarray(img, np.complex128)
    rows = [_filter_axis(a, h, 1), _filter_axis(a, g, 1)]          # fx = 0, 1
    out = np.empty((4,) + a.shape, np.complex128)
    for fy, ty in enumerate((h, g)):
        for fx in range(2):
            out[fx + 2 * fy] = _filter_axis(rows[fx], ty, 0)
    return out


def iswt2(c: np.ndarray, name: str) -> np.ndarray:
    """W^H: the adjoint of ``swt2`` (its left inverse, W^H W = I)."""
    h, g = wv.filters(name)
    c = np.asarray(c, np.complex128)
    rows = [np.zeros(c.shape[1:], np.complex128) for _ in range(2)]
    for fy, ty in enumerate((h, g)):
        for fx in range(2):
            rows[fx] += _filter_axis_adjoint(c[fx + 2 * fy], ty, 0)
    return _filter_axis_adjoint(rows[0], h, 1) + _filter_axis_adjoint(rows[1], g, 1)


def prox(v: np.ndarray, ny: int, nx: int, name: str, tau: float) -> np.ndarray:
    """W^H soft_detail(W v, tau) on an ny x nx image (flattened or 2-D)."""
    c = swt2(np.asarray(v, np.complex128).reshape(ny, nx), name)
    c[1:] = wv.soft(c[1:], tau)
    return iswt2(c, name).reshape(-1)


def rayleigh_sigma(detail: np.ndarray) -> float:
    """sigma of the Rayleigh law of |detail| from the maximum of its histogram (see header)."""
    m = np.abs(np.asarray(detail)).reshape(-1)
    m = m[m > 0]
    if m.size == 0:
        return 0.0
    m_max = float(m.max())
    fine = np.minimum(np.floor(m * (FINE_BINS / m_max)).astype(np.int64), FINE_BINS - 1)
    cum = np.cumsum(np.bincount(fine, minlength=FINE_BINS))
    b_med = int(np.searchsorted(cum, (m.size + 1) // 2))
    med = (b_med + 0.5) * m_max / FINE_BINS
    u = 4.0 * med
    inside = m < u
    coarse = np.floor(m[inside] * (COARSE_BINS / u)).astype(np.int64)
    counts = np.bincount(np.minimum(coarse, COARSE_BINS - 1), minlength=COARSE_BINS)
    return (int(np.argmax(counts)) + 0.5) * u / COARSE_BINS


def rayleigh_lambda(prob, y, name: str) -> float:
    """lambda = sigma / 2 with sigma from the detail subbands of W A^H y (Supporting Information S1)."""
    from . import adjoint
    z = adjoint(prob, y).reshape(prob["ny"], prob["nx"])
    return 0.5 * rayleigh_sigma(swt2(z, name)[1:])


def fista(prob, y, lam, iters, lipschitz, name, x0=None, ops=None):
    """FISTA with the balanced tight-frame step: x_k = W^H soft(W v_k, lam / L_f).
    ``ops``: optional (A, A^H) callables in place of the exact double sums."""
    from . import adjoint, forward
    fwd, adj = ops if ops is not None else ((lambda v: forward(prob, v)), (lambda r: adjoint(prob, r)))
    ny, nx = prob["ny"], prob["nx"]
    y = np.asarray(y, np.complex128)
    x_prev = np.zeros(nx * ny, np.complex128) if x0 is None else np.asarray(x0, np.complex128).reshape(-1)
    z = x_prev.copy()
    t = 1.0
    tau = lam / lipschitz
    for _ in range(iters):
        v = z - 2.0 * adj(fwd(z) - y) / lipschitz
        x = prox(v, ny, nx, name, tau)
        t_next = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        z = x + ((t - 1.0) / t_next) * (x - x_prev)
        x_prev = x
        t = t_next
    return x_prev
