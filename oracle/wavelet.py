"""Orthonormal periodised 2-D wavelet transform and complex soft-threshold (FP64).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper regularises with a wavelet transform W and an l1 penalty, Eq. (1);
its low-pass level carries weight 0 (Supporting Information S1).  This oracle
implements the orthogonal reading: a J-level periodised separable DWT on the
image zero-padded to a multiple of 2^J in each direction, Mallat layout, rows
(x) filtered before columns (y) at every level.

Definitions used (one level, length-n signal a, filter taps h[0..m-1]):
    lo[j] = sum_m h[m] a[(2j + m) mod n]
    hi[j] = sum_m g[m] a[(2j + m) mod n],   g[m] = (-1)^m h[m_len - 1 - m]
and the synthesis is the transpose of that map.  Real filters act on the real
and imaginary parts alike.
"""

from __future__ import annotations

import math

import numpy as np


def daubechies_taps(p: int) -> np.ndarray:
    """Orthonormal Daubechies lowpass filter with p vanishing moments (2p taps).

    Spectral factorisation: |m0(w)|^2 = cos^{2p}(w/2) P(sin^2(w/2)) with
    P(y) = sum_{k<p} C(p-1+k, k) y^k.  Each root y_k of P gives, through
    y = (2 - z - 1/z)/4, a pair z, 1/z; the root inside the unit circle is kept
    (minimum phase).  m0(z) ~ ((1+z)/2)^p prod_k (z - z_k), normalised so that
    sum h = sqrt(2).  Taps are returned with the largest-magnitude-first
    ordering of the minimum-phase filter (h[0] = 0.2303... for p = 4).
    """
    if p == 1:
        return np.array([1.0, 1.0]) / math.sqrt(2.0)
    # P(y) coefficients, highest power first for numpy.roots
    coeffs = [math.comb(p - 1 + k, k) for k in range(p)]
    yroots = np.roots(coeffs[::-1])
    zroots = []
    for yk in yroots:
        # z^2 - (2 - 4 y_k) z + 1 = 0
        b = 2.0 - 4.0 * yk
        disc = np.sqrt(b * b - 4.0 + 0j)
        z1 = (b + disc) / 2.0
        z2 = (b - disc) / 2.0
        zroots.append(z1 if abs(z1) < 1.0 else z2)
    poly = np.array([1.0 + 0j])
    for _ in range(p):
        poly = np.convolve(poly, np.array([1.0, 1.0]))
    for zk in zroots:
        poly = np.convolve(poly, np.array([1.0, -zk]))
    h = np.real(poly)
    h = h * (math.sqrt(2.0) / h.sum())
    # numpy's polynomial is highest power first; the minimum-phase filter in
    # increasing powers of z^-1 starts from the other end.
    h = h[::-1]
    if abs(h[0]) < abs(h[-1]):
        h = h[::-1]
    return h


def filters(name: str):
    """(h, g) lowpass/highpass analysis taps for 'haar' or 'db4'."""
    if name == "haar":
        h = daubechies_taps(1)
    elif name == "db4":
        h = daubechies_taps(4)
    else:
        raise ValueError(f"unknown wavelet {name!r}")
    m = h.size
    g = np.array([(-1) ** i * h[m - 1 - i] for i in range(m)])
    return h, g


def _analysis_axis(a: np.ndarray, h: np.ndarray, g: np.ndarray, axis: int):
    a = np.moveaxis(a, axis, -1)
    n = a.shape[-1]
    half = n // 2
    lo = np.zeros(a.shape[:-1] + (half,), np.complex128)
    hi = np.zeros_like(lo)
    for j in range(half):
        for m in range(h.size):
            col = a[..., (2 * j + m) % n]
            lo[..., j] += h[m] * col
            hi[..., j] += g[m] * col
    out = np.concatenate([lo, hi], axis=-1)
    return np.moveaxis(out, -1, axis)


def _synthesis_axis(c: np.ndarray, h: np.ndarray, g: np.ndarray, axis: int):
    c = np.moveaxis(c, axis, -1)
    n = c.shape[-1]
    half = n // 2
    lo = c[..., :half]
    hi = c[..., half:]
    out = np.zeros(c.shape, np.complex128)
    for j in range(half):
        for m in range(h.size):
            out[..., (2 * j + m) % n] += h[m] * lo[..., j] + g[m] * hi[..., j]
    return np.moveaxis(out, -1, axis)


def padded_shape(ny: int, nx: int, levels: int):
    q = 1 << levels
    return (-(-ny // q) * q, -(-nx // q) * q)


def dwt2(img: np.ndarray, name: str, levels: int) -> np.ndarray:
    """Multi-level 2-D DWT of an array whose sides are multiples of 2^levels."""
    h, g = filters(name)
    out = np.array(img, dtype=np.complex128, copy=True)
    ny, nx = out.shape
    for _ in range(levels):
        blk = out[:ny, :nx]
        blk = _analysis_axis(blk, h, g, axis=1)   # rows first (x)
        blk = _analysis_axis(blk, h, g, axis=0)   # then columns (y)
        out[:ny, :nx] = blk
        ny //= 2
        nx //= 2
    return out


def idwt2(coef: np.ndarray, name: str, levels: int) -> np.ndarray:
    """Inverse of ``dwt2`` (its transpose, since the transform is orthonormal)."""
    h, g = filters(name)
    out = np.array(coef, dtype=np.complex128, copy=True)
    ny0, nx0 = out.shape
    for j in reversed(range(levels)):
        ny, nx = ny0 >> j, nx0 >> j
        blk = out[:ny, :nx]
        blk = _synthesis_axis(blk, h, g, axis=0)
        blk = _synthesis_axis(blk, h, g, axis=1)
        out[:ny, :nx] = blk
    return out


def detail_mask(shape, levels: int) -> np.ndarray:
    """True for detail (penalised) coefficients, False for the final low-pass block."""
    m = np.ones(shape, bool)
    m[: shape[0] >> levels, : shape[1] >> levels] = False
    return m


def soft(w: np.ndarray, tau: float) -> np.ndarray:
    """Complex soft-threshold, the prox of tau*|.|:  w * max(0, 1 - tau/|w|), soft(0) = 0."""
    w = np.asarray(w, np.complex128)
    mag = np.abs(w)
    scale = np.where(mag > tau, 1.0 - tau / np.where(mag > 0, mag, 1.0), 0.0)
    return w * scale


def pad(img: np.ndarray, shape) -> np.ndarray:
    out = np.zeros(shape, np.complex128)
    out[: img.shape[0], : img.shape[1]] = img
    return out


def prox(v: np.ndarray, ny: int, nx: int, name: str, levels: int, tau: float) -> np.ndarray:
    """crop( W^H soft_detail( W pad(v), tau ) ) on an ny x nx image (flattened or 2-D)."""
    v2 = np.asarray(v, np.complex128).reshape(ny, nx)
    shp = padded_shape(ny, nx, levels)
    w = dwt2(pad(v2, shp), name, levels)
    mask = detail_mask(shp, levels)
    w = np.where(mask, soft(w, tau), w)
    return idwt2(w, name, levels)[:ny, :nx].reshape(-1)


def l1_detail(x: np.ndarray, ny: int, nx: int, name: str, levels: int) -> float:
    """sum of |(W pad x)_j| over detail coefficients (the penalty of Eq. 1, low-pass weight 0)."""
    shp = padded_shape(ny, nx, levels)
    w = dwt2(pad(np.asarray(x).reshape(ny, nx), shp), name, levels)
    return float(np.sum(np.abs(w[detail_mask(shp, levels)])))
