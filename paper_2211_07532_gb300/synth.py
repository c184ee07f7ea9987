"""Seeded synthetic inputs for the expanded-encoding reconstruction.

This module only *draws inputs*: the phantom, receive-coil maps, the spiral
trajectory with its eddy-perturbed spherical-harmonic field coefficients
k_l(t), the basis values h_l(r) at the voxel positions, the B0 map, the sample
times and unit-variance complex noise.  It holds none of the method's
arithmetic (no phase, no encoding operator, no wavelet, no solver), so that
both the FP64 oracle and the CUDA path can read the very same arrays.

Every array is rounded once to its storage type (float32 / complex64); both
sides then read identical values, so input quantisation is never counted as
disagreement between them.

Stand-ins for the paper's data (the in-vivo GRE image, ESPIRiT maps, measured
B0 map and monitored field coefficients, Sec. 2.2 and Fig. S3, are not
available):

* image   -- 10 random complex ellipses inside a 0.8*FOV disc;
* coils   -- Gaussian bumps on a ring with a smooth phase ramp, normalised to
             sum_c |S_c(r)|^2 = 1 (the ESPIRiT normalisation, Sec. 2.2.1);
* field   -- nominal spiral k_x, k_y plus exponential eddy decays
             (tau 0.5-5 ms, amplitude 1-5 %) in every spherical-harmonic term
             up to 2nd, 3rd or 4th order (Sec. 1: field dynamics to 2nd/3rd order;
             higher orders and second-order concomitant-field rows, Fig. S3d, as
             extra terms of the same operator);
* B0      -- a smooth sum of Gaussians rescaled to a stated +-Hz range;
* spiral  -- variable-density Archimedean (64^2 case) or uniform single-shot
             with acceleration R (N/(2R) turns).

Geometry: voxel r = iy*nx + ix sits at (u, v cos(tilt), v sin(tilt) + z0) with
u = (ix - nx/2)*dx, v = (iy - ny/2)*dy: an axial slice at z0, or an oblique one
rotated by ``tilt`` about the x axis.
Units: k_l in rad/m^deg(l), h_l in m^deg(l), omega in rad/s, t in s.
"""

from __future__ import annotations

import math

import numpy as np

BASE_SEED = 2211075320

GAMMA = 2.675221874e8  # proton gyromagnetic ratio, rad / s / T


# Number of real solid harmonics up to a given order: 1, 4, 9, 16, 25.
def n_terms(order: int) -> int:
    return (order + 1) ** 2


def term_degree(l: int) -> int:
    """Polynomial degree of the l-th basis term (0 | 1,2,3 | 4..8 | 9..15 | 16..24)."""
    return int(math.isqrt(l))


def sh_basis(x: np.ndarray, y: np.ndarray, z: np.ndarray, order: int) -> np.ndarray:
    """Unnormalised real solid harmonics up to ``order`` (<= 4), by degree, m = -l..l.

    Ordering: 1; x, y, z; xy, yz, 2z^2-x^2-y^2, xz, x^2-y^2;
    3x^2y-y^3, xyz, y(4z^2-x^2-y^2), z(2z^2-3x^2-3y^2), x(4z^2-x^2-y^2),
    z(x^2-y^2), x^3-3xy^2;
    xy(x^2-y^2), yz(3x^2-y^2), xy(7z^2-r^2), yz(7z^2-3r^2), 35z^4-30z^2r^2+3r^4,
    xz(7z^2-3r^2), (x^2-y^2)(7z^2-r^2), xz(x^2-3y^2), x^4-6x^2y^2+y^4.
    The paper fits field dynamics to spherical
    harmonics up to 2nd or 3rd order (Sec. 1, Sec. 2.2.1) without fixing a
    normalisation; since h_l(r) is an input array to the operator, this choice
    only shapes the synthetic data.
    """
    if order < 0 or order > 4:
        raise ValueError("order must be 0..4")
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    z = np.asarray(z, np.float64) + np.zeros_like(x)
    r2 = x * x + y * y + z * z
    terms = [np.ones_like(x)]
    if order >= 1:
        terms += [x, y, z]
    if order >= 2:
        terms += [x * y, y * z, 3 * z * z - r2, x * z, x * x - y * y]
    if order >= 3:
        terms += [
            3 * x * x * y - y ** 3,
            x * y * z,
            y * (5 * z * z - r2),
            z * (5 * z * z - 3 * r2),
            x * (5 * z * z - r2),
            z * (x * x - y * y),
            x ** 3 - 3 * x * y * y,
        ]
    if order >= 4:
        z2 = z * z
        terms += [
            x * y * (x * x - y * y),
            y * z * (3 * x * x - y * y),
            x * y * (7 * z2 - r2),
            y * z * (7 * z2 - 3 * r2),
            35 * z2 * z2 - 30 * z2 * r2 + 3 * r2 * r2,
            x * z * (7 * z2 - 3 * r2),
            (x * x - y * y) * (7 * z2 - r2),
            x * z * (x * x - 3 * y * y),
            x ** 4 - 6 * x * x * y * y + y ** 4,
        ]
    return np.stack(terms, axis=0)


def concomitant_basis(x: np.ndarray, y: np.ndarray, z: np.ndarray) -> np.ndarray:
    """Spatial rows of the second-order concomitant (Maxwell) field: z^2, x^2 + y^2, xz, yz."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    z = np.asarray(z, np.float64) + np.zeros_like(x)
    return np.stack([z * z, x * x + y * y, x * z, y * z], axis=0)


def concomitant_coefficients(G: np.ndarray, dt: float, b0_tesla: float) -> np.ndarray:
    """Phase coefficients [4][nt] (rad / m^2) of the concomitant rows for gradients G [3][nt] (T/m).

    Lowest-order Maxwell field of a gradient G along a main field B0 z^:
        B_c = [(Gx^2 + Gy^2) z^2 + Gz^2 (x^2 + y^2) / 4 - Gx Gz xz - Gy Gz yz] / (2 B0),
    and the phase gamma * int_0^t B_c, accumulated per dwell (rectangle rule, the same as
    the gradients drawn from the sampled trajectory).
    """
    gx, gy, gz = (np.asarray(g, np.float64) for g in G)
    rate = np.stack([gx * gx + gy * gy, gz * gz / 4.0, -gx * gz, -gy * gz], axis=0) / (2.0 * b0_tesla)
    return GAMMA * dt * np.cumsum(rate, axis=1)


def gradients_from_k(k_phys: np.ndarray, dt: float) -> np.ndarray:
    """G [3][nt] in T/m from physical k [3][nt] (rad/m), k = gamma int G: backward differences,
    k before the first sample = 0."""
    k = np.asarray(k_phys, np.float64)
    return np.diff(k, axis=1, prepend=0.0) / (GAMMA * dt)


def voxel_positions(nx: int, ny: int, fov_x: float, fov_y: float):
    """In-plane coordinates (u, v) of every voxel, row-major (iy, ix)."""
    dx = fov_x / nx
    dy = fov_y / ny
    ix = np.arange(nx)
    iy = np.arange(ny)
    X = (ix[None, :] - nx // 2) * dx + np.zeros((ny, 1))
    Y = (iy[:, None] - ny // 2) * dy + np.zeros((1, nx))
    return X.reshape(-1), Y.reshape(-1)


def spiral_k(nt: int, kmax: float, turns: float, density_power: float) -> np.ndarray:
    """Complex k_x + i k_y of an Archimedean spiral, k(u) = kmax u^p e^{i 2 pi turns u}."""
    u = np.arange(nt, dtype=np.float64) / max(nt - 1, 1)
    return kmax * u ** density_power * np.exp(1j * 2 * np.pi * turns * u)


def exp_smooth(sig: np.ndarray, dt: float, tau: float) -> np.ndarray:
    """Causal convolution with the unit-area kernel e^{-t/tau}/tau, as the first-order
    recursion s[n] = a s[n-1] + (1 - a) x[n], a = exp(-dt/tau)."""
    from scipy.signal import lfilter
    a = math.exp(-dt / tau)
    return lfilter([1.0 - a], [1.0, -a], np.asarray(sig, np.float64))


def ellipse_phantom(rng, X, Y, fov: float, n_ellipses: int = 10) -> np.ndarray:
    img = np.zeros(X.shape, np.complex128)
    for _ in range(n_ellipses):
        rad = 0.4 * fov * math.sqrt(rng.uniform())
        ang = rng.uniform(0, 2 * np.pi)
        cx, cy = rad * math.cos(ang), rad * math.sin(ang)
        a = rng.uniform(0.05, 0.35) * fov
        b = rng.uniform(0.05, 0.35) * fov
        th = rng.uniform(0, np.pi)
        amp = rng.uniform(0.2, 1.0) * np.exp(1j * rng.uniform(-np.pi, np.pi))
        u = (X - cx) * math.cos(th) + (Y - cy) * math.sin(th)
        v = -(X - cx) * math.sin(th) + (Y - cy) * math.cos(th)
        img += amp * ((u / a) ** 2 + (v / b) ** 2 <= 1.0)
    return img


def coil_maps(rng, X, Y, fov: float, nc: int) -> np.ndarray:
    S = np.empty((nc, X.size), np.complex128)
    width = 0.35 * fov
    for c in range(nc):
        ang = 2 * np.pi * c / nc
        cx, cy = 0.6 * fov / 2 * math.cos(ang), 0.6 * fov / 2 * math.sin(ang)
        mag = np.exp(-((X - cx) ** 2 + (Y - cy) ** 2) / (2 * width ** 2))
        g = rng.uniform(-1, 1, size=2) * np.pi / fov
        ph = rng.uniform(-np.pi, np.pi) + g[0] * X + g[1] * Y
        S[c] = mag * np.exp(1j * ph)
    S /= np.sqrt(np.sum(np.abs(S) ** 2, axis=0, keepdims=True))
    return S


def b0_map(rng, X, Y, fov: float, max_hz: float, n_blobs: int = 6) -> np.ndarray:
    f = np.zeros(X.shape)
    for _ in range(n_blobs):
        rad = 0.4 * fov * math.sqrt(rng.uniform())
        ang = rng.uniform(0, 2 * np.pi)
        w = rng.uniform(0.1, 0.3) * fov
        amp = rng.uniform(-1, 1)
        f += amp * np.exp(-((X - rad * math.cos(ang)) ** 2 + (Y - rad * math.sin(ang)) ** 2) / (2 * w * w))
    f *= max_hz / max(np.max(np.abs(f)), 1e-30)
    return 2 * np.pi * f


def field_coefficients(rng, kxy: np.ndarray, h: np.ndarray, dt: float, order: int,
                       rho: float, eddy: bool = True, tilt: float = 0.0, eddy_scale: float = 1.0) -> np.ndarray:
    """k_l(t) for l < (order+1)^2: nominal k_x, k_v cos(tilt), k_v sin(tilt) in terms 1, 2, 3
    (the readout of a slice tilted about x) plus eddy decays.

    Each term receives a_l * s_l * [k_src - (k_src * g_tau)](t), a_l ~ eddy_scale * U[0.01, 0.05],
    tau_l ~ U[0.5, 5] ms, k_src = k_x or k_y (seeded), s_l = rho / max_r |h_l(r)|
    so that the term's phase stays below a_l * kmax * rho at the FOV edge.
    """
    L = n_terms(order)
    nt = kxy.size
    k = np.zeros((L, nt))
    if L > 1:
        k[1] = kxy.real
        k[2] = kxy.imag * math.cos(tilt)
        k[3] = kxy.imag * math.sin(tilt)
    if not eddy:
        return k
    for l in range(L):
        a = rng.uniform(0.01, 0.05)
        tau = rng.uniform(0.5e-3, 5e-3)
        src = kxy.real if rng.uniform() < 0.5 else kxy.imag
        hmax = np.max(np.abs(h[l]))
        scale = rho / hmax if hmax > 0 else rho ** (1 - term_degree(l))
        k[l] += eddy_scale * a * scale * (src - exp_smooth(src, dt, tau))
    return k


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, np.float32))


def _c64(a):
    return np.ascontiguousarray(np.asarray(a, np.complex64))


def make_problem(nx: int, ny: int | None = None, nt: int = 2048, nc: int = 8, order: int = 2,
                 fov: float = 0.22, dwell: float = 4e-6, turns: float | None = None,
                 density_power: float = 1.0, b0_hz: float = 100.0, z0: float = 0.0015,
                 seed: int = BASE_SEED, eddy: bool = True, with_b0: bool = True,
                 shared_geometry_seed: int | None = None, tilt: float = 0.0,
                 concomitant: bool = False, b0_tesla: float = 7.0, eddy_scale: float = 1.0) -> dict:
    """One synthetic slice problem; every array is rounded to float32/complex64.

    Returned keys: nx, ny, nt, nc, nl, k[nl][nt], h[nl][nr], omega[nr], t[nt],
    S[nc][nr], x_gt[nr], noise[nc][nt] (E|n|^2 = 1), fov, dwell, z0, seed.
    ``shared_geometry_seed`` draws the phantom, coils and B0 from a second stream
    (used when many diffusion volumes share one slice and differ only in the field).
    ``tilt`` (rad) rotates the slice about the x axis; the readout's in-plane k_v then drives
    the physical y and z gradients (k_y = k_v cos tilt, k_z = k_v sin tilt).
    ``concomitant`` appends the four second-order concomitant-field rows (z^2, x^2 + y^2, xz,
    yz) of the readout gradients at ``b0_tesla`` after the spherical-harmonic rows.
    """
    ny = nx if ny is None else ny
    rng = np.random.default_rng(seed)
    grng = rng if shared_geometry_seed is None else np.random.default_rng(shared_geometry_seed)
    U, V = voxel_positions(nx, ny, fov, fov * ny / nx)
    ct, st = math.cos(tilt), math.sin(tilt)
    X, Y, Z = U, V * ct, V * st + z0
    h = sh_basis(X, Y, Z, order)
    kmax = math.pi / (fov / nx)
    if turns is None:
        turns = nx / 8.0
    kxy = spiral_k(nt, kmax, turns, density_power)
    k = field_coefficients(rng, kxy, h, dwell, order, fov / 2, eddy, tilt, eddy_scale)
    t = np.arange(nt) * dwell
    omega = b0_map(grng, U, V, fov, b0_hz) if with_b0 else np.zeros(U.size)
    S = coil_maps(grng, U, V, fov, nc)
    x_gt = ellipse_phantom(grng, U, V, fov)
    noise = (rng.standard_normal((nc, nt)) + 1j * rng.standard_normal((nc, nt))) / math.sqrt(2)
    if concomitant:
        kphys = np.stack([kxy.real, kxy.imag * ct, kxy.imag * st], axis=0)
        h = np.concatenate([h, concomitant_basis(X, Y, Z)], axis=0)
        k = np.concatenate([k, concomitant_coefficients(gradients_from_k(kphys, dwell), dwell, b0_tesla)], axis=0)
    return dict(nx=nx, ny=ny, nt=nt, nc=nc, nl=h.shape[0], k=_f32(k), h=_f32(h),
                omega=_f32(omega), t=_f32(t), S=_c64(S), x_gt=_c64(x_gt), noise=_c64(noise),
                fov=fov, dwell=dwell, z0=z0, seed=seed, tilt=tilt)


# --------------------------------------------------------------------------
# The workloads, by what they are.
# --------------------------------------------------------------------------

def tiny_64(index: int = 0) -> dict:
    """64x64, FOV 220 mm, 8 coils, variable-density spiral (16 turns, u^1.5),
    2048 samples at 4 us, 2nd-order field (9 terms), B0 within +-100 Hz.
    Reconstructed with a 3-level Haar wavelet, 20 FISTA iterations, SNR 20."""
    p = make_problem(64, nt=2048, nc=8, order=2, dwell=4e-6, turns=16.0, density_power=1.5,
                     b0_hz=100.0, seed=BASE_SEED + 1000 * 1 + index)
    p.update(snr=20.0, wavelet="haar", levels=3, iters=20, lambda_rel=1e-3)
    return p


def slice_200(index: int = 0) -> dict:
    """200x200 (1.1 mm), 32 coils, uniform single-shot spiral at R = 4 (25 turns),
    24 000 samples at 1 us, 3rd-order field (16 terms) plus B0 within +-150 Hz.
    Reconstructed with a 4-level Daubechies-4 wavelet, 50 FISTA iterations, SNR 10."""
    p = make_problem(200, nt=24000, nc=32, order=3, dwell=1e-6, turns=200 / 8.0,
                     density_power=1.0, b0_hz=150.0, seed=BASE_SEED + 1000 * 2 + index)
    p.update(snr=10.0, wavelet="db4", levels=4, iters=50, lambda_rel=1e-3)
    return p


def slice_200_expanded(index: int = 0) -> dict:
    """The 200x200 slice with a field model beyond 3rd order: 4th-order solid harmonics
    (25 terms), the four second-order concomitant-field rows of the readout at 7 T, plus B0
    (30 terms), on a slice tilted by 20 degrees about x, 20 mm off isocentre."""
    p = make_problem(200, nt=24000, nc=32, order=4, dwell=1e-6, turns=200 / 8.0,
                     density_power=1.0, b0_hz=150.0, seed=BASE_SEED + 1000 * 2 + index,
                     tilt=math.radians(20.0), z0=0.02, concomitant=True)
    p.update(snr=10.0, wavelet="db4", levels=4, iters=50, lambda_rel=1e-3)
    return p


def diff_170(index: int = 0) -> dict:
    """170x170, 16 coils, uniform spiral at R = 4, 12 000 samples at 2 us,
    2nd-order field (9 terms) plus B0 within +-100 Hz (differentiation workload)."""
    p = make_problem(170, nt=12000, nc=16, order=2, dwell=2e-6, turns=170 / 8.0,
                     density_power=1.0, b0_hz=100.0, seed=BASE_SEED + 1000 * 5 + index)
    p.update(snr=20.0, wavelet="db4", levels=4, iters=10, lambda_rel=1e-3)
    return p


def ragged_protocol_nt(n: int, r: float) -> int:
    """Samples of a single-shot spiral at N^2 and acceleration R, clipped to 8k..30k."""
    return int(min(max(round(24000 * (n / 200.0) ** 2 * (4.0 / r)), 8000), 30000))


RAGGED_PROTOCOLS = ((148, 6.0), (170, 3.0), (200, 2.0))  # 1.5 / 1.3 / 1.1 mm
RAGGED_SLICES_Z = (-0.0045, -0.0015, 0.0015, 0.0045)    # 3 mm slices


def ragged_problem(res: int, volume: int, slice_: int, nc: int = 32) -> dict:
    """One slice of the ragged batch: resolution index ``res`` (148/170/200),
    diffusion volume ``volume`` (0 = b0, 1..30 directions: own field), slice ``slice_``.
    Geometry (phantom, coils, B0) is shared by all volumes of a slice."""
    n, r = RAGGED_PROTOCOLS[res]
    nt = ragged_protocol_nt(n, r)
    seed = BASE_SEED + 1000 * 4 + 10000 * res + 100 * slice_ + volume
    gseed = BASE_SEED + 1000 * 4 + 10000 * res + 100 * slice_ + 99
    p = make_problem(n, nt=nt, nc=nc, order=3, dwell=1e-6, turns=n / (2.0 * r),
                     density_power=1.0, b0_hz=150.0, z0=RAGGED_SLICES_Z[slice_],
                     seed=seed, shared_geometry_seed=gseed)
    p.update(snr=10.0, wavelet="db4", levels=4, iters=50, lambda_rel=1e-3)
    return p


def cartesian_problem(n: int, fov: float = 0.2) -> dict:
    """Cartesian DFT set-up: k = 2 pi (m - n/2)/FOV on an n x n grid, terms (1, x, y)
    with k_0 = 0, no B0, one coil with S = 1, nt = n^2 (row-major m_y, m_x)."""
    X, Y = voxel_positions(n, n, fov, fov)
    h = sh_basis(X, Y, 0.0, 1)[:3]
    m = (np.arange(n) - n // 2) * 2 * np.pi / fov
    KY, KX = np.meshgrid(m, m, indexing="ij")
    k = np.zeros((3, n * n))
    k[1] = KX.reshape(-1)
    k[2] = KY.reshape(-1)
    return dict(nx=n, ny=n, nt=n * n, nc=1, nl=3, k=_f32(k), h=_f32(h),
                omega=_f32(np.zeros(n * n)), t=_f32(np.zeros(n * n)),
                S=_c64(np.ones((1, n * n))), fov=fov)


def random_image(rng, n: int) -> np.ndarray:
    return _c64(rng.standard_normal(n) + 1j * rng.standard_normal(n))


def random_kspace(rng, nc: int, nt: int) -> np.ndarray:
    return _c64(rng.standard_normal((nc, nt)) + 1j * rng.standard_normal((nc, nt)))
