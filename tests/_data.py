"""Seeded test data shared by the GPU parity tests.  Every expected value comes from
the FP64 oracle (never from the CUDA path)."""

import functools

import numpy as np

from paper_2211_07532_gb300 import synth


def rel(a, b):
    a = np.asarray(a, np.complex128).reshape(-1)
    b = np.asarray(b, np.complex128).reshape(-1)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@functools.lru_cache(maxsize=None)
def simulated(name: str, index: int = 0):
    """(problem, y complex64 [nc][nt], lam float32) for a named workload:
    y = A x_gt + n with E|n|^2 = sigma^2, sigma = rms|A x_gt| / SNR (oracle forward),
    lam = 1e-3 * ||A^H y||_inf (oracle adjoint), both rounded to storage precision."""
    import oracle
    p = getattr(synth, name)(index)
    y0 = oracle.forward(p, p["x_gt"])
    sigma = np.sqrt(np.mean(np.abs(y0) ** 2)) / p["snr"]
    y = (y0 + sigma * p["noise"]).astype(np.complex64)
    lam = np.float32(p["lambda_rel"] * np.max(np.abs(oracle.adjoint(p, y))))
    return p, y, float(lam)
