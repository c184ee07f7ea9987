"""Rounding emulation of the BF16 tensor-core form of A_exp and A_exp^H (FP64 otherwise).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The BF16 form (Sec. 1's operator of Eq. 1 evaluated on tensor cores) rounds, once each, every
real component of
  * the encoding elements E(t, r) = cos phi(t, r) - i sin phi(t, r) (its conjugate in the adjoint),
  * the contraction operand: the coil-weighted image b_c(r) = S_c(r) x(r) in the forward, the
    k-space data y_c(t) in the adjoint,
to BF16 (8 significant bits, round to nearest, ties to even), after the value was formed in
FP32; products and sums then run in FP32, which adds only ~1e-7 relative.  Written out densely
below (E is formed as an [nt][nr] matrix, so small problems only):

    (A_bf x)_c(t)  = sum_r bf(E(t, r)) bf(f32(S_c(r) x(r)))
    (A_bf^H y)(r)  = sum_c conj(S_c(r)) sum_t conj(bf(E(t, r))) bf(f32(y_c(t)))

with bf(a + ib) = bf(a) + i bf(b).  Running the oracle's own solvers on this pair gives the
image the rounding alone would produce; its distance to the exact oracle sets the scale of a
reduced-precision reconstruction's error after a given number of iterations.
"""

from __future__ import annotations

import numpy as np


def bf16_round(a) -> np.ndarray:
    """float32 values rounded to BF16 (round to nearest, ties to even), returned as float64."""
    f = np.ascontiguousarray(np.asarray(a, np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_complex(z) -> np.ndarray:
    """Both components of FP32-rounded complex values rounded to BF16 (complex128)."""
    z = np.asarray(z, np.complex128)
    return bf16_round(z.real) + 1j * bf16_round(z.imag)


def encoding_matrix(prob) -> np.ndarray:
    """E(t, r) = exp(-i phi(t, r)), phi = sum_l k_l(t) h_l(r) + omega(r) t, FP64, [nt][nr]."""
    k = np.asarray(prob["k"], np.float64)
    h = np.asarray(prob["h"], np.float64)
    phi = k.T @ h
    if prob.get("omega") is not None:
        phi += np.outer(np.asarray(prob["t"], np.float64), np.asarray(prob["omega"], np.float64))
    return np.exp(-1j * phi)


def bf16_operators(prob, rounding: bool = True):
    """(A_bf, A_bf^H) callables on flat complex vectors; ``rounding=False`` gives the exact
    dense operator (the same sums without the BF16 steps)."""
    E = encoding_matrix(prob)
    S = np.asarray(prob["S"], np.complex128)
    nc, nt = S.shape[0], E.shape[0]
    if rounding:
        E = bf16_complex(E.astype(np.complex64))
    rnd = (lambda z: bf16_complex(np.asarray(z, np.complex128).astype(np.complex64))) if rounding else (lambda z: z)

    def fwd(x):
        b = S * np.asarray(x, np.complex128).reshape(1, -1)     # [nc][nr]
        return rnd(b) @ E.T                                      # [nc][nt]

    def adj(y):
        u = rnd(np.asarray(y, np.complex128).reshape(nc, nt)) @ np.conj(E)   # [nc][nr]
        return np.sum(np.conj(S) * u, axis=0)

    return fwd, adj
