"""Coil compression (FP64): principal components of the k-space data.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Sec. 2.2.1 reduces the 32 receive channels to 20 virtual coils so that the reconstruction runs
faster, and Sec. 2.2.2 studies 8, 16 and 32 virtual coils; the method is not stated.  Reading:
principal components of the measured data, the same matrix applied to data and coil maps:
    C = y y^H  (nc x nc, y: [nc][nt]),  C = U diag(e) U^H with e descending,
    every column u_k scaled by conj(u_ak*) / |u_ak*| where a* = argmax_a |u_ak| (lowest a on a
    tie), so that its largest component is real and positive (unique up to equal eigenvalues),
    y_v = U_v^H y ([nv][nt]),  S_v = U_v^H S ([nv][nr]),  U_v = the first nv columns.
Because the encoding matrix E(t, r) does not depend on the coil, the compressed problem
(same field terms, nc = nv, S = S_v) has (A_v x)_k = sum_a conj(U_ak) (A x)_a: with nv = nc it
is the original problem up to a unitary mixing of the coils.
"""

from __future__ import annotations

import numpy as np


def compression_matrix(y: np.ndarray):
    """(eigenvalues descending, U with normalised columns) of C = y y^H."""
    y = np.asarray(y, np.complex128)
    C = y @ y.conj().T
    e, U = np.linalg.eigh(C)                 # ascending
    e, U = e[::-1], U[:, ::-1].copy()
    for k in range(U.shape[1]):
        a = int(np.argmax(np.abs(U[:, k])))
        U[:, k] *= np.conj(U[a, k]) / abs(U[a, k])
    return e, U


def compress(prob: dict, y: np.ndarray, nv: int):
    """(compressed problem dict, y_v [nv][nt], eigenvalues descending)."""
    e, U = compression_matrix(y)
    Uv = U[:, :nv]
    yv = Uv.conj().T @ np.asarray(y, np.complex128)
    Sv = Uv.conj().T @ np.asarray(prob["S"], np.complex128)
    q = dict(prob)
    q["nc"] = nv
    q["S"] = Sv
    return q, yv, e
