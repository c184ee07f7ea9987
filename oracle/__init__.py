"""FP64 CPU oracle of the expanded-encoding CS reconstruction (Eq. 1).

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  It shares no code
with the CUDA library and never imports it; the product path fails loudly
without its CUDA extension instead of falling back to anything here.

Contents
--------
* ``forward`` / ``adjoint`` (and the one-output-at-a-time ``*_rows`` forms):
  plain FP64 double sums of A_exp and A_exp^H in C (``aexp_oracle.c``).
* ``oracle.wavelet``: periodised orthonormal 2-D DWT (Haar, Daubechies-4 from
  its spectral factorisation), complex soft-threshold, the prox step.
* ``oracle.coilcomp``: coil compression by principal components of the k-space data;
* ``oracle.swt``: the paper's own regulariser -- one-level undecimated wavelet (a tight frame),
  the balanced-FISTA step with it and lambda = sigma / 2 from the histogram of W A^H y;
* ``oracle.recon``: power-iteration Lipschitz estimate, FISTA, CGLS, objective,
  NRMSE, and reverse-mode gradients of unrolled FISTA;
* ``oracle.precision``: the BF16 form's rounding written out (dense, small problems), which
  the solvers above can run on to show what the rounding alone does to a reconstruction.

Every function takes a problem dict with keys nt, nx, ny, nc, nl and arrays
k[nl][nt], h[nl][nr], omega[nr] (or None), t[nt], S[nc][nr]; inputs are promoted
to FP64 before any arithmetic.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "aexp_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C part of the oracle (gcc, FP64, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fPIC",
                               "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        I = ctypes.c_int
        for name in ("oracle_forward", "oracle_adjoint", "oracle_forward_dk", "oracle_adjoint_dk"):
            getattr(lib, name).argtypes = [I, I, I, I, P, P, P, P, P, P, P] + (
                [P] if name.endswith("_dk") else [])
            getattr(lib, name).restype = None
        for name in ("oracle_forward_rows", "oracle_adjoint_rows"):
            getattr(lib, name).argtypes = [I, I, I, I, P, P, P, P, P, P, I, P, P]
            getattr(lib, name).restype = None
        _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _c128(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.complex128))


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _geom(prob):
    nl, nt = np.shape(prob["k"])
    nr = np.shape(prob["h"])[1]
    nc = np.shape(prob["S"])[0]
    k = _f64(prob["k"])
    h = _f64(prob["h"])
    om = prob.get("omega")
    om = None if om is None else _f64(om)
    tt = _f64(prob["t"]) if om is not None else None
    S = _c128(prob["S"])
    return nt, nr, nc, nl, k, h, om, tt, S


def forward(prob, x):
    """y = A_exp x, returned as complex128 [nc][nt]."""
    nt, nr, nc, nl, k, h, om, tt, S = _geom(prob)
    x = _c128(x).reshape(nr)
    y = np.zeros((nc, nt), np.complex128)
    _load().oracle_forward(nt, nr, nc, nl, _ptr(k), _ptr(h), _ptr(om), _ptr(tt), _ptr(S), _ptr(x), _ptr(y))
    return y


def adjoint(prob, y):
    """x = A_exp^H y, returned as complex128 [nr]."""
    nt, nr, nc, nl, k, h, om, tt, S = _geom(prob)
    y = _c128(y).reshape(nc, nt)
    x = np.zeros(nr, np.complex128)
    _load().oracle_adjoint(nt, nr, nc, nl, _ptr(k), _ptr(h), _ptr(om), _ptr(tt), _ptr(S), _ptr(y), _ptr(x))
    return x


def forward_rows(prob, x, ts):
    """y_c(t) for the sample indices ``ts`` only: complex128 [nc][len(ts)]."""
    nt, nr, nc, nl, k, h, om, tt, S = _geom(prob)
    x = _c128(x).reshape(nr)
    ts = np.ascontiguousarray(np.asarray(ts, np.int32))
    y = np.zeros((nc, ts.size), np.complex128)
    _load().oracle_forward_rows(nt, nr, nc, nl, _ptr(k), _ptr(h), _ptr(om), _ptr(tt), _ptr(S), _ptr(x),
                                int(ts.size), _ptr(ts), _ptr(y))
    return y


def adjoint_rows(prob, y, rs):
    """(A^H y)(r) for the voxel indices ``rs`` only: complex128 [len(rs)]."""
    nt, nr, nc, nl, k, h, om, tt, S = _geom(prob)
    y = _c128(y).reshape(nc, nt)
    rs = np.ascontiguousarray(np.asarray(rs, np.int32))
    x = np.zeros(rs.size, np.complex128)
    _load().oracle_adjoint_rows(nt, nr, nc, nl, _ptr(k), _ptr(h), _ptr(om), _ptr(tt), _ptr(S), _ptr(y),
                                int(rs.size), _ptr(rs), _ptr(x))
    return x


def forward_dk(prob, x, g):
    """G_l(t) = sum_c conj(g_c(t)) d(A x)_c(t)/dk_l(t)  (complex128 [nl][nt])."""
    nt, nr, nc, nl, k, h, om, tt, S = _geom(prob)
    x = _c128(x).reshape(nr)
    g = _c128(g).reshape(nc, nt)
    G = np.zeros((nl, nt), np.complex128)
    _load().oracle_forward_dk(nt, nr, nc, nl, _ptr(k), _ptr(h), _ptr(om), _ptr(tt), _ptr(S), _ptr(x),
                              _ptr(g), _ptr(G))
    return G


def adjoint_dk(prob, y, g):
    """G_l(t) = sum_r conj(g(r)) d(A^H y)(r)/dk_l(t)  (complex128 [nl][nt])."""
    nt, nr, nc, nl, k, h, om, tt, S = _geom(prob)
    y = _c128(y).reshape(nc, nt)
    g = _c128(g).reshape(nr)
    G = np.zeros((nl, nt), np.complex128)
    _load().oracle_adjoint_dk(nt, nr, nc, nl, _ptr(k), _ptr(h), _ptr(om), _ptr(tt), _ptr(S), _ptr(y),
                              _ptr(g), _ptr(G))
    return G


def threads() -> int:
    """Number of OpenMP threads the C oracle will use."""
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else (os.cpu_count() or 1)
