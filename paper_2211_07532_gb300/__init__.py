"""GB300 (sm_103a) expanded-encoding compressed-sensing reconstruction (Eq. 1).

Thin Python binding over the C ABI of ``libaexp.so`` (declared in include/aexp.h).
Every numeric step runs in the library's CUDA kernels; this module only marshals
arguments: PyTorch provides device memory and the current stream.  There is no CPU
fallback: without the built library every entry point raises.

Names follow the C ABI: ``a_exp_forward``, ``a_exp_adjoint``, ``cs_recon``,
``power_lipschitz``, ``wavelet_prox``, ``wavelet_forward``.
"""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libaexp.so")

FP32, BF16_TC, FP16X2_TC = 0, 1, 2
HAAR, DB4 = 0, 1
WAVELETS = {"haar": HAAR, "db4": DB4}

OK = 0
STATUS = {0: "AEXP_OK", -1: "AEXP_ERR_INVALID_ARG", -2: "AEXP_ERR_MISALIGNED", -3: "AEXP_ERR_UNSUPPORTED",
          -4: "AEXP_ERR_WORKSPACE", -5: "AEXP_ERR_CUDA", -6: "AEXP_ERR_DEVICE_TIMEOUT",
          -7: "AEXP_ERR_NONFINITE", -8: "AEXP_ERR_NOT_PREPARED"}


class AexpError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        msg = f"{what} failed: {STATUS.get(code, code)}"
        if code == -5 and _lib is not None:
            msg += f" (cudaError {_lib.aexp_last_cuda_error()})"
        super().__init__(msg)


class CProblem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nt", ctypes.c_int), ("nc", ctypes.c_int),
                ("nl", ctypes.c_int), ("k", ctypes.c_void_p), ("h", ctypes.c_void_p),
                ("omega", ctypes.c_void_p), ("t", ctypes.c_void_p), ("S", ctypes.c_void_p)]


class CReconOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("wavelet", ctypes.c_int), ("levels", ctypes.c_int),
                ("n_power", ctypes.c_int), ("lipschitz", ctypes.c_double), ("x0", ctypes.c_void_p),
                ("power_init", ctypes.c_void_p), ("use_graph", ctypes.c_int), ("undecimated", ctypes.c_int),
                ("lambda_rule", ctypes.c_int), ("lambda_out", ctypes.c_void_p), ("items_per_sm", ctypes.c_int),
                ("tile_variant", ctypes.c_int)]


_lib = None

# (name, restype, argtypes) of every entry point in include/aexp.h
_P = ctypes.c_void_p
_I = ctypes.c_int
_SZ = ctypes.c_size_t
_PROB = ctypes.POINTER(CProblem)
_OPTS = ctypes.POINTER(CReconOpts)
SIGNATURES = [
    ("aexp_workspace_size", _I, [_PROB, _I, ctypes.POINTER(_SZ)]),
    ("aexp_prepare", _I, [_PROB, _I, _P, _SZ, _P]),
    ("aexp_workspace_size_tiled", _I, [_PROB, _I, _I, _I, ctypes.POINTER(_SZ)]),
    ("aexp_prepare_tiled", _I, [_PROB, _I, _I, _I, _P, _SZ, _P]),
    ("a_exp_forward", _I, [_PROB, _I, _P, _P, _P, _SZ, _P]),
    ("a_exp_adjoint", _I, [_PROB, _I, _P, _P, _P, _SZ, _P]),
    ("aexp_recon_opts_default", None, [_OPTS]),
    ("aexp_recon_workspace_size", _I, [_PROB, _OPTS, ctypes.POINTER(_SZ)]),
    ("cs_recon", _I, [_PROB, _P, ctypes.c_float, _I, _OPTS, _P, _P, _P, _SZ, _P]),
    ("aexp_power_lipschitz", _I, [_PROB, _I, _P, _I, _P, _P, _SZ, _P]),
    ("aexp_batch_workspace_size", _I, [_PROB, _I, _OPTS, ctypes.POINTER(_SZ)]),
    ("cs_recon_batched", _I, [_PROB, _I, ctypes.POINTER(_P), ctypes.POINTER(ctypes.c_float), _I, _OPTS,
                              ctypes.POINTER(_P), _P, _P, _SZ, _P]),
    ("aexp_unroll_workspace_size", _I, [_PROB, _OPTS, ctypes.POINTER(_SZ)]),
    ("aexp_fista_step", _I, [_PROB, _OPTS, _P, ctypes.c_float, ctypes.c_double, _P, _P, ctypes.c_double, _P, _P, _P,
                             _SZ, _P]),
    ("aexp_fista_step_vjp", _I, [_PROB, _OPTS, _P, ctypes.c_float, ctypes.c_double, _P, ctypes.c_double,
                                 ctypes.c_double, _P, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    ("aexp_wavelet_workspace_size", _I, [_I, _I, _I, _I, ctypes.POINTER(_SZ)]),
    ("aexp_wavelet_prox", _I, [_I, _I, _I, _I, ctypes.c_float, _P, _P, _P, _SZ, _P]),
    ("aexp_wavelet_forward", _I, [_I, _I, _I, _I, _P, _P, _P, _SZ, _P]),
    ("aexp_wavelet_prox_static", _I, [_I, _I, _I, _I, ctypes.c_float, _P, _P, _P]),
    ("aexp_coil_compress_workspace_size", _I, [_I, ctypes.POINTER(_SZ)]),
    ("aexp_coil_compress", _I, [_PROB, _P, _I, _P, _P, _P, _P, _SZ, _P]),
    ("aexp_coil_compress_status", _I, [_P, _I, _P, ctypes.POINTER(_I)]),
    ("aexp_coil_compress_sweeps", _I, [_PROB, _P, _I, _I, _P, _P, _P, _P, _SZ, _P]),
    ("aexp_probe_bounded_wait", _I, [_I, _P, _P, _SZ, _P]),
    ("aexp_header_bytes", _SZ, []),
    ("aexp_swt_workspace_size", _I, [_I, _I, ctypes.POINTER(_SZ)]),
    ("aexp_swt_forward", _I, [_I, _I, _I, _P, _P, _P]),
    ("aexp_swt_prox", _I, [_I, _I, _I, ctypes.c_float, _P, _P, _P, _SZ, _P]),
    ("aexp_swt_lambda", _I, [_I, _I, _I, _P, _P, _P, _SZ, _P]),
    ("aexp_cgls_workspace_size", _I, [_PROB, _OPTS, ctypes.POINTER(_SZ)]),
    ("cgls_recon", _I, [_PROB, _P, _I, _OPTS, _P, _P, _SZ, _P]),
    ("aexp_autotune_workspace_size", _I, [_PROB, _I, _OPTS, ctypes.POINTER(_SZ)]),
    ("aexp_autotune", _I, [_PROB, _I, _OPTS, _P, _SZ, _P, ctypes.POINTER(_I), ctypes.POINTER(_I),
                           ctypes.POINTER(ctypes.c_float)]),
    ("aexp_read_status", _I, [_P, _P, ctypes.POINTER(_I)]),
    ("aexp_status_string", ctypes.c_char_p, [_I]),
    ("aexp_last_cuda_error", _I, []),
    ("aexp_version", _I, []),
]


def lib():
    """Load libaexp.so (raises when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2211_07532_gb300.build.build()")
        h = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(h, name)
            fn.restype = res
            fn.argtypes = args
        _lib = h
    return _lib


def _check(code: int, what: str):
    if code != OK:
        raise AexpError(code, what)


def _torch():
    import torch
    return torch


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    torch = _torch()
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


class Problem:
    """Device arrays of one slice problem (see aexp_problem in include/aexp.h).

    k: float32 [nl][nt]; h: float32 [nl][nr]; omega: float32 [nr] or None;
    t: float32 [nt]; S: complex64 [nc][nr].  Tensors are kept alive by this object.
    """

    def __init__(self, nx, ny, k, h, S, omega=None, t=None):
        torch = _torch()
        self.nx, self.ny = int(nx), int(ny)
        self.k = k.contiguous()
        self.h = h.contiguous()
        self.S = S.contiguous()
        self.omega = None if omega is None else omega.contiguous()
        self.t = None if t is None else t.contiguous()
        assert self.k.dtype == torch.float32 and self.h.dtype == torch.float32
        assert self.S.dtype == torch.complex64
        self.nl, self.nt = self.k.shape
        self.nc = self.S.shape[0]
        self.nr = self.nx * self.ny
        self._c = CProblem(self.nx, self.ny, self.nt, self.nc, self.nl, self.k.data_ptr(), self.h.data_ptr(),
                           None if self.omega is None else self.omega.data_ptr(),
                           None if self.t is None else self.t.data_ptr(), self.S.data_ptr())

    @classmethod
    def from_arrays(cls, d: dict, device="cuda", with_b0: bool = True):
        """From a dict of numpy arrays (keys nx, ny, k, h, omega, t, S)."""
        torch = _torch()
        dev = torch.device(device)
        om = d.get("omega")
        use_b0 = with_b0 and om is not None
        return cls(d["nx"], d["ny"], torch.as_tensor(d["k"], dtype=torch.float32, device=dev),
                   torch.as_tensor(d["h"], dtype=torch.float32, device=dev),
                   torch.as_tensor(d["S"], dtype=torch.complex64, device=dev),
                   torch.as_tensor(om, dtype=torch.float32, device=dev) if use_b0 else None,
                   torch.as_tensor(d["t"], dtype=torch.float32, device=dev) if use_b0 else None)

    def with_coils(self, S):
        """The same field model with other coil maps S [nc'][nr] (e.g. virtual coils)."""
        return Problem(self.nx, self.ny, self.k, self.h, S, self.omega, self.t)

    @property
    def c(self):
        return ctypes.byref(self._c)

    @property
    def device(self):
        return self.S.device


def workspace_size(prob: Problem, precision: int = FP32, items_per_sm: int = 0, tile_variant: int = 0) -> int:
    n = ctypes.c_size_t()
    if items_per_sm or tile_variant:
        _check(lib().aexp_workspace_size_tiled(prob.c, precision, items_per_sm, tile_variant, ctypes.byref(n)),
               "aexp_workspace_size_tiled")
    else:
        _check(lib().aexp_workspace_size(prob.c, precision, ctypes.byref(n)), "aexp_workspace_size")
    return n.value


def _alloc(nbytes: int, device):
    torch = _torch()
    ws = torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)
    if ws.data_ptr() % 256:
        raise RuntimeError("workspace is not 256-byte aligned")
    return ws


def workspace(prob: Problem, precision: int = FP32, items_per_sm: int = 0, tile_variant: int = 0):
    return _alloc(workspace_size(prob, precision, items_per_sm, tile_variant), prob.device)


def prepare(prob: Problem, ws, precision: int = FP32, stream=None, items_per_sm: int = 0, tile_variant: int = 0):
    """Prepare ws for the operator calls; a nonzero items_per_sm / tile_variant selects that
    launch shape (aexp_prepare_tiled), which the operator calls on ws then use."""
    if items_per_sm or tile_variant:
        _check(lib().aexp_prepare_tiled(prob.c, precision, items_per_sm, tile_variant, _ptr(ws), ws.numel(),
                                        _stream(stream)), "aexp_prepare_tiled")
    else:
        _check(lib().aexp_prepare(prob.c, precision, _ptr(ws), ws.numel(), _stream(stream)), "aexp_prepare")


def a_exp_forward(prob: Problem, x, ws, y=None, precision: int = FP32, stream=None):
    """y = A_exp x  (x: complex64 [nr]; returns complex64 [nc][nt])."""
    torch = _torch()
    x = x.contiguous()
    if y is None:
        y = torch.empty((prob.nc, prob.nt), dtype=torch.complex64, device=x.device)
    _check(lib().a_exp_forward(prob.c, precision, _ptr(x), _ptr(y), _ptr(ws), ws.numel(), _stream(stream)),
           "a_exp_forward")
    return y


def a_exp_adjoint(prob: Problem, y, ws, x=None, precision: int = FP32, stream=None):
    """x = A_exp^H y  (y: complex64 [nc][nt]; returns complex64 [nr])."""
    torch = _torch()
    y = y.contiguous()
    if x is None:
        x = torch.empty(prob.nr, dtype=torch.complex64, device=y.device)
    _check(lib().a_exp_adjoint(prob.c, precision, _ptr(y), _ptr(x), _ptr(ws), ws.numel(), _stream(stream)),
           "a_exp_adjoint")
    return x


LAMBDA_GIVEN, LAMBDA_RAYLEIGH = 0, 1


def recon_opts(precision=FP32, wavelet="haar", levels=3, n_power=30, lipschitz=0.0, x0=None, power_init=None,
               use_graph=True, items_per_sm=0, undecimated=False, lambda_rule=LAMBDA_GIVEN,
               lambda_out=None, tile_variant=0) -> CReconOpts:
    o = CReconOpts()
    lib().aexp_recon_opts_default(ctypes.byref(o))
    o.precision = precision
    o.wavelet = WAVELETS[wavelet] if isinstance(wavelet, str) else int(wavelet)
    o.levels = levels
    o.n_power = n_power
    o.lipschitz = float(lipschitz)
    o.x0 = None if x0 is None else x0.data_ptr()
    o.power_init = None if power_init is None else power_init.data_ptr()
    o.use_graph = 1 if use_graph else 0
    o.items_per_sm = int(items_per_sm)
    o.tile_variant = int(tile_variant)
    o.undecimated = 1 if undecimated else 0
    o.lambda_rule = int(lambda_rule)
    o.lambda_out = None if lambda_out is None else lambda_out.data_ptr()
    return o


def recon_workspace_size(prob: Problem, opts: CReconOpts) -> int:
    n = ctypes.c_size_t()
    _check(lib().aexp_recon_workspace_size(prob.c, ctypes.byref(opts), ctypes.byref(n)),
           "aexp_recon_workspace_size")
    return n.value


def recon_workspace(prob: Problem, opts: CReconOpts):
    return _alloc(recon_workspace_size(prob, opts), prob.device)


def cs_recon(prob: Problem, y, lam: float, iters: int, opts: CReconOpts | None = None, ws=None, x_out=None,
             lipschitz_out=None, stream=None, **kw):
    """FISTA on Eq. (1); returns (x complex64 [nr], L_f float64 device tensor [1])."""
    torch = _torch()
    opts = recon_opts(**kw) if opts is None else opts
    y = y.contiguous()
    if ws is None:
        ws = recon_workspace(prob, opts)
    if x_out is None:
        x_out = torch.empty(prob.nr, dtype=torch.complex64, device=y.device)
    if lipschitz_out is None:
        lipschitz_out = torch.empty(1, dtype=torch.float64, device=y.device)
    _check(lib().cs_recon(prob.c, _ptr(y), float(lam), int(iters), ctypes.byref(opts), _ptr(x_out),
                          _ptr(lipschitz_out), _ptr(ws), ws.numel(), _stream(stream)), "cs_recon")
    return x_out, lipschitz_out


def _prob_array(probs):
    arr = (CProblem * len(probs))()
    for i, pr in enumerate(probs):
        arr[i] = pr._c
    return arr


def batch_workspace_size(probs, opts: CReconOpts) -> int:
    n = ctypes.c_size_t()
    _check(lib().aexp_batch_workspace_size(_prob_array(probs), len(probs), ctypes.byref(opts), ctypes.byref(n)),
           "aexp_batch_workspace_size")
    return n.value


def cs_recon_batched(probs, ys, lams, iters: int, opts: CReconOpts | None = None, ws=None, x_outs=None,
                     lipschitz_out=None, stream=None, **kw):
    """FISTA on Eq. (1) for a ragged batch of problems in one graph; returns (list of x, L_f [n])."""
    torch = _torch()
    opts = recon_opts(**kw) if opts is None else opts
    n = len(probs)
    probs_c = _prob_array(probs)
    ys = [y.contiguous() for y in ys]
    dev = ys[0].device
    if ws is None:
        ws = _alloc(batch_workspace_size(probs, opts), dev)
    if x_outs is None:
        x_outs = [torch.empty(pr.nr, dtype=torch.complex64, device=dev) for pr in probs]
    if lipschitz_out is None:
        lipschitz_out = torch.empty(n, dtype=torch.float64, device=dev)
    yp = (ctypes.c_void_p * n)(*[y.data_ptr() for y in ys])
    xp = (ctypes.c_void_p * n)(*[x.data_ptr() for x in x_outs])
    lp = (ctypes.c_float * n)(*[float(v) for v in lams])
    _check(lib().cs_recon_batched(probs_c, n, yp, lp, int(iters), ctypes.byref(opts), xp, _ptr(lipschitz_out),
                                  _ptr(ws), ws.numel(), _stream(stream)), "cs_recon_batched")
    return x_outs, lipschitz_out


def coil_compress(prob: Problem, y, nv: int, stream=None, max_sweeps: int = 40):
    """Principal-component coil compression: returns (compressed Problem with nc = nv,
    y_v [nv][nt] complex64, eigenvalues float64 [nc] descending), all on the device.
    Raises AexpError (AEXP_ERR_NONFINITE) when the Jacobi iteration has not converged within
    ``max_sweeps`` sweeps."""
    torch = _torch()
    y = y.contiguous()
    dev = y.device
    n = ctypes.c_size_t()
    _check(lib().aexp_coil_compress_workspace_size(prob.nc, ctypes.byref(n)), "aexp_coil_compress_workspace_size")
    ws = _alloc(n.value, dev)
    yv = torch.empty((nv, prob.nt), dtype=torch.complex64, device=dev)
    Sv = torch.empty((nv, prob.nr), dtype=torch.complex64, device=dev)
    eig = torch.empty(prob.nc, dtype=torch.float64, device=dev)
    _check(lib().aexp_coil_compress_sweeps(prob.c, _ptr(y), int(nv), int(max_sweeps), _ptr(yv), _ptr(Sv), _ptr(eig),
                                           _ptr(ws), ws.numel(), _stream(stream)), "aexp_coil_compress")
    st = ctypes.c_int()
    _check(lib().aexp_coil_compress_status(_ptr(ws), prob.nc, _stream(stream), ctypes.byref(st)),
           "aexp_coil_compress_status")
    _check(st.value, "coil compression (Jacobi)")
    return prob.with_coils(Sv), yv, eig


def probe_bounded_wait(polls: int, device="cuda", stream=None):
    """Run the bounded-wait probe; returns (status word, [plain wait gave up, abort-aware wait
    gave up]) -- (AEXP_ERR_DEVICE_TIMEOUT, [1, 1]) when the waits end as designed."""
    torch = _torch()
    ws = _alloc(lib().aexp_header_bytes(), device)
    ws.zero_()
    res = torch.zeros(2, dtype=torch.int32, device=device)
    _check(lib().aexp_probe_bounded_wait(int(polls), _ptr(res), _ptr(ws), ws.numel(), _stream(stream)),
           "aexp_probe_bounded_wait")
    return read_status(ws, stream), [int(v) for v in res.cpu()]


def swt_forward(img, wavelet="db4", stream=None):
    """One-level undecimated transform of an [ny][nx] complex64 image -> [4][ny][nx]."""
    torch = _torch()
    img = img.contiguous()
    ny, nx = img.shape
    coef = torch.empty((4, ny, nx), dtype=torch.complex64, device=img.device)
    w = WAVELETS[wavelet] if isinstance(wavelet, str) else int(wavelet)
    _check(lib().aexp_swt_forward(nx, ny, w, _ptr(img), _ptr(coef), _stream(stream)), "aexp_swt_forward")
    return coef


def _swt_ws(nx, ny, device):
    n = ctypes.c_size_t()
    _check(lib().aexp_swt_workspace_size(nx, ny, ctypes.byref(n)), "aexp_swt_workspace_size")
    return _alloc(n.value, device)


def swt_prox(img, tau: float, wavelet="db4", ws=None, stream=None):
    """W^H soft_detail(W img, tau) with the undecimated one-level transform."""
    torch = _torch()
    img = img.contiguous()
    ny, nx = img.shape
    ws = _swt_ws(nx, ny, img.device) if ws is None else ws
    out = torch.empty_like(img)
    w = WAVELETS[wavelet] if isinstance(wavelet, str) else int(wavelet)
    _check(lib().aexp_swt_prox(nx, ny, w, float(tau), _ptr(img), _ptr(out), _ptr(ws), ws.numel(), _stream(stream)),
           "aexp_swt_prox")
    return out


def swt_lambda(img, wavelet="db4", ws=None, stream=None):
    """lambda = sigma / 2 from the detail coefficients of W img (device float64 [1])."""
    torch = _torch()
    img = img.contiguous()
    ny, nx = img.shape
    ws = _swt_ws(nx, ny, img.device) if ws is None else ws
    out = torch.empty(1, dtype=torch.float64, device=img.device)
    w = WAVELETS[wavelet] if isinstance(wavelet, str) else int(wavelet)
    _check(lib().aexp_swt_lambda(nx, ny, w, _ptr(img), _ptr(out), _ptr(ws), ws.numel(), _stream(stream)),
           "aexp_swt_lambda")
    return out


def cgls_workspace_size(prob: Problem, opts: CReconOpts) -> int:
    n = ctypes.c_size_t()
    _check(lib().aexp_cgls_workspace_size(prob.c, ctypes.byref(opts), ctypes.byref(n)), "aexp_cgls_workspace_size")
    return n.value


def cgls_recon(prob: Problem, y, iters: int, opts: CReconOpts | None = None, ws=None, x_out=None, stream=None, **kw):
    """Least squares by CGLS from x = 0 (the paper's LS baseline); returns x [nr] complex64."""
    torch = _torch()
    opts = recon_opts(**kw) if opts is None else opts
    y = y.contiguous()
    if ws is None:
        ws = _alloc(cgls_workspace_size(prob, opts), y.device)
    if x_out is None:
        x_out = torch.empty(prob.nr, dtype=torch.complex64, device=y.device)
    _check(lib().cgls_recon(prob.c, _ptr(y), int(iters), ctypes.byref(opts), _ptr(x_out), _ptr(ws), ws.numel(),
                            _stream(stream)), "cgls_recon")
    return x_out


def lib_autotune_workspace_size(probs, opts: CReconOpts) -> int:
    """Bytes of workspace aexp_autotune needs for `probs` (covers every candidate layout)."""
    probs = list(probs) if isinstance(probs, (list, tuple)) else [probs]
    need = ctypes.c_size_t()
    _check(lib().aexp_autotune_workspace_size(_prob_array(probs), len(probs), ctypes.byref(opts), ctypes.byref(need)),
           "aexp_autotune_workspace_size")
    return need.value


def autotune(probs, opts: CReconOpts, ws=None, stream=None):
    """Time the candidate launch shapes (work-item granularity x kernel tiling) for `probs`
    (one problem: cs_recon's layout; several: cs_recon_batched's) and return
    (items_per_sm, tile_variant, median ms per A^H A application).  Synchronizes the stream;
    `opts` is not modified."""
    probs = list(probs) if isinstance(probs, (list, tuple)) else [probs]
    n = len(probs)
    probs_c = _prob_array(probs)
    if ws is None:
        ws = _alloc(lib_autotune_workspace_size(probs, opts), probs[0].device)
    best = ctypes.c_int()
    variant = ctypes.c_int()
    ms = ctypes.c_float()
    _check(lib().aexp_autotune(probs_c, n, ctypes.byref(opts), _ptr(ws), ws.numel(), _stream(stream),
                               ctypes.byref(best), ctypes.byref(variant), ctypes.byref(ms)), "aexp_autotune")
    return best.value, variant.value, ms.value


def power_lipschitz(prob: Problem, v0, n_power: int, ws=None, precision: int = FP32, stream=None):
    """L_f = 2 lambda_max(A^H A) by n_power power iterations from v0 (device float64 [1])."""
    torch = _torch()
    if ws is None:
        ws = recon_workspace(prob, recon_opts(precision=precision, levels=1))
    out = torch.empty(1, dtype=torch.float64, device=v0.device)
    _check(lib().aexp_power_lipschitz(prob.c, precision, _ptr(v0.contiguous()), int(n_power), _ptr(out),
                                      _ptr(ws), ws.numel(), _stream(stream)), "aexp_power_lipschitz")
    return out


def wavelet_workspace(nx, ny, wavelet, levels, device):
    n = ctypes.c_size_t()
    w = WAVELETS[wavelet] if isinstance(wavelet, str) else int(wavelet)
    _check(lib().aexp_wavelet_workspace_size(nx, ny, w, levels, ctypes.byref(n)), "aexp_wavelet_workspace_size")
    return _alloc(n.value, device)


def wavelet_prox(img, wavelet: str, levels: int, tau: float, ws=None, out=None, stream=None):
    """crop(W^H soft_detail(W pad img, tau)) for a complex64 [ny][nx] image."""
    torch = _torch()
    img = img.contiguous()
    ny, nx = img.shape
    ws = wavelet_workspace(nx, ny, wavelet, levels, img.device) if ws is None else ws
    out = torch.empty_like(img) if out is None else out
    _check(lib().aexp_wavelet_prox(nx, ny, WAVELETS[wavelet], levels, float(tau), _ptr(img), _ptr(out), _ptr(ws),
                                   ws.numel(), _stream(stream)), "aexp_wavelet_prox")
    return out


def wavelet_forward(img, wavelet: str, levels: int, ws=None, stream=None):
    """W pad img, Mallat layout, complex64 [npy][npx]."""
    torch = _torch()
    img = img.contiguous()
    ny, nx = img.shape
    q = 1 << levels
    npy, npx = -(-ny // q) * q, -(-nx // q) * q
    ws = wavelet_workspace(nx, ny, wavelet, levels, img.device) if ws is None else ws
    coef = torch.empty((npy, npx), dtype=torch.complex64, device=img.device)
    _check(lib().aexp_wavelet_forward(nx, ny, WAVELETS[wavelet], levels, _ptr(img), _ptr(coef), _ptr(ws),
                                      ws.numel(), _stream(stream)), "aexp_wavelet_forward")
    return coef


def read_status(ws, stream=None) -> int:
    s = ctypes.c_int()
    _check(lib().aexp_read_status(_ptr(ws), _stream(stream), ctypes.byref(s)), "aexp_read_status")
    return s.value
