"""Differentiable unrolled FISTA on Eq. (1) (Sec. 5: unrolled CS as future work).

``unrolled_fista(prob_arrays, y, x0, lam, k, iters, lipschitz, ...)`` returns x_K after K
FISTA steps and back-propagates to the start image x0, the regularisation weight lam and
the field coefficients k_l(t) (L_f is held fixed).  The forward pass calls the library's
``aexp_fista_step`` K times and keeps the per-step checkpoints z_k; the backward pass calls
``aexp_fista_step_vjp`` for k = K..1.  This module only marshals arguments: every
arithmetic step runs in the library's CUDA kernels.
"""

from __future__ import annotations

import ctypes
import math

import torch

from . import FP32, WAVELETS, Problem, _alloc, _check, _ptr, _stream, lib, prepare, recon_opts


def fista_betas(iters: int):
    """Momentum weights b_k = (t_k - 1)/t_{k+1}, t_1 = 1, t_{k+1} = (1 + sqrt(1 + 4 t_k^2))/2 (FP64)."""
    b = [0.0] * (iters + 2)
    t = 1.0
    for k in range(1, iters + 1):
        tn = (1.0 + math.sqrt(1.0 + 4.0 * t * t)) / 2.0
        b[k] = (t - 1.0) / tn
        t = tn
    return b


def unroll_workspace(prob: Problem, opts):
    n = ctypes.c_size_t()
    _check(lib().aexp_unroll_workspace_size(prob.c, ctypes.byref(opts), ctypes.byref(n)), "aexp_unroll_workspace_size")
    return _alloc(n.value, prob.device)


class UnrolledFISTA(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x0, lam, k, h, S, omega, t, y, nx, ny, iters, lipschitz, wavelet, levels, precision):
        prob = Problem(nx, ny, k.detach().contiguous(), h, S, omega, t)
        opts = recon_opts(precision=precision, wavelet=wavelet, levels=levels, lipschitz=lipschitz)
        ws = unroll_workspace(prob, opts)
        prepare(prob, ws, precision)
        betas = fista_betas(iters)
        lam_f = float(lam)
        y = y.contiguous()
        x_prev = x0.detach().contiguous()
        z = x_prev.clone()
        zs = [z]
        for kk in range(1, iters + 1):
            x_new = torch.empty_like(z)
            z_new = torch.empty_like(z)
            _check(lib().aexp_fista_step(prob.c, ctypes.byref(opts), _ptr(y), lam_f, float(lipschitz), _ptr(z),
                                         _ptr(x_prev), betas[kk], _ptr(x_new), _ptr(z_new), _ptr(ws), ws.numel(),
                                         _stream()), "aexp_fista_step")
            x_prev, z = x_new, z_new
            zs.append(z)
        ctx.prob, ctx.opts, ctx.ws, ctx.zs, ctx.betas = prob, opts, ws, zs[:iters], betas
        ctx.lam, ctx.L, ctx.y, ctx.iters = lam_f, float(lipschitz), y, iters
        ctx.lam_meta = (lam.dtype, lam.device)
        return x_prev

    @staticmethod
    def backward(ctx, gx):
        prob, opts, ws, zs, b = ctx.prob, ctx.opts, ctx.ws, ctx.zs, ctx.betas
        gx = gx.contiguous()
        kbar = torch.zeros_like(prob.k)
        lambar = torch.zeros(1, dtype=torch.float64, device=gx.device)
        zbar_next, zbar_next2 = None, None
        for kk in range(ctx.iters, 0, -1):
            zbar = torch.empty_like(gx)
            _check(lib().aexp_fista_step_vjp(prob.c, ctypes.byref(opts), _ptr(ctx.y), ctx.lam, ctx.L, _ptr(zs[kk - 1]),
                                             b[kk], b[kk + 1], _ptr(gx) if kk == ctx.iters else None,
                                             _ptr(zbar_next), _ptr(zbar_next2), _ptr(zbar), _ptr(kbar),
                                             _ptr(lambar), _ptr(ws), ws.numel(), _stream()), "aexp_fista_step_vjp")
            zbar_next2, zbar_next = zbar_next, zbar
        x0bar = zbar_next if zbar_next is not None else gx  # b_1 = 0: the start image's cotangent is zbar_1
        dt, dev = ctx.lam_meta
        return (x0bar, lambar.reshape(()).to(device=dev, dtype=dt), kbar, None, None, None, None, None, None, None, None, None, None,
                None, None)


def unrolled_fista(d: dict, y, x0, lam, k, iters: int, lipschitz: float, wavelet: str = "db4", levels: int = 4,
                   precision: int = FP32, device="cuda", with_b0: bool = True):
    """x_K of K FISTA steps on the problem `d` (numpy arrays: h, S, omega, t; `k` is the
    differentiable torch tensor [nl][nt]); differentiable in x0, lam (0-d tensor) and k."""
    dev = torch.device(device)
    h = torch.as_tensor(d["h"], dtype=torch.float32, device=dev)
    S = torch.as_tensor(d["S"], dtype=torch.complex64, device=dev)
    om = torch.as_tensor(d["omega"], dtype=torch.float32, device=dev) if with_b0 else None
    t = torch.as_tensor(d["t"], dtype=torch.float32, device=dev) if with_b0 else None
    return UnrolledFISTA.apply(x0, lam, k, h, S, om, t, y, d["nx"], d["ny"], iters, lipschitz,
                               WAVELETS[wavelet], levels, precision)
