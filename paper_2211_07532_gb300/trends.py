"""Simulation study of Sec. 2.2.2 (Figs. 4 and 5) on synthetic inputs.

NRMSE, against the noiseless image, of the paper's two reconstructions:
  LS -- conjugate gradients on the normal equations from x = 0, 20 iterations (Sec. 2.1);
  CS -- balanced FISTA with the one-level undecimated Daubechies-4 transform and
        lambda = sigma / 2 from the histogram of W A^H y, 100 iterations (Sec. 2.1,
        Supporting Information S1 and S2);
with the full encoding model ("Expanded": B0 and every field term up to 2nd order) or a
reduced one ("Partial": B0 and the 0th/1st-order terms only, Fig. 4; "NoB0": every field
term, no B0 map), against the acceleration factor R, the number of virtual coils and the SNR.

Data as in Sec. 2.2.2: complex white noise is added to the image, the full model with all
physical coils maps the noisy image to k-space, and the data are compressed to nv virtual coils
by principal components before the reconstruction.  SNR reading: the noise has
E|n(r)|^2 = sigma^2 with sigma = mean |x| over the object (|x| > 0.1 max |x|) / SNR.

Every step runs in the library (forward model, coil compression, CGLS, FISTA); this module only
draws the inputs and tabulates the errors.
"""

from __future__ import annotations

import math

import numpy as np

from . import synth

RS = (2.0, 3.0, 4.0, 5.0, 6.0)
COILS = (8, 16, 32)
SNRS = (20.0, 10.0, 5.0)
MODELS = ("Expanded", "Partial", "NoB0")


def trend_problem(n: int, r: float, nc: int = 32, eddy_scale: float = 0.1, seed_index: int = 0) -> dict:
    """Single-shot spiral at N^2 and acceleration R (N / (2R) turns, 1 us dwell), 2nd-order
    field (9 terms) with eddy terms of amplitude eddy_scale * U[1, 5] % plus B0 within
    +-150 Hz; phantom, coils and B0 are shared by every R (one slice, several protocols)."""
    nt = synth.ragged_protocol_nt(n, r)
    seed = synth.BASE_SEED + 1000 * 6 + 100 * seed_index + int(10 * r)
    gseed = synth.BASE_SEED + 1000 * 6 + 100 * seed_index + 99
    return synth.make_problem(n, nt=nt, nc=nc, order=2, dwell=1e-6, turns=n / (2.0 * r),
                              density_power=1.0, b0_hz=150.0, seed=seed, shared_geometry_seed=gseed,
                              eddy_scale=eddy_scale)


def object_sigma(x: np.ndarray, snr: float) -> float:
    a = np.abs(np.asarray(x))
    return float(np.mean(a[a > 0.1 * a.max()])) / snr


def model_terms(model: str):
    """(field terms kept, B0 kept) of a reconstruction model: "Partial" keeps the 0th- and
    1st-order terms (Fig. 4), "NoB0" every term but no B0 map."""
    if model not in MODELS:
        raise ValueError(model)
    return (4 if model == "Partial" else None), model != "NoB0"


def _model(ax, prob, model: str):
    if model == "Expanded":
        return prob
    if model == "Partial":
        return ax.Problem(prob.nx, prob.ny, prob.k[:4], prob.h[:4], prob.S, prob.omega, prob.t)
    if model == "NoB0":
        return ax.Problem(prob.nx, prob.ny, prob.k, prob.h, prob.S, None, None)
    raise ValueError(model)


def noisy_image(p: dict, snr: float, noise_seed: int) -> np.ndarray:
    """The phantom plus complex white noise with E|n(r)|^2 = sigma^2 (complex64)."""
    rng = np.random.default_rng(noise_seed)
    sigma = object_sigma(p["x_gt"], snr)
    return (p["x_gt"] + (sigma / math.sqrt(2.0)) * synth.random_image(rng, p["x_gt"].size)).astype(np.complex64)


def simulate(ax, p: dict, snr: float, noise_seed: int, device="cuda"):
    """(full-model Problem, k-space data of the noisy image [nc][nt], noiseless image)."""
    import torch
    prob = ax.Problem.from_arrays(p, device=device)
    noisy = noisy_image(p, snr, noise_seed)
    ws = ax.workspace(prob, ax.FP32)
    ax.prepare(prob, ws, ax.FP32)
    y = ax.a_exp_forward(prob, torch.as_tensor(noisy, device=device), ws)
    torch.cuda.synchronize()
    if ax.read_status(ws) != 0:
        raise RuntimeError("forward model reported a device error")
    return prob, y, torch.as_tensor(p["x_gt"], device=device)


def reconstruct(ax, prob, y, method: str, precision, cs_iters: int = 100, ls_iters: int = 20):
    import torch
    if method == "LS":
        x = ax.cgls_recon(prob, y, ls_iters, opts=ax.recon_opts(precision=precision))
    elif method == "CS":
        lam = torch.zeros(1, dtype=torch.float64, device=y.device)
        o = ax.recon_opts(precision=precision, wavelet="db4", undecimated=True, lambda_rule=ax.LAMBDA_RAYLEIGH,
                          lambda_out=lam)
        x, _ = ax.cs_recon(prob, y, 0.0, cs_iters, opts=o)
    else:
        raise ValueError(method)
    torch.cuda.synchronize()
    return x


def nrmse(x, x_gt) -> float:
    import torch
    return float(torch.linalg.vector_norm(x - x_gt) / torch.linalg.vector_norm(x_gt))


def run(ax, n: int = 148, rs=RS, coils=COILS, snrs=SNRS, models=MODELS, r_for_snr: float = 4.0,
        vc_default: int = 16, snr_default: float = 20.0, eddy_scale: float = 0.1, precision=None,
        cs_iters: int = 100, device="cuda") -> dict:
    """The three panels: fig4 [model][method][R] (SNR 20, 16 virtual coils), fig5a
    [coils][method][R] (Expanded, SNR 20), fig5b [coils][method][SNR] (Expanded, R = 4)."""
    precision = ax.FP32 if precision is None else precision
    cache = {}

    def data(r, snr):
        key = (r, snr)
        if key not in cache:
            p = trend_problem(n, r, eddy_scale=eddy_scale)
            cache[key] = simulate(ax, p, snr, noise_seed=int(1000 * r + snr), device=device)
        return cache[key]

    def point(r, snr, nv, model, method):
        prob, y, x_gt = data(r, snr)
        if nv < prob.nc:
            prob_v, y_v, _ = ax.coil_compress(prob, y, nv)
        else:
            prob_v, y_v = prob, y
        return nrmse(reconstruct(ax, _model(ax, prob_v, model), y_v, method, precision, cs_iters), x_gt)

    out = {"n": n, "eddy_scale": eddy_scale, "fig4": {}, "fig5a": {}, "fig5b": {}}
    for model in models:
        out["fig4"][model] = {m: [point(r, snr_default, vc_default, model, m) for r in rs] for m in ("LS", "CS")}
    for nv in coils:
        out["fig5a"][nv] = {m: [point(r, snr_default, nv, "Expanded", m) for r in rs] for m in ("LS", "CS")}
        out["fig5b"][nv] = {m: [point(r_for_snr, s, nv, "Expanded", m) for s in snrs] for m in ("LS", "CS")}
    out.update(rs=list(rs), snrs=list(snrs), coils=list(coils), r_for_snr=r_for_snr)
    return out
