// Solver around the operator: Lipschitz estimate by power iteration and FISTA on Eq. (1)
// (Sec. 2.1: CS reconstructions with balanced FISTA; with an orthonormal W the prox
// step below is the exact one).  FP64 on the device is used only for the norm and
// inner-product reductions and the Lipschitz scalar; the FISTA momentum scalars are
// FP64 host values (they do not depend on data).
#include <math.h>

#include <algorithm>

#include "aexp_internal.cuh"
#include "reduce_f64.cuh"

namespace aexp {

namespace {

// mu = Re <v, w>, nrm2 = ||w||^2 in FP64 (each product of two floats is exact in FP64), one
// deterministic grid reduction.
__global__ void __launch_bounds__(kDotThreads) dot_norm_kernel(const float2 *__restrict__ v,
                                                               const float2 *__restrict__ w, int n, double *part,
                                                               unsigned *ticket, double *mu, double *nrm2) {
    double a = 0.0, b = 0.0;
    for (int i = blockIdx.x * kDotThreads + threadIdx.x; i < n; i += gridDim.x * kDotThreads) {
        const float2 wv = w[i];
        if (v) {
            const float2 vv = v[i];
            a = fma((double)vv.x, (double)wv.x, a);
            a = fma((double)vv.y, (double)wv.y, a);
        }
        b = fma((double)wv.x, (double)wv.x, b);
        b = fma((double)wv.y, (double)wv.y, b);
    }
    if (grid_sum2(a, b, blockIdx.x, gridDim.x, part, ticket)) {
        if (mu) *mu = a;
        *nrm2 = b;
    }
}

__global__ void scale_inv_sqrt_kernel(const float2 *w, float2 *v, int n, const double *nrm2) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double nn = *nrm2;
    float s = nn > 0.0 ? (float)(1.0 / sqrt(nn)) : 0.f;
    float2 a = w[i];
    v[i] = make_float2(a.x * s, a.y * s);
}

// L_f = 2 mu; records AEXP_ERR_NONFINITE if it is not a positive finite number.
__global__ void finalize_lipschitz_kernel(WsHeader *hdr, double *out) {
    double L = 2.0 * hdr->mu;
    if (!(L > 0.0) || !isfinite(L)) {
        atomicCAS(&hdr->status, 0, AEXP_ERR_NONFINITE);
        L = 1.0;
    }
    hdr->lipschitz = L;
    if (out) *out = L;
}

__global__ void set_lipschitz_kernel(WsHeader *hdr, double L, double *out) {
    hdr->lipschitz = L;
    if (out) *out = L;
}

#define CK(x)                               \
    do {                                    \
        cudaError_t e__ = (x);              \
        if (e__ != cudaSuccess) return e__; \
    } while (0)

}  // namespace

cudaError_t dot_norm_f64(const float2 *v, const float2 *w, int n, double *mu, double *nrm2, WsHeader *hdr,
                         cudaStream_t st) {
    const int blocks = std::max(1, std::min(kRedMaxBlocks, cdiv(n, 2 * kDotThreads)));
    dot_norm_kernel<<<blocks, kDotThreads, 0, st>>>(v, w, n, hdr->red_part, &hdr->red_ticket, mu, nrm2);
    return cudaGetLastError();
}

cudaError_t scale_inv_sqrt(const float2 *w, float2 *v, int n, const double *nrm2, cudaStream_t st) {
    scale_inv_sqrt_kernel<<<cdiv(n, 256), 256, 0, st>>>(w, v, n, nrm2);
    return cudaGetLastError();
}

// w = A^H A v (v in natural order); uses the operator workspace only.
cudaError_t normal_apply(const OpLayout &L, char *ws, const float2 *v, float2 *w, cudaStream_t st) {
    CK(op_apply_forward(L, v, ws, st));
    CK(op_residual_adjoint(L, ws, nullptr, st));
    CK(op_adjoint_reduce(L, ws, w, st));
    return cudaSuccess;
}

// Power iteration: v <- v0/||v0||; repeat n: w = A^H A v, mu = Re<v,w>, v = w/||w||.
// L_f = 2 mu of the last iteration, into the header (and *out when given).
cudaError_t power_iteration(const OpLayout &L, char *ws, const float2 *v0, float2 *v, float2 *w, int n_power,
                            double *out, cudaStream_t st) {
    WsHeader *hdr = (WsHeader *)(ws + L.off_hdr);
    CK(dot_norm_f64(nullptr, v0, L.nr, nullptr, &hdr->nrm2, hdr, st));
    CK(scale_inv_sqrt(v0, v, L.nr, &hdr->nrm2, st));
    for (int i = 0; i < n_power; ++i) {
        CK(normal_apply(L, ws, v, w, st));
        CK(dot_norm_f64(v, w, L.nr, &hdr->mu, &hdr->nrm2, hdr, st));
        CK(scale_inv_sqrt(w, v, L.nr, &hdr->nrm2, st));
    }
    finalize_lipschitz_kernel<<<1, 1, 0, st>>>(hdr, out);
    return cudaGetLastError();
}

cudaError_t set_lipschitz(const OpLayout &L, char *ws, double value, double *out, cudaStream_t st) {
    set_lipschitz_kernel<<<1, 1, 0, st>>>((WsHeader *)(ws + L.off_hdr), value, out);
    return cudaGetLastError();
}

// The whole reconstruction, issued on `st` (capturable).
cudaError_t recon_issue(const aexp_problem *p, const RecLayout &R, const aexp_recon_opts *o, const float2 *y,
                        float lam, int iters, float2 *x_out, double *lip_out, char *ws, cudaStream_t st) {
    const OpLayout &L = R.op;
    WsHeader *hdr = (WsHeader *)(ws + L.off_hdr);
    float2 *ymeas = (float2 *)(ws + R.off_ymeas);
    float2 *xa = (float2 *)(ws + R.off_xa);
    float2 *xb = (float2 *)(ws + R.off_xb);
    float2 *z = (float2 *)(ws + R.off_z);
    float2 *v = (float2 *)(ws + R.off_v);
    float2 *w = (float2 *)(ws + R.off_w);
    char *wws = ws + R.off_wave;
    const size_t img_bytes = sizeof(float2) * (size_t)L.nr;

    CK(op_prepare(p, L, ws, st));
    CK(op_transpose_y(L, y, ymeas, st));

    // A^H y, the zero-filled reconstruction: the power iteration's default start and the
    // input of the paper's lambda rule
    const bool rayleigh = o->undecimated && o->lambda_rule == AEXP_LAMBDA_RAYLEIGH;
    const bool need_ahy = rayleigh || (!(o->lipschitz > 0.0) && !o->power_init);
    if (need_ahy) {
        CK(op_apply_adjoint(L, ymeas, ws, st));
        CK(op_adjoint_reduce(L, ws, w, st));
    }
    char *swt_aux = o->undecimated ? ws + R.off_swtaux : nullptr;
    float2 *swt_c = o->undecimated ? (float2 *)(ws + R.off_swt) : nullptr;
    if (rayleigh) {
        CK(swt_analysis(o->wavelet, w, swt_c, L.nx, L.ny, -1.f, nullptr, nullptr, st));
        CK(swt_rayleigh_lambda(swt_c, L.nx, L.ny, swt_aux, o->lambda_out, st));
    } else if (o->undecimated) {
        CK(swt_set_lambda(swt_aux, (double)lam, o->lambda_out, st));
    }

    if (o->lipschitz > 0.0) {
        CK(set_lipschitz(L, ws, o->lipschitz, lip_out, st));
    } else {
        const float2 *v0 = o->power_init ? (const float2 *)o->power_init : w;
        CK(power_iteration(L, ws, v0, v, w, o->n_power, lip_out, st));
    }

    // FISTA (Beck-Teboulle): x_0 given or 0, z_1 = x_0, t_1 = 1.
    float2 *x_prev = xa, *x_new = xb;
    if (o->x0)
        CK(cudaMemcpyAsync(x_prev, o->x0, img_bytes, cudaMemcpyDeviceToDevice, st));
    else
        CK(cudaMemsetAsync(x_prev, 0, img_bytes, st));
    CK(cudaMemcpyAsync(z, x_prev, img_bytes, cudaMemcpyDeviceToDevice, st));
    double t = 1.0;
    for (int k = 0; k < iters; ++k) {
        // v = z - (2/L_f) A^H (A z - y)
        CK(op_apply_forward(L, z, ws, st));
        CK(op_residual_adjoint(L, ws, ymeas, st));
        CK(op_adjoint_reduce_step(L, ws, z, v, st));
        // x_k = crop W^H soft(W pad v, lam / L_f);  z_{k+1} = x_k + beta_k (x_k - x_{k-1})
        double t_next = (1.0 + sqrt(1.0 + 4.0 * t * t)) / 2.0;
        double beta = (t - 1.0) / t_next;
        if (o->undecimated) {
            // x_k = W^H soft(W v, lambda / L_f) with the tight frame ("balanced" FISTA)
            CK(swt_analysis(o->wavelet, v, swt_c, L.nx, L.ny, -1.f, swt_lambda_slot(swt_aux), &hdr->lipschitz, st));
            CK(swt_synthesis(o->wavelet, swt_c, x_new, L.nx, L.ny, 1, beta, x_prev, z, st));
        } else {
            CK(wave_prox(R.wv, v, wws, lam, &hdr->lipschitz, x_new, 1, beta, x_prev, z, st));
        }
        t = t_next;
        float2 *tmp = x_prev;
        x_prev = x_new;
        x_new = tmp;
    }
    CK(cudaMemcpyAsync(x_out, x_prev, img_bytes, cudaMemcpyDeviceToDevice, st));
    return cudaSuccess;
}

}  // namespace aexp
