// Differentiation through unrolled FISTA (FP32 CUDA cores).
//
// One step of Eq. (1)'s FISTA, with L_f fixed:
//   r_k = A z_k - y,  v_k = z_k - (2/L) A^H r_k,  x_k = P(v_k) = crop W^H S_tau W pad v_k,
//   z_{k+1} = (1 + b_k) x_k - b_k x_{k-1}.
// Its vector-Jacobian product for a real loss (cotangent = dLoss/dRe + i dLoss/dIm):
//   xbar_k = (1 + b_k) zbar_{k+1} - b_{k+1} zbar_{k+2} (+ upstream cotangent of x_k),
//   vbar_k = crop W^H S'^T W pad xbar_k          (S' = soft-threshold Jacobian at W pad v_k),
//   lambar += (1/L) sum_j Re(conj(g_j) dS_j/dtau),
//   zbar_k = vbar_k - (2/L) A^H A vbar_k,
//   kbar_l(t) += -(2/L) Re sum_r h_l(r) [ -i E z_k(r) sum_c conj(u_c(t)) S_c(r)
//                                         + i conj(E) conj(vbar_k(r)) sum_c conj(S_c(r)) r_c(t) ],
// with u = A vbar_k and E = E(t, r).  The last line is one pass of the grad_k kernel: a
// block owns 128 samples (u_c(t), r_c(t) and the phase coefficients in registers) and a run
// of 8x8 voxel tiles staged by bulk TMA copies, exactly like the forward operator kernel.
#include <math.h>

#include <algorithm>

#include "aexp_internal.cuh"
#include "reduce_f64.cuh"

namespace aexp {

namespace {

constexpr int kGradThreads = 128;
constexpr float kTwoPi = 6.283185307179586f;

template <int CB, int LP>
__global__ void __launch_bounds__(kGradThreads, 2)
    grad_k_kernel(const float *__restrict__ khi_l, const float *__restrict__ f0, const float *__restrict__ dh,
                  const float *__restrict__ hp, const float2 *__restrict__ Sp, const float2 *__restrict__ zq,
                  const float2 *__restrict__ gq, const float2 *__restrict__ ut, const float2 *__restrict__ rt,
                  float *__restrict__ gpart, int ntp, int ntiles, int tiles_per_split, int *status) {
    constexpr unsigned DH_BYTES = kTileVox * LP * 4;
    constexpr unsigned S_BYTES = kTileVox * CB * 8;
    constexpr unsigned V_BYTES = kTileVox * 8;
    constexpr unsigned STAGE = 2 * DH_BYTES + S_BYTES + 2 * V_BYTES;  // dh | hp | S | z | vbar
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar[2];

    const int tid = threadIdx.x;
    const int split = blockIdx.y;
    const int tile0 = split * tiles_per_split;
    const int ntl = min(ntiles, tile0 + tiles_per_split) - tile0;
    const int t = blockIdx.x * kGradThreads + tid;

    float kh[LP], acc[LP];
    float ur[CB], ui[CB], rr[CB], ri[CB];
#pragma unroll
    for (int l = 0; l < LP; ++l) {
        kh[l] = khi_l[(size_t)l * ntp + t];
        acc[l] = 0.f;
    }
#pragma unroll
    for (int q = 0; q < CB / 2; ++q) {
        float4 a = reinterpret_cast<const float4 *>(ut + (size_t)t * CB)[q];
        float4 b = reinterpret_cast<const float4 *>(rt + (size_t)t * CB)[q];
        ur[2 * q] = a.x;
        ui[2 * q] = a.y;
        ur[2 * q + 1] = a.z;
        ui[2 * q + 1] = a.w;
        rr[2 * q] = b.x;
        ri[2 * q] = b.y;
        rr[2 * q + 1] = b.z;
        ri[2 * q + 1] = b.w;
    }

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();
    auto issue = [&](int i) {
        const int buf = i & 1;
        unsigned char *dst = smem + buf * STAGE;
        const size_t tile = (size_t)(tile0 + i);
        mbar_arrive_expect_tx(&bar[buf], STAGE);
        bulk_g2s(dst, dh + tile * kTileVox * LP, DH_BYTES, &bar[buf]);
        bulk_g2s(dst + DH_BYTES, hp + tile * kTileVox * LP, DH_BYTES, &bar[buf]);
        bulk_g2s(dst + 2 * DH_BYTES, Sp + tile * kTileVox * CB, S_BYTES, &bar[buf]);
        bulk_g2s(dst + 2 * DH_BYTES + S_BYTES, zq + tile * kTileVox, V_BYTES, &bar[buf]);
        bulk_g2s(dst + 2 * DH_BYTES + S_BYTES + V_BYTES, gq + tile * kTileVox, V_BYTES, &bar[buf]);
    };
    if (tid == 0) {
        if (ntl > 0) issue(0);
        if (ntl > 1) issue(1);
    }

    for (int i = 0; i < ntl; ++i) {
        const int buf = i & 1;
        bool ok = mbar_wait_bounded(&bar[buf], (i >> 1) & 1, status);
        if (__syncthreads_or(!ok)) {
            if (tid == 0)
                for (int k = i; k < min(ntl, i + 2); ++k) mbar_wait_bounded(&bar[k & 1], (k >> 1) & 1, status);
            __syncthreads();
            return;
        }
        const unsigned char *stg = smem + buf * STAGE;
        const float4 *sdh = reinterpret_cast<const float4 *>(stg);
        const float4 *shp = reinterpret_cast<const float4 *>(stg + DH_BYTES);
        const float4 *sS = reinterpret_cast<const float4 *>(stg + 2 * DH_BYTES);
        const float2 *sz = reinterpret_cast<const float2 *>(stg + 2 * DH_BYTES + S_BYTES);
        const float2 *sg = reinterpret_cast<const float2 *>(stg + 2 * DH_BYTES + S_BYTES + V_BYTES);
        const float fr = f0[(size_t)(tile0 + i) * ntp + t];
#pragma unroll 1
        for (int v = 0; v < kTileVox; ++v) {
            float p0 = fr, p1 = 0.f;
#pragma unroll
            for (int q = 0; q < LP / 4; ++q) {
                float4 d = sdh[v * (LP / 4) + q];
                p0 = fmaf(kh[4 * q], d.x, p0);
                p1 = fmaf(kh[4 * q + 1], d.y, p1);
                p0 = fmaf(kh[4 * q + 2], d.z, p0);
                p1 = fmaf(kh[4 * q + 3], d.w, p1);
            }
            float ph = p0 + p1;
            ph = ph - rintf(ph);
            float s, c;
            __sincosf(ph * kTwoPi, &s, &c);
            // a = sum_c conj(u_c) S_c,  b = sum_c conj(S_c) r_c
            float ar = 0.f, ai = 0.f, br = 0.f, bi = 0.f;
#pragma unroll
            for (int q = 0; q < CB / 2; ++q) {
                float4 S2 = sS[v * (CB / 2) + q];
                ar = fmaf(ur[2 * q], S2.x, ar);
                ar = fmaf(ui[2 * q], S2.y, ar);
                ai = fmaf(ur[2 * q], S2.y, ai);
                ai = fmaf(-ui[2 * q], S2.x, ai);
                br = fmaf(S2.x, rr[2 * q], br);
                br = fmaf(S2.y, ri[2 * q], br);
                bi = fmaf(S2.x, ri[2 * q], bi);
                bi = fmaf(-S2.y, rr[2 * q], bi);
                ar = fmaf(ur[2 * q + 1], S2.z, ar);
                ar = fmaf(ui[2 * q + 1], S2.w, ar);
                ai = fmaf(ur[2 * q + 1], S2.w, ai);
                ai = fmaf(-ui[2 * q + 1], S2.z, ai);
                br = fmaf(S2.z, rr[2 * q + 1], br);
                br = fmaf(S2.w, ri[2 * q + 1], br);
                bi = fmaf(S2.z, ri[2 * q + 1], bi);
                bi = fmaf(-S2.w, rr[2 * q + 1], bi);
            }
            // E = c - i s; Ez, Eg;  Re T = Im(Ez a) - Im(conj(Eg) b)
            const float2 zv = sz[v], gv = sg[v];
            const float ezr = c * zv.x + s * zv.y, ezi = c * zv.y - s * zv.x;
            const float egr = c * gv.x + s * gv.y, egi = c * gv.y - s * gv.x;
            const float reT = (ezr * ai + ezi * ar) - (egr * bi - egi * br);
#pragma unroll
            for (int q = 0; q < LP / 4; ++q) {
                float4 hv = shp[v * (LP / 4) + q];
                acc[4 * q] = fmaf(reT, hv.x, acc[4 * q]);
                acc[4 * q + 1] = fmaf(reT, hv.y, acc[4 * q + 1]);
                acc[4 * q + 2] = fmaf(reT, hv.z, acc[4 * q + 2]);
                acc[4 * q + 3] = fmaf(reT, hv.w, acc[4 * q + 3]);
            }
        }
        __syncthreads();
        if (tid == 0 && i + 2 < ntl) issue(i + 2);
    }
#pragma unroll
    for (int l = 0; l < LP; ++l) gpart[((size_t)split * LP + l) * ntp + t] = acc[l];
}

// kbar[l][t] += -(2/L) * sum over splits (l < nl, t < nt)
__global__ void grad_k_reduce_kernel(const float *gpart, int splits, int LP, int ntp, int nl, int nt,
                                     const WsHeader *hdr, float *kbar) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)nl * nt) return;
    const int l = (int)(i / nt), t = (int)(i % nt);
    float s = 0.f;
    for (int k = 0; k < splits; ++k) s += gpart[((size_t)k * LP + l) * ntp + t];
    kbar[i] += (float)(-2.0 / hdr->lipschitz) * s;
}

// natural order [nx*ny] -> tile order [nr_pad] (zero for padded voxels)
__global__ void to_tile_order_kernel(const float2 *x, int nx, int ny, int ntx, int nr_pad, float2 *xq) {
    const int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= nr_pad) return;
    const int tile = p / kTileVox, v = p % kTileVox;
    const int ix = (tile % ntx) * kTileSide + v % kTileSide, iy = (tile / ntx) * kTileSide + v / kTileSide;
    xq[p] = (ix < nx && iy < ny) ? x[(size_t)iy * nx + ix] : make_float2(0.f, 0.f);
}

// out = a * X + b * Y + Z over n complex values (null operands are zero)
__global__ void combine_kernel(int n, float a, const float2 *X, float b, const float2 *Y, const float2 *Z,
                               float2 *out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float2 o = make_float2(0.f, 0.f);
    if (X) {
        o.x += a * X[i].x;
        o.y += a * X[i].y;
    }
    if (Y) {
        o.x += b * Y[i].x;
        o.y += b * Y[i].y;
    }
    if (Z) {
        o.x += Z[i].x;
        o.y += Z[i].y;
    }
    out[i] = o;
}

// Soft-threshold VJP on the detail coefficients of a Mallat pyramid (npy x npx, J levels):
// gw <- (1 - tau/r) gw + (tau/r^3) w Re(conj(w) gw) where |w| > tau, 0 where |w| <= tau;
// the low-pass block is left as is.  lambar += (1/L) sum -Re(conj(gw) w)/r (FP64, one
// deterministic grid reduction through the header's partials and ticket).
__global__ void __launch_bounds__(kDotThreads) soft_vjp_kernel(const float2 *w, float2 *gw, int npx, int npy,
                                                               int levels, float lam, WsHeader *hdr, double *lambar) {
    const double L = hdr->lipschitz;
    const float tau = (float)((double)lam / L);
    const int lpx = npx >> levels, lpy = npy >> levels;
    double acc = 0.0, unused = 0.0;
    for (int i = blockIdx.x * kDotThreads + threadIdx.x; i < npx * npy; i += gridDim.x * kDotThreads) {
        const int iy = i / npx, ix = i % npx;
        if (iy < lpy && ix < lpx) continue;  // low-pass block: weight 0
        const float2 wv = w[i], g = gw[i];
        const float r2 = wv.x * wv.x + wv.y * wv.y;
        float2 o = make_float2(0.f, 0.f);
        if (r2 > tau * tau) {
            const float r = sqrtf(r2);
            const float a = 1.f - tau / r;
            const float proj = wv.x * g.x + wv.y * g.y;  // Re(conj(w) g)
            const float bcoef = tau * proj / (r2 * r);
            o = make_float2(a * g.x + bcoef * wv.x, a * g.y + bcoef * wv.y);
            acc += -(double)proj / (double)r;
        }
        gw[i] = o;
    }
    if (grid_sum2(acc, unused, blockIdx.x, gridDim.x, hdr->red_part, &hdr->red_ticket) && lambar)
        *lambar += acc / L;
}

template <int CB, int LP>
cudaError_t launch_grad(const OpLayout &L, const RecLayout &R, char *ws, cudaStream_t st) {
    constexpr unsigned STAGE = 2 * kTileVox * LP * 4 + kTileVox * CB * 8 + 2 * kTileVox * 8;
    auto kern = grad_k_kernel<CB, LP>;
    {  // always opted in: the static barriers count against the 48 KB default too
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * STAGE);
        if (e != cudaSuccess) return e;
    }
    WsHeader *hdr = (WsHeader *)(ws + L.off_hdr);
    kern<<<dim3(L.ntp / kGradThreads, R.grad_splits), kGradThreads, 2 * STAGE, st>>>(
        (const float *)(ws + L.off_khi_l), (const float *)(ws + L.off_f0), (const float *)(ws + L.off_dh),
        (const float *)(ws + L.off_hp), (const float2 *)(ws + L.off_S), (const float2 *)(ws + R.off_zq),
        (const float2 *)(ws + R.off_gq), (const float2 *)(ws + L.off_yt), (const float2 *)(ws + R.off_rk),
        (float *)(ws + R.off_gpart), L.ntp, L.ntiles, R.grad_tiles_per_split, &hdr->status);
    return cudaGetLastError();
}

#define AEXP_GRAD_LP(CBV)                                                  \
    switch (L.LP) {                                                        \
        case 4: return launch_grad<CBV, 4>(L, R, ws, st);                  \
        case 8: return launch_grad<CBV, 8>(L, R, ws, st);                  \
        case 12: return launch_grad<CBV, 12>(L, R, ws, st);                \
        case 20: return launch_grad<CBV, 20>(L, R, ws, st);                \
        default: return launch_grad<CBV, 32>(L, R, ws, st);                \
    }

cudaError_t grad_k_launch(const RecLayout &R, char *ws, cudaStream_t st) {
    const OpLayout &L = R.op;
    switch (L.CB) {
        case 4: AEXP_GRAD_LP(4)
        case 8: AEXP_GRAD_LP(8)
        case 16: AEXP_GRAD_LP(16)
        case 20: AEXP_GRAD_LP(20)
        default: AEXP_GRAD_LP(32)
    }
}

#define CK(x)                               \
    do {                                    \
        cudaError_t e__ = (x);              \
        if (e__ != cudaSuccess) return e__; \
    } while (0)

}  // namespace

cudaError_t unroll_step(const RecLayout &R, const float2 *y, float lam, double lipschitz, const float2 *z,
                        const float2 *x_prev, double beta, float2 *x_out, float2 *z_out, char *ws, cudaStream_t st) {
    const OpLayout &L = R.op;
    float2 *ymeas = (float2 *)(ws + R.off_ymeas);
    float2 *rt = (float2 *)(ws + L.off_yt);
    float2 *v = (float2 *)(ws + R.off_v);
    WsHeader *hdr = (WsHeader *)(ws + L.off_hdr);
    CK(set_lipschitz(L, ws, lipschitz, nullptr, st));
    CK(op_transpose_y(L, y, ymeas, st));
    CK(op_apply_forward(L, z, ws, st));
    CK(op_reduce_forward_residual(L, ws, ymeas, rt, st));
    CK(op_apply_adjoint(L, rt, ws, st));
    CK(op_adjoint_reduce_step(L, ws, z, v, st));
    CK(wave_prox(R.wv, v, ws + R.off_wave, lam, &hdr->lipschitz, x_out, 1, beta, x_prev, z_out, st));
    return cudaSuccess;
}

cudaError_t unroll_step_vjp(const RecLayout &R, const float2 *y, float lam, double lipschitz, const float2 *z,
                            double beta, double beta_next, const float2 *xbar_in, const float2 *zbar_next,
                            const float2 *zbar_next2, float2 *zbar_out, float *kbar, double *lambar, char *ws,
                            cudaStream_t st) {
    const OpLayout &L = R.op;
    const int T = 256;
    float2 *ymeas = (float2 *)(ws + R.off_ymeas);
    float2 *ut = (float2 *)(ws + L.off_yt);  // u = A vbar, sample-major
    float2 *rk = (float2 *)(ws + R.off_rk);  // r_k = A z_k - y, sample-major
    float2 *v = (float2 *)(ws + R.off_v);
    float2 *xbar = (float2 *)(ws + R.off_xbar);
    float2 *vbar = (float2 *)(ws + R.off_vbar);
    float2 *pyr_w = (float2 *)(ws + R.off_wave + R.wv.off_pyr);
    float2 *pyr_g = (float2 *)(ws + R.off_wave2 + R.wv.off_pyr);
    WsHeader *hdr = (WsHeader *)(ws + L.off_hdr);

    CK(set_lipschitz(L, ws, lipschitz, nullptr, st));
    CK(op_transpose_y(L, y, ymeas, st));
    // xbar_k = (1 + b_k) zbar_{k+1} - b_{k+1} zbar_{k+2} + upstream
    combine_kernel<<<cdiv(L.nr, T), T, 0, st>>>(L.nr, (float)(1.0 + beta), zbar_next, (float)(-beta_next), zbar_next2,
                                               xbar_in, xbar);
    // r_k and v_k from the checkpoint z_k
    CK(op_apply_forward(L, z, ws, st));
    CK(op_reduce_forward_residual(L, ws, ymeas, rk, st));
    CK(op_apply_adjoint(L, rk, ws, st));
    CK(op_adjoint_reduce_step(L, ws, z, v, st));
    // vbar_k = crop W^H S'^T W pad xbar_k, lambar += taubar / L
    CK(wave_forward(R.wv, v, ws + R.off_wave, 0.f, nullptr, 0, st));
    CK(wave_forward(R.wv, xbar, ws + R.off_wave2, 0.f, nullptr, 0, st));
    {
        const int n = R.wv.npx * R.wv.npy;
        const int blocks = std::max(1, std::min(kRedMaxBlocks, cdiv(n, 2 * kDotThreads)));
        soft_vjp_kernel<<<blocks, kDotThreads, 0, st>>>(pyr_w, pyr_g, R.wv.npx, R.wv.npy, R.wv.levels, lam, hdr,
                                                        lambar);
    }
    CK(wave_inverse(R.wv, ws + R.off_wave2, vbar, 0, 0.0, nullptr, nullptr, st));
    // u = A vbar; kbar += -(2/L) Re[d/dk <u, A z_k> + d/dk <vbar, A^H r_k>]
    CK(op_apply_forward(L, vbar, ws, st));
    CK(op_reduce_forward_residual(L, ws, nullptr, ut, st));
    if (kbar) {
        to_tile_order_kernel<<<cdiv(L.nr_pad, T), T, 0, st>>>(z, L.nx, L.ny, L.ntx, L.nr_pad,
                                                            (float2 *)(ws + R.off_zq));
        to_tile_order_kernel<<<cdiv(L.nr_pad, T), T, 0, st>>>(vbar, L.nx, L.ny, L.ntx, L.nr_pad,
                                                            (float2 *)(ws + R.off_gq));
        CK(grad_k_launch(R, ws, st));
        const size_t n = (size_t)L.nl * L.nt;
        if (n > 0)
            grad_k_reduce_kernel<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(
                (const float *)(ws + R.off_gpart), R.grad_splits, L.LP, L.ntp, L.nl, L.nt, hdr, kbar);
    }
    // zbar_k = vbar - (2/L) A^H u
    CK(op_apply_adjoint(L, ut, ws, st));
    CK(op_adjoint_reduce_step(L, ws, vbar, zbar_out, st));
    return cudaGetLastError();
}

}  // namespace aexp
