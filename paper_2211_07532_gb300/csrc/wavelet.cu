// Orthonormal periodised 2-D wavelet transform W and complex soft-threshold: the
// regulariser lambda ||W x||_1 of Eq. (1), low-pass weight 0 (Supporting Information S1).
//
// One level, length-n signal a (n even), lowpass taps h, highpass g[m] = (-1)^m h[M-1-m]:
//   lo[j] = sum_m h[m] a[(2j+m) mod n],   hi[j] = sum_m g[m] a[(2j+m) mod n]
// rows (x) are filtered before columns (y); Mallat layout: LL top-left, (lo-y, hi-x)
// top-right, (hi-y, lo-x) bottom-left, HH bottom-right.  The synthesis is the transpose.
// The image is zero-padded to npy x npx (multiples of 2^J) and cropped after synthesis.
//
// Each level is one launch; a block loads the input patch it needs (with periodic halo)
// into shared memory, filters rows then columns there, and writes four OB x OB output
// blocks, thresholding detail coefficients on the way out.
#include "aexp_internal.cuh"
#include "wavelet_taps.cuh"

namespace aexp {

namespace {



__device__ __forceinline__ float2 shrink(float2 w, float tau) {
    float m2 = w.x * w.x + w.y * w.y;
    if (!(m2 > tau * tau)) return make_float2(0.f, 0.f);
    float s = 1.f - tau / sqrtf(m2);
    return make_float2(w.x * s, w.y * s);
}

// tau = lam / L_f, formed once per block (an FP64 division per thread costs more than the
// level's filtering on this part's FP64 pipe); every thread of the block must call it.
__device__ __forceinline__ float block_tau(float lam, const double *lipschitz) {
    __shared__ float s_tau;
    if (threadIdx.x == 0) s_tau = lipschitz ? (float)((double)lam / *lipschitz) : lam;
    __syncthreads();
    return s_tau;
}

constexpr int OB = 16;   // forward: output coefficients per subband per block side
constexpr int OBI = 32;  // inverse: output samples per block side

// One level of analysis for output block (bx, by): reads the n_y x n_x input (zero outside
// valid_y x valid_x), writes LL to `ll` and the three detail bands into the quadrants of the
// n_y x n_x block of `pyr`, shrinking details by tau when `threshold`.
template <int TAPS>
__device__ __forceinline__ void dwt_fwd_level_body(const float2 *__restrict__ in, int in_stride, int valid_y,
                                                   int valid_x, int n_y, int n_x, float2 *__restrict__ ll,
                                                   int ll_stride, float2 *__restrict__ pyr, int pyr_stride,
                                                   float tau, int threshold, int bx, int by) {
    constexpr int IN = 2 * OB + TAPS - 2;
    __shared__ float2 s_in[IN][IN];
    __shared__ float2 s_row[IN][2 * OB];
    const int my = n_y / 2, mx = n_x / 2;
    const int oy0 = by * OB, ox0 = bx * OB;

    for (int idx = threadIdx.x; idx < IN * IN; idx += blockDim.x) {
        int i = idx / IN, j = idx % IN;
        int gy = (2 * oy0 + i) % n_y, gx = (2 * ox0 + j) % n_x;
        s_in[i][j] = (gy < valid_y && gx < valid_x) ? in[(size_t)gy * in_stride + gx] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < IN * OB; idx += blockDim.x) {
        int i = idx / OB, q = idx % OB;
        float2 lo = make_float2(0.f, 0.f), hi = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 0; m < TAPS; ++m) {
            float2 a = s_in[i][2 * q + m];
            const Tap hm = tap_h<TAPS>(m), gm = tap_g<TAPS>(m);
            lo.x = tfma(hm, a.x, lo.x);
            lo.y = tfma(hm, a.y, lo.y);
            hi.x = tfma(gm, a.x, hi.x);
            hi.y = tfma(gm, a.y, hi.y);
        }
        s_row[i][q] = lo;
        s_row[i][OB + q] = hi;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < OB * 2 * OB; idx += blockDim.x) {
        int oy = idx / (2 * OB), col = idx % (2 * OB);
        float2 lo = make_float2(0.f, 0.f), hi = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 0; m < TAPS; ++m) {
            float2 a = s_row[2 * oy + m][col];
            const Tap hm = tap_h<TAPS>(m), gm = tap_g<TAPS>(m);
            lo.x = tfma(hm, a.x, lo.x);
            lo.y = tfma(hm, a.y, lo.y);
            hi.x = tfma(gm, a.x, hi.x);
            hi.y = tfma(gm, a.y, hi.y);
        }
        int gy = oy0 + oy, gx = ox0 + (col % OB);
        if (gy >= my || gx >= mx) continue;
        if (threshold) hi = shrink(hi, tau);
        if (col < OB) {  // lo in x
            ll[(size_t)gy * ll_stride + gx] = lo;
            pyr[(size_t)(my + gy) * pyr_stride + gx] = hi;
        } else {         // hi in x
            if (threshold) lo = shrink(lo, tau);
            pyr[(size_t)gy * pyr_stride + mx + gx] = lo;
            pyr[(size_t)(my + gy) * pyr_stride + mx + gx] = hi;
        }
    }
}

template <int TAPS>
__global__ void __launch_bounds__(256)
    dwt_fwd_level(const float2 *__restrict__ in, int in_stride, int valid_y, int valid_x, int n_y, int n_x,
                  float2 *__restrict__ ll, int ll_stride, float2 *__restrict__ pyr, int pyr_stride, float lam,
                  const double *lipschitz, int threshold) {
    const float tau = threshold ? block_tau(lam, lipschitz) : 0.f;
    dwt_fwd_level_body<TAPS>(in, in_stride, valid_y, valid_x, n_y, n_x, ll, ll_stride, pyr, pyr_stride, tau,
                             threshold, blockIdx.x, blockIdx.y);
}

// One level of synthesis for output block (bx, by) of the n_y x n_x result; writes inside
// valid_y x valid_x only; with `momentum` also z = x + beta (x - x_old) (same layout as out).
template <int TAPS>
__device__ __forceinline__ void dwt_inv_level_body(const float2 *__restrict__ ll, int ll_stride,
                                                   const float2 *__restrict__ pyr, int pyr_stride, int n_y, int n_x,
                                                   float2 *__restrict__ out, int out_stride, int valid_y,
                                                   int valid_x, int momentum, float beta,
                                                   const float2 *__restrict__ x_old, float2 *__restrict__ z_out,
                                                   int bx, int by) {
    constexpr int HALO = TAPS / 2 - 1;
    constexpr int SB = OBI / 2 + HALO;
    __shared__ float2 s_sb[4][SB][SB];     // LL, (lo-y,hi-x), (hi-y,lo-x), HH
    __shared__ float2 s_col[OBI][2 * SB];  // after y-synthesis: [row][lo-x j | hi-x j]
    const int my = n_y / 2, mx = n_x / 2;
    const int qy0 = by * OBI, qx0 = bx * OBI;
    const int jy0 = qy0 / 2 - HALO, jx0 = qx0 / 2 - HALO;

    for (int idx = threadIdx.x; idx < 4 * SB * SB; idx += blockDim.x) {
        int sb = idx / (SB * SB), rem = idx % (SB * SB);
        int i = rem / SB, j = rem % SB;
        int gy = pmod(jy0 + i, my), gx = pmod(jx0 + j, mx);
        float2 v;
        if (sb == 0) v = ll[(size_t)gy * ll_stride + gx];
        else if (sb == 1) v = pyr[(size_t)gy * pyr_stride + mx + gx];
        else if (sb == 2) v = pyr[(size_t)(my + gy) * pyr_stride + gx];
        else v = pyr[(size_t)(my + gy) * pyr_stride + mx + gx];
        s_sb[sb][i][j] = v;
    }
    __syncthreads();
    // synthesis along y: out_row(q) = sum_{m = q mod 2} h[m] lo[(q-m)/2] + g[m] hi[(q-m)/2]
    for (int idx = threadIdx.x; idx < OBI * 2 * SB; idx += blockDim.x) {
        int a = idx / (2 * SB), col = idx % (2 * SB);
        int xband = col / SB, j = col % SB;  // xband 0: lo-x (LL, hi-y lo-x); 1: hi-x
        int q = qy0 + a;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 0; m < TAPS; ++m) {
            if (((q - m) & 1) != 0) continue;
            int i = ((q - m) >> 1) - jy0;
            float2 lo = s_sb[xband == 0 ? 0 : 1][i][j];
            float2 hi = s_sb[xband == 0 ? 2 : 3][i][j];
            const Tap hm = tap_h<TAPS>(m), gm = tap_g<TAPS>(m);
            acc.x = tfma(hm, lo.x, tfma(gm, hi.x, acc.x));
            acc.y = tfma(hm, lo.y, tfma(gm, hi.y, acc.y));
        }
        s_col[a][col] = acc;
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < OBI * OBI; idx += blockDim.x) {
        int a = idx / OBI, b = idx % OBI;
        int qy = qy0 + a, qx = qx0 + b;
        if (qy >= n_y || qx >= n_x || qy >= valid_y || qx >= valid_x) continue;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int m = 0; m < TAPS; ++m) {
            if (((qx - m) & 1) != 0) continue;
            int j = ((qx - m) >> 1) - jx0;
            float2 lo = s_col[a][j];
            float2 hi = s_col[a][SB + j];
            const Tap hm = tap_h<TAPS>(m), gm = tap_g<TAPS>(m);
            acc.x = tfma(hm, lo.x, tfma(gm, hi.x, acc.x));
            acc.y = tfma(hm, lo.y, tfma(gm, hi.y, acc.y));
        }
        size_t o = (size_t)qy * out_stride + qx;
        if (momentum) {  // FISTA: z_{k+1} = x_k + beta_k (x_k - x_{k-1})
            float2 xo = x_old[o];
            z_out[o] = make_float2(acc.x + beta * (acc.x - xo.x), acc.y + beta * (acc.y - xo.y));
        }
        out[o] = acc;
    }
}

template <int TAPS>
__global__ void __launch_bounds__(256)
    dwt_inv_level(const float2 *__restrict__ ll, int ll_stride, const float2 *__restrict__ pyr, int pyr_stride,
                  int n_y, int n_x, float2 *__restrict__ out, int out_stride, int valid_y, int valid_x,
                  int momentum, float beta, const float2 *__restrict__ x_old, float2 *__restrict__ z_out) {
    dwt_inv_level_body<TAPS>(ll, ll_stride, pyr, pyr_stride, n_y, n_x, out, out_stride, valid_y, valid_x, momentum,
                             beta, x_old, z_out, blockIdx.x, blockIdx.y);
}

// ---- batched levels: grid.z = problem; blocks beyond a problem's level extent return ----
template <int TAPS>
__global__ void __launch_bounds__(256)
    batch_dwt_fwd_level(const ProbDesc *__restrict__ pd, int j, int img_role, int threshold) {
    const ProbDesc &P = pd[blockIdx.z];
    const int n_y = P.npy >> (j - 1), n_x = P.npx >> (j - 1);
    if ((int)blockIdx.x * OB >= n_x / 2 || (int)blockIdx.y * OB >= n_y / 2) return;
    const float2 *in;
    int in_stride, vy, vx;
    if (j == 1) {
        in = P.vec[img_role];
        in_stride = P.nx;
        vy = P.ny;
        vx = P.nx;
    } else {
        in = (const float2 *)(P.wws + P.off_approx[j - 1]);
        in_stride = n_x;
        vy = n_y;
        vx = n_x;
    }
    float2 *pyr = (float2 *)(P.wws + P.off_pyr);
    float2 *llp = j == P.levels ? pyr : (float2 *)(P.wws + P.off_approx[j]);
    const int ll_stride = j == P.levels ? P.npx : n_x / 2;
    const float tau = threshold ? block_tau(P.lam, &P.hdr->lipschitz) : 0.f;
    dwt_fwd_level_body<TAPS>(in, in_stride, vy, vx, n_y, n_x, llp, ll_stride, pyr, P.npx, tau, threshold, blockIdx.x,
                             blockIdx.y);
}

template <int TAPS>
__global__ void __launch_bounds__(256)
    batch_dwt_inv_level(const ProbDesc *__restrict__ pd, int j, int out_role, int momentum, float beta,
                        int xold_role, int z_role) {
    const ProbDesc &P = pd[blockIdx.z];
    const int n_y = P.npy >> (j - 1), n_x = P.npx >> (j - 1);
    if ((int)blockIdx.x * OBI >= n_x || (int)blockIdx.y * OBI >= n_y) return;
    const float2 *pyr = (const float2 *)(P.wws + P.off_pyr);
    const float2 *llp = j == P.levels ? pyr : (const float2 *)(P.wws + P.off_approx[j]);
    const int ll_stride = j == P.levels ? P.npx : n_x / 2;
    float2 *o;
    int o_stride, vy, vx, mom;
    if (j == 1) {
        o = P.vec[out_role];
        o_stride = P.nx;
        vy = P.ny;
        vx = P.nx;
        mom = momentum;
    } else {
        o = (float2 *)(P.wws + P.off_approx[j - 1]);
        o_stride = n_x;
        vy = n_y;
        vx = n_x;
        mom = 0;
    }
    dwt_inv_level_body<TAPS>(llp, ll_stride, pyr, P.npx, n_y, n_x, o, o_stride, vy, vx, mom, beta,
                             mom ? P.vec[xold_role] : nullptr, mom ? P.vec[z_role] : nullptr, blockIdx.x,
                             blockIdx.y);
}

template <int TAPS>
cudaError_t run_forward(const WaveLayout &W, const float2 *img, char *wws, float lam, const double *lipschitz,
                        int threshold, cudaStream_t st) {
    float2 *pyr = (float2 *)(wws + W.off_pyr);
    for (int j = 1; j <= W.levels; ++j) {
        int n_y = W.npy >> (j - 1), n_x = W.npx >> (j - 1);
        const float2 *in;
        int in_stride, vy, vx;
        if (j == 1) {
            in = img;
            in_stride = W.nx;
            vy = W.ny;
            vx = W.nx;
        } else {
            in = (const float2 *)(wws + W.off_approx[j - 1]);
            in_stride = n_x;
            vy = n_y;
            vx = n_x;
        }
        float2 *llp;
        int ll_stride;
        if (j == W.levels) {
            llp = pyr;
            ll_stride = W.npx;
        } else {
            llp = (float2 *)(wws + W.off_approx[j]);
            ll_stride = n_x / 2;
        }
        dim3 grid(cdiv(n_x / 2, OB), cdiv(n_y / 2, OB));
        dwt_fwd_level<TAPS><<<grid, 256, 0, st>>>(in, in_stride, vy, vx, n_y, n_x, llp, ll_stride, pyr, W.npx, lam,
                                                 lipschitz, threshold);
    }
    return cudaGetLastError();
}

template <int TAPS>
cudaError_t run_inverse(const WaveLayout &W, char *wws, float2 *out, int momentum, double beta,
                        const float2 *x_old, float2 *z_out, cudaStream_t st) {
    const float2 *pyr = (const float2 *)(wws + W.off_pyr);
    for (int j = W.levels; j >= 1; --j) {
        int n_y = W.npy >> (j - 1), n_x = W.npx >> (j - 1);
        const float2 *llp;
        int ll_stride;
        if (j == W.levels) {
            llp = pyr;
            ll_stride = W.npx;
        } else {
            llp = (const float2 *)(wws + W.off_approx[j]);
            ll_stride = n_x / 2;
        }
        float2 *o;
        int o_stride, vy, vx, mom;
        if (j == 1) {
            o = out;
            o_stride = W.nx;
            vy = W.ny;
            vx = W.nx;
            mom = momentum;
        } else {
            o = (float2 *)(wws + W.off_approx[j - 1]);
            o_stride = n_x;
            vy = n_y;
            vx = n_x;
            mom = 0;
        }
        dim3 grid(cdiv(n_x, OBI), cdiv(n_y, OBI));
        dwt_inv_level<TAPS><<<grid, 256, 0, st>>>(llp, ll_stride, pyr, W.npx, n_y, n_x, o, o_stride, vy, vx, mom,
                                                 (float)beta, x_old, z_out);
    }
    return cudaGetLastError();
}

template <int TAPS>
cudaError_t run_batch_forward(const ProbDesc *pd, int nprob, int levels, int max_npx, int max_npy, int img_role,
                              int threshold, cudaStream_t st) {
    for (int j = 1; j <= levels; ++j) {
        int n_y = max_npy >> (j - 1), n_x = max_npx >> (j - 1);
        dim3 grid(cdiv(n_x / 2, OB), cdiv(n_y / 2, OB), nprob);
        batch_dwt_fwd_level<TAPS><<<grid, 256, 0, st>>>(pd, j, img_role, threshold);
    }
    return cudaGetLastError();
}

template <int TAPS>
cudaError_t run_batch_inverse(const ProbDesc *pd, int nprob, int levels, int max_npx, int max_npy, int out_role,
                              int momentum, double beta, int xold_role, int z_role, cudaStream_t st) {
    for (int j = levels; j >= 1; --j) {
        int n_y = max_npy >> (j - 1), n_x = max_npx >> (j - 1);
        dim3 grid(cdiv(n_x, OBI), cdiv(n_y, OBI), nprob);
        batch_dwt_inv_level<TAPS><<<grid, 256, 0, st>>>(pd, j, out_role, momentum, (float)beta, xold_role, z_role);
    }
    return cudaGetLastError();
}

}  // namespace

cudaError_t batch_wave_forward(int wavelet, const ProbDesc *pd, int nprob, int levels, int max_npx, int max_npy,
                               int img_role, int threshold, cudaStream_t st) {
    return wavelet == AEXP_WAVELET_HAAR
               ? run_batch_forward<2>(pd, nprob, levels, max_npx, max_npy, img_role, threshold, st)
               : run_batch_forward<8>(pd, nprob, levels, max_npx, max_npy, img_role, threshold, st);
}

cudaError_t batch_wave_inverse(int wavelet, const ProbDesc *pd, int nprob, int levels, int max_npx, int max_npy,
                               int out_role, int momentum, double beta, int xold_role, int z_role, cudaStream_t st) {
    return wavelet == AEXP_WAVELET_HAAR
               ? run_batch_inverse<2>(pd, nprob, levels, max_npx, max_npy, out_role, momentum, beta, xold_role,
                                      z_role, st)
               : run_batch_inverse<8>(pd, nprob, levels, max_npx, max_npy, out_role, momentum, beta, xold_role,
                                      z_role, st);
}

cudaError_t wave_forward(const WaveLayout &W, const float2 *img, char *wws, float lam, const double *lipschitz,
                         int threshold, cudaStream_t st) {
    return W.wavelet == AEXP_WAVELET_HAAR ? run_forward<2>(W, img, wws, lam, lipschitz, threshold, st)
                                          : run_forward<8>(W, img, wws, lam, lipschitz, threshold, st);
}

cudaError_t wave_inverse(const WaveLayout &W, char *wws, float2 *out, int momentum, double beta,
                         const float2 *x_old, float2 *z_out, cudaStream_t st) {
    return W.wavelet == AEXP_WAVELET_HAAR ? run_inverse<2>(W, wws, out, momentum, beta, x_old, z_out, st)
                                          : run_inverse<8>(W, wws, out, momentum, beta, x_old, z_out, st);
}

}  // namespace aexp
