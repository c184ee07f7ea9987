// Orthonormal periodised 2-D wavelet transform W and complex soft-threshold: the
// regulariser lambda ||W x||_1 of Eq. (1), low-pass weight 0 (Supporting Information S1).
//
// One level, length-n signal a (n even), lowpass taps h, highpass g[m] = (-1)^m h[M-1-m]:
//   lo[j] = sum_m h[m] a[(2j+m) mod n],   hi[j] = sum_m g[m] a[(2j+m) mod n]
// rows (x) are filtered before columns (y); Mallat layout: LL top-left, (lo-y, hi-x)
// top-right, (hi-y, lo-x) bottom-left, HH bottom-right.  The synthesis is the transpose.
// The image is zero-padded to npy x npx (multiples of 2^J) and cropped after synthesis.
//
// The first level is one launch each way; a block loads the input patch it needs (with periodic
// halo) into shared memory, filters rows then columns there, and writes four OB x OB output
// blocks, thresholding detail coefficients on the way out.  The prox step (analysis, threshold,
// synthesis) runs levels 2..J in one more launch: one CTA per image holds the level-1
// approximation (N_p/2 x N_p/2) and a scratch copy in shared memory and runs every coarser level
// of analysis, threshold and synthesis there, so a prox step is three launches instead of 2J
// (each level launch is latency bound at these sizes, ~8-11 us whatever its grid).  Images whose
// level-1 approximation does not fit (over 12800 coefficients) take one launch per level.
#include <cooperative_groups.h>

#include <algorithm>

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
    if (threadIdx.x == 0 && threadIdx.y == 0) s_tau = lipschitz ? (float)((double)lam / *lipschitz) : lam;
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

// ---- levels 2..J of the prox step in one CTA (shared memory) ----
constexpr int kMidTx = 32, kMidTy = 32;  // 1024 threads: x across a row, y across rows
constexpr int kMidThreads = kMidTx * kMidTy;
constexpr int kMidMaxCoef = 12800;  // level-1 approximation coefficients held: 2 x 100 KB of shared memory

// acc + t v on both components of a complex value, as packed FP32x2 FMAs (tap lo part first)
__device__ __forceinline__ float2 tmad2(Tap t, float2 v, float2 acc) {
    return __ffma2_rn(make_float2(t.hi, t.hi), v, __ffma2_rn(make_float2(t.lo, t.lo), v, acc));
}

// v reduced into [0, n) for 0 <= v < 2n (one subtraction) when n >= TAPS; regions narrower
// than the filter (n < TAPS) take the general periodic reduction
template <int TAPS>
__device__ __forceinline__ int wrap(int v, int n) {
    return n >= TAPS ? (v >= n ? v - n : v) : pmod(v, n);
}

// A: the level-1 approximation (m1y x m1x, row stride m1x) in shared memory, B: scratch of the
// same size.  Analysis of levels 2..levels in place in A (Mallat layout inside the region),
// details shrunk by tau, then synthesis back to the level-1 approximation in A.  The same
// filters, periodic extension and order (rows before columns; synthesis the transpose) as the
// per-level kernels.
// Flat loop over an h x w output grid with the block's threads (index = row * w + col, stride
// kMidThreads), row and column stepped without a division per iteration.
template <class Body>
__device__ __forceinline__ void mid_for(int h, int w, Body body) {
    const int tid = threadIdx.y * kMidTx + threadIdx.x;
    const int di = kMidThreads / w, dc = kMidThreads - di * w;
    int r = tid / w, c = tid - r * w;
    while (r < h) {
        body(r, c);
        r += di;
        c += dc;
        if (c >= w) {
            c -= w;
            ++r;
        }
    }
}

template <int TAPS>
__device__ void mid_levels(float2 *A, float2 *B, int m1y, int m1x, int levels, float tau) {
    for (int j = 2; j <= levels; ++j) {
        const int my = m1y >> (j - 2), mx = m1x >> (j - 2);
        const int hy = my / 2, hx = mx / 2;
        // rows (x): B[i][q] = sum_t h[t] A[i][(2q + t) mod mx], B[i][hx + q] the same with g
        mid_for(my, hx, [&](int i, int q) {
            const float2 *row = A + i * m1x;
            float2 lo = make_float2(0.f, 0.f), hi = make_float2(0.f, 0.f);
#pragma unroll
            for (int t = 0; t < TAPS; ++t) {
                const float2 v = row[wrap<TAPS>(2 * q + t, mx)];
                lo = tmad2(tap_h<TAPS>(t), v, lo);
                hi = tmad2(tap_g<TAPS>(t), v, hi);
            }
            B[i * m1x + q] = lo;
            B[i * m1x + hx + q] = hi;
        });
        __syncthreads();
        // columns (y): A[o][c] = sum_t h[t] B[(2o + t) mod my][c], A[hy + o][c] the same with g;
        // every quadrant but the top-left (the next level's approximation) is a detail band
        mid_for(hy, mx, [&](int o, int c) {
            float2 lo = make_float2(0.f, 0.f), hi = make_float2(0.f, 0.f);
#pragma unroll
            for (int t = 0; t < TAPS; ++t) {
                const float2 v = B[wrap<TAPS>(2 * o + t, my) * m1x + c];
                lo = tmad2(tap_h<TAPS>(t), v, lo);
                hi = tmad2(tap_g<TAPS>(t), v, hi);
            }
            A[o * m1x + c] = c < hx ? lo : shrink(lo, tau);
            A[(hy + o) * m1x + c] = shrink(hi, tau);
        });
        __syncthreads();
    }
    for (int j = levels; j >= 2; --j) {
        const int my = m1y >> (j - 2), mx = m1x >> (j - 2);
        const int hy = my / 2, hx = mx / 2;
        // columns (y): B[q][c] = sum over t with q - t even of h[t] A[k][c] + g[t] A[hy + k][c],
        // k = (q - t) / 2 mod hy; output rows q = 2a and 2a + 1 take the even and odd taps
        mid_for(hy, mx, [&](int a, int c) {
            float2 ev = make_float2(0.f, 0.f), od = make_float2(0.f, 0.f);
#pragma unroll
            for (int t = 0; t < TAPS; t += 2) {
                const int k = wrap<TAPS>(a - t / 2 + hy, hy);  // (2a - t) / 2 mod hy, also (2a + 1 - (t + 1)) / 2
                const float2 lo = A[k * m1x + c], hi = A[(hy + k) * m1x + c];
                ev = tmad2(tap_h<TAPS>(t), lo, tmad2(tap_g<TAPS>(t), hi, ev));
                od = tmad2(tap_h<TAPS>(t + 1), lo, tmad2(tap_g<TAPS>(t + 1), hi, od));
            }
            B[2 * a * m1x + c] = ev;
            B[(2 * a + 1) * m1x + c] = od;
        });
        __syncthreads();
        // rows (x): A[r][p] = sum over t with p - t even of h[t] B[r][k] + g[t] B[r][hx + k]
        mid_for(my, hx, [&](int r, int a) {
            const float2 *row = B + r * m1x;
            float2 ev = make_float2(0.f, 0.f), od = make_float2(0.f, 0.f);
#pragma unroll
            for (int t = 0; t < TAPS; t += 2) {
                const int k = wrap<TAPS>(a - t / 2 + hx, hx);
                const float2 lo = row[k], hi = row[hx + k];
                ev = tmad2(tap_h<TAPS>(t), lo, tmad2(tap_g<TAPS>(t), hi, ev));
                od = tmad2(tap_h<TAPS>(t + 1), lo, tmad2(tap_g<TAPS>(t + 1), hi, od));
            }
            A[r * m1x + 2 * a] = ev;
            A[r * m1x + 2 * a + 1] = od;
        });
        __syncthreads();
    }
}

// Level-1 approximation (m1y x m1x, m1x even) between global and shared memory, two values per
// 16-byte access.
__device__ __forceinline__ void mid_copy(float4 *dst, const float4 *src, int n4) {
    const int tid = threadIdx.y * kMidTx + threadIdx.x;
    for (int i = tid; i < n4; i += kMidThreads) dst[i] = src[i];
}

// One CTA: approx (the level-1 approximation, m1y x m1x in global memory) -> levels 2..levels
// -> approx (overwritten with the synthesised level-1 approximation).
template <int TAPS>
__global__ void __launch_bounds__(kMidThreads)
    dwt_mid_kernel(float2 *__restrict__ approx, int m1y, int m1x, int levels, float lam, const double *lipschitz) {
    extern __shared__ float2 smid[];
    const float tau = block_tau(lam, lipschitz);
    float2 *A = smid, *B = smid + m1y * m1x;
    mid_copy(reinterpret_cast<float4 *>(A), reinterpret_cast<const float4 *>(approx), m1y * m1x / 2);
    __syncthreads();
    mid_levels<TAPS>(A, B, m1y, m1x, levels, tau);
    mid_copy(reinterpret_cast<float4 *>(approx), reinterpret_cast<const float4 *>(A), m1y * m1x / 2);
}

// The same per problem of a batch (grid.x = problem).
template <int TAPS>
__global__ void __launch_bounds__(kMidThreads) batch_dwt_mid_kernel(const ProbDesc *__restrict__ pd) {
    extern __shared__ float2 smid[];
    const ProbDesc &P = pd[blockIdx.x];
    const float tau = block_tau(P.lam, &P.hdr->lipschitz);
    const int m1y = P.npy / 2, m1x = P.npx / 2;
    float2 *approx = (float2 *)(P.wws + P.off_approx[1]);
    float2 *A = smid, *B = smid + m1y * m1x;
    mid_copy(reinterpret_cast<float4 *>(A), reinterpret_cast<const float4 *>(approx), m1y * m1x / 2);
    __syncthreads();
    mid_levels<TAPS>(A, B, m1y, m1x, P.levels, tau);
    mid_copy(reinterpret_cast<float4 *>(approx), reinterpret_cast<const float4 *>(A), m1y * m1x / 2);
}

// ---- levels 2..J of the prox step in one cluster of kMidCluster CTAs ----
// Each CTA owns a band of output rows per level, o in [rank hy / NC, (rank + 1) hy / NC), the
// same band for the synthesis.  Two full-size arrays X, Y alternate between levels: level j
// reads its input approximation from one and writes its outputs (the next approximation and its
// thresholded details) into the other, in every CTA of the cluster (distributed shared memory),
// so that each CTA holds a full copy of every level's coefficients and no level overwrites
// what another CTA may still be reading; a per-CTA scratch B holds only the filtered rows the
// band needs.  Per output the arithmetic and its order are those of mid_levels.
constexpr int kMidCluster = 8;

// Rows of B: the most any level's band needs (its 2 nb rows plus the filter's TAPS - 2 halo).
inline int mid_cluster_brows(int m1y, int taps) {
    const int hy = m1y / 2;
    return std::min(m1y, 2 * ((hy + kMidCluster - 1) / kMidCluster) + taps - 2);
}
// dynamic shared memory a cluster CTA may take (227 KB less the static s_tau, rounded down)
constexpr size_t kMidClusterSmemMax = 227 * 1024 - 256;
inline size_t mid_cluster_smem(int m1y, int m1x, int taps) {
    return sizeof(float2) * ((size_t)2 * m1y * m1x + (size_t)mid_cluster_brows(m1y, taps) * m1x);
}

template <int TAPS>
__device__ void mid_levels_cluster(float2 *__restrict__ approx, float2 *sm, int m1y, int m1x, int levels, float tau) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    // no CTA may write into another's shared memory before that CTA has started: arrive here,
    // wait before the first distributed-shared-memory store
    auto started = cl.barrier_arrive();
    const int rank = (int)cl.block_rank();
    const int n1 = m1y * m1x;
    float2 *X = sm, *Y = sm + n1, *B = sm + 2 * n1;
    // every CTA's copy of `arr` at flat index i gets v
    auto put_all = [&](float2 *arr, int i, float2 v) {
#pragma unroll
        for (int r = 0; r < kMidCluster; ++r) cl.map_shared_rank(arr, r)[i] = v;
    };
    {   // level 2 reads rows (2 o0 + i) mod m1y, i < L, of the level-1 approximation
        const int hy = m1y / 2, o0 = rank * hy / kMidCluster, nb = (rank + 1) * hy / kMidCluster - o0;
        const int L = min(m1y, 2 * nb + TAPS - 2);
        if (nb > 0)
            mid_for(L, m1x / 2, [&](int i, int q) {
                const int r = (2 * o0 + i) % m1y;
                reinterpret_cast<float4 *>(X + r * m1x)[q] = reinterpret_cast<const float4 *>(approx + r * m1x)[q];
            });
    }
    __syncthreads();
    cl.barrier_wait(std::move(started));
    float2 *P = X, *Q = Y;
    for (int j = 2; j <= levels; ++j) {
        const int my = m1y >> (j - 2), mx = m1x >> (j - 2);
        const int hy = my / 2, hx = mx / 2;
        const int o0 = rank * hy / kMidCluster, nb = (rank + 1) * hy / kMidCluster - o0;
        const int L = min(my, 2 * nb + TAPS - 2);
        // rows (x): B[i] = the filtered row (2 o0 + i) mod my of P
        if (nb > 0)
            mid_for(L, hx, [&](int i, int q) {
                const float2 *row = P + ((2 * o0 + i) % my) * m1x;
                float2 lo = make_float2(0.f, 0.f), hi = make_float2(0.f, 0.f);
#pragma unroll
                for (int t = 0; t < TAPS; ++t) {
                    const float2 v = row[wrap<TAPS>(2 * q + t, mx)];
                    lo = tmad2(tap_h<TAPS>(t), v, lo);
                    hi = tmad2(tap_g<TAPS>(t), v, hi);
                }
                B[i * m1x + q] = lo;
                B[i * m1x + hx + q] = hi;
            });
        __syncthreads();
        // columns (y) of the band, into Q in every CTA
        if (nb > 0)
            mid_for(nb, mx, [&](int oi, int c) {
                const int o = o0 + oi;
                float2 lo = make_float2(0.f, 0.f), hi = make_float2(0.f, 0.f);
#pragma unroll
                for (int t = 0; t < TAPS; ++t) {
                    const float2 v = B[wrap<TAPS>(2 * oi + t, L) * m1x + c];
                    lo = tmad2(tap_h<TAPS>(t), v, lo);
                    hi = tmad2(tap_g<TAPS>(t), v, hi);
                }
                put_all(Q, o * m1x + c, c < hx ? lo : shrink(lo, tau));
                put_all(Q, (hy + o) * m1x + c, shrink(hi, tau));
            });
        cl.sync();
        float2 *tmp = P;
        P = Q;
        Q = tmp;
    }
    for (int j = levels; j >= 2; --j) {
        const int my = m1y >> (j - 2), mx = m1x >> (j - 2);
        const int hy = my / 2, hx = mx / 2;
        const int a0 = rank * hy / kMidCluster, nb = (rank + 1) * hy / kMidCluster - a0;
        // level j's details and the approximation of level j + 1 sit in the array level j wrote
        // (Y for even j); its output, the approximation of level j, goes where level j - 1's
        // synthesis reads it (the other array), or to `approx` for j = 2
        const float2 *Qj = (j & 1) ? X : Y;
        float2 *Out = (j & 1) ? Y : X;
        // columns (y): B rows 2 (a - a0) and 2 (a - a0) + 1
        if (nb > 0)
            mid_for(nb, mx, [&](int ai, int c) {
                const int a = a0 + ai;
                float2 ev = make_float2(0.f, 0.f), od = make_float2(0.f, 0.f);
#pragma unroll
                for (int t = 0; t < TAPS; t += 2) {
                    const int k = wrap<TAPS>(a - t / 2 + hy, hy);
                    const float2 lo = Qj[k * m1x + c], hi = Qj[(hy + k) * m1x + c];
                    ev = tmad2(tap_h<TAPS>(t), lo, tmad2(tap_g<TAPS>(t), hi, ev));
                    od = tmad2(tap_h<TAPS>(t + 1), lo, tmad2(tap_g<TAPS>(t + 1), hi, od));
                }
                B[2 * ai * m1x + c] = ev;
                B[(2 * ai + 1) * m1x + c] = od;
            });
        __syncthreads();
        // rows (x): output rows 2 a0 + i, i < 2 nb
        if (nb > 0)
            mid_for(2 * nb, hx, [&](int i, int a) {
                const float2 *row = B + i * m1x;
                float2 ev = make_float2(0.f, 0.f), od = make_float2(0.f, 0.f);
#pragma unroll
                for (int t = 0; t < TAPS; t += 2) {
                    const int k = wrap<TAPS>(a - t / 2 + hx, hx);
                    const float2 lo = row[k], hi = row[hx + k];
                    ev = tmad2(tap_h<TAPS>(t), lo, tmad2(tap_g<TAPS>(t), hi, ev));
                    od = tmad2(tap_h<TAPS>(t + 1), lo, tmad2(tap_g<TAPS>(t + 1), hi, od));
                }
                const int r = 2 * a0 + i;
                if (j > 2) {
                    put_all(Out, r * m1x + 2 * a, ev);
                    put_all(Out, r * m1x + 2 * a + 1, od);
                } else {
                    reinterpret_cast<float4 *>(approx + r * m1x)[a] = make_float4(ev.x, ev.y, od.x, od.y);
                }
            });
        if (j > 2) cl.sync();
    }
}

template <int TAPS>
__global__ void __cluster_dims__(kMidCluster, 1, 1) __launch_bounds__(kMidThreads)
    dwt_mid_cluster_kernel(float2 *__restrict__ approx, int m1y, int m1x, int levels, float lam,
                           const double *lipschitz) {
    extern __shared__ float4 smc4[];
    const float tau = block_tau(lam, lipschitz);
    mid_levels_cluster<TAPS>(approx, reinterpret_cast<float2 *>(smc4), m1y, m1x, levels, tau);
}

// The same per problem of a batch (cluster = problem blockIdx.y).
template <int TAPS>
__global__ void __cluster_dims__(kMidCluster, 1, 1) __launch_bounds__(kMidThreads)
    batch_dwt_mid_cluster_kernel(const ProbDesc *__restrict__ pd) {
    extern __shared__ float4 smc4[];
    const ProbDesc &P = pd[blockIdx.y];
    const float tau = block_tau(P.lam, &P.hdr->lipschitz);
    mid_levels_cluster<TAPS>((float2 *)(P.wws + P.off_approx[1]), reinterpret_cast<float2 *>(smc4), P.npy / 2,
                             P.npx / 2, P.levels, tau);
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

// Prox step: level 1 analysis (threshold), levels 2..J in one CTA, level 1 synthesis (momentum).
template <int TAPS>
cudaError_t run_prox(const WaveLayout &W, const float2 *img, char *wws, float lam, const double *lipschitz,
                     float2 *out, int momentum, double beta, const float2 *x_old, float2 *z_out, cudaStream_t st) {
    WaveLayout W1 = W;
    W1.levels = 1;  // level 1 of the full pyramid: LL into the level-1 approximation, details into pyr
    float2 *pyr = (float2 *)(wws + W.off_pyr);
    float2 *ll1 = (float2 *)(wws + W.off_approx[1]);
    const int m1y = W.npy / 2, m1x = W.npx / 2;
    {
        dim3 grid(cdiv(m1x, OB), cdiv(m1y, OB));
        dwt_fwd_level<TAPS><<<grid, 256, 0, st>>>(img, W.nx, W.ny, W.nx, W.npy, W.npx, ll1, m1x, pyr, W.npx, lam,
                                                 lipschitz, 1);
    }
    const size_t csmem = mid_cluster_smem(m1y, m1x, TAPS);
    if (csmem <= kMidClusterSmemMax) {
        auto kern = dwt_mid_cluster_kernel<TAPS>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csmem);
        if (e != cudaSuccess) return e;
        kern<<<kMidCluster, dim3(kMidTx, kMidTy), csmem, st>>>(ll1, m1y, m1x, W.levels, lam, lipschitz);
    } else {
        const size_t smem = 2 * sizeof(float2) * (size_t)m1y * m1x;
        auto kern = dwt_mid_kernel<TAPS>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<1, dim3(kMidTx, kMidTy), smem, st>>>(ll1, m1y, m1x, W.levels, lam, lipschitz);
    }
    {
        dim3 grid(cdiv(W.npx, OBI), cdiv(W.npy, OBI));
        dwt_inv_level<TAPS><<<grid, 256, 0, st>>>(ll1, m1x, pyr, W.npx, W.npy, W.npx, out, W.nx, W.ny, W.nx, momentum,
                                                 (float)beta, x_old, z_out);
    }
    return cudaGetLastError();
}

template <int TAPS>
cudaError_t run_batch_prox(const ProbDesc *pd, int nprob, int levels, int max_npx, int max_npy, int img_role,
                           int out_role, int momentum, double beta, int xold_role, int z_role, cudaStream_t st) {
    {
        dim3 grid(cdiv(max_npx / 2, OB), cdiv(max_npy / 2, OB), nprob);
        batch_dwt_fwd_level<TAPS><<<grid, 256, 0, st>>>(pd, 1, img_role, 1);
    }
    const size_t csmem = mid_cluster_smem(max_npy / 2, max_npx / 2, TAPS);
    if (csmem <= kMidClusterSmemMax) {
        auto kern = batch_dwt_mid_cluster_kernel<TAPS>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)csmem);
        if (e != cudaSuccess) return e;
        kern<<<dim3(kMidCluster, nprob), dim3(kMidTx, kMidTy), csmem, st>>>(pd);
    } else {
        const size_t smem = 2 * sizeof(float2) * (size_t)(max_npy / 2) * (max_npx / 2);
        auto kern = batch_dwt_mid_kernel<TAPS>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        kern<<<nprob, dim3(kMidTx, kMidTy), smem, st>>>(pd);
    }
    {
        dim3 grid(cdiv(max_npx, OBI), cdiv(max_npy, OBI), nprob);
        batch_dwt_inv_level<TAPS><<<grid, 256, 0, st>>>(pd, 1, out_role, momentum, (float)beta, xold_role, z_role);
    }
    return cudaGetLastError();
}

}  // namespace

bool wave_mid_fits(int npx, int npy, int levels) {
    return levels >= 2 && (npx / 2) * (npy / 2) <= kMidMaxCoef;
}

cudaError_t wave_prox(const WaveLayout &W, const float2 *img, char *wws, float lam, const double *lipschitz,
                      float2 *out, int momentum, double beta, const float2 *x_old, float2 *z_out, cudaStream_t st) {
    if (!wave_mid_fits(W.npx, W.npy, W.levels)) {
        cudaError_t e = wave_forward(W, img, wws, lam, lipschitz, 1, st);
        return e == cudaSuccess ? wave_inverse(W, wws, out, momentum, beta, x_old, z_out, st) : e;
    }
    return W.wavelet == AEXP_WAVELET_HAAR
               ? run_prox<2>(W, img, wws, lam, lipschitz, out, momentum, beta, x_old, z_out, st)
               : run_prox<8>(W, img, wws, lam, lipschitz, out, momentum, beta, x_old, z_out, st);
}

cudaError_t batch_wave_prox(int wavelet, const ProbDesc *pd, int nprob, int levels, int max_npx, int max_npy,
                            int img_role, int out_role, int momentum, double beta, int xold_role, int z_role,
                            cudaStream_t st) {
    if (!wave_mid_fits(max_npx, max_npy, levels)) {
        cudaError_t e = batch_wave_forward(wavelet, pd, nprob, levels, max_npx, max_npy, img_role, 1, st);
        return e == cudaSuccess ? batch_wave_inverse(wavelet, pd, nprob, levels, max_npx, max_npy, out_role, momentum,
                                                     beta, xold_role, z_role, st)
                                : e;
    }
    return wavelet == AEXP_WAVELET_HAAR
               ? run_batch_prox<2>(pd, nprob, levels, max_npx, max_npy, img_role, out_role, momentum, beta, xold_role,
                                   z_role, st)
               : run_batch_prox<8>(pd, nprob, levels, max_npx, max_npy, img_role, out_role, momentum, beta, xold_role,
                                   z_role, st);
}

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
