// The paper's own regulariser (Sec. 2.1): the undecimated wavelet transform at one level,
// its balanced-FISTA step and lambda = sigma / 2 read off the histogram of W A^H y
// (Supporting Information S1, Method 2).
//
// W: periodic, no downsampling, separable, every filter scaled by 1/sqrt(2) per dimension so
// that W^H W = I (a tight frame):
//   c_s[y][x] = 1/2 sum_{my,mx} f_{s,y}[my] f_{s,x}[mx] v[(y + my) mod ny][(x + mx) mod nx],
//   subband s = fx + 2 fy, f = h (0) or g (1): 0 LL, 1 HL, 2 LH, 3 HH; coefficients [4][ny][nx].
// W^H is its transpose.  The image is at most a few hundred pixels per side and L2 resident,
// so both directions compute one output pixel per thread straight from global memory.
//
// lambda: m = |c_s| over the three detail subbands, zeros discarded; m_max; a 4096-bin
// histogram over [0, m_max] gives the median bin (first bin whose cumulative count reaches
// ceil(n/2)), med = its centre; a 64-bin histogram over [0, 4 med); sigma = centre of its fullest
// bin (lowest on a tie); lambda = sigma / 2.  Integer atomics only, so the result does not
// depend on the order of the additions.
#include <math.h>

#include <algorithm>

#include "aexp_internal.cuh"
#include "wavelet_taps.cuh"

namespace aexp {

namespace {

constexpr int kFine = 4096;
constexpr int kCoarse = 64;

// auxiliary block: histograms and device scalars of the lambda rule
struct SwtAux {
    unsigned fine[kFine];
    unsigned coarse[kCoarse];
    unsigned mmax_bits;  // largest detail magnitude (float bits)
    unsigned n;          // detail coefficients with m > 0
    float upper;         // 4 med
    float pad;
    double lam;          // lambda in use
};

__device__ __forceinline__ float2 soft(float2 w, float tau) {
    const float m = sqrtf(w.x * w.x + w.y * w.y);
    const float s = m > tau ? 1.f - tau / m : 0.f;
    return make_float2(w.x * s, w.y * s);
}

// Analysis: all four subbands of pixel (y, x); detail subbands soft-thresholded with
// tau = lam / L (device scalars) when `lam` is given, else with tau_host when >= 0.
template <int TAPS>
__global__ void swt_analysis_kernel(const float2 *__restrict__ v, float2 *__restrict__ c, int ny, int nx,
                                    float tau_host, const double *lam, const double *lip) {
    __shared__ float s_tau;  // formed once per block: an FP64 division per thread is slow here
    if (threadIdx.x == 0) s_tau = lam ? (float)(*lam / *lip) : tau_host;
    __syncthreads();
    const float tau = s_tau;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx * ny) return;
    const int y = i / nx, x = i % nx;
    float2 a[4] = {};
#pragma unroll
    for (int my = 0; my < TAPS; ++my) {
        const float2 *row = v + (size_t)((y + my) % ny) * nx;
        float2 lo = make_float2(0.f, 0.f), hi = make_float2(0.f, 0.f);
#pragma unroll
        for (int mx = 0; mx < TAPS; ++mx) {
            const float2 s = row[(x + mx) % nx];
            lo = tmad(tap_h<TAPS>(mx), s, lo);
            hi = tmad(tap_g<TAPS>(mx), s, hi);
        }
        const Tap hy = tap_h<TAPS>(my), gy = tap_g<TAPS>(my);
        a[0] = tmad(hy, lo, a[0]);
        a[1] = tmad(hy, hi, a[1]);
        a[2] = tmad(gy, lo, a[2]);
        a[3] = tmad(gy, hi, a[3]);
    }
    const size_t plane = (size_t)nx * ny;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        float2 w = make_float2(0.5f * a[s].x, 0.5f * a[s].y);
        if (s > 0 && tau >= 0.f) w = soft(w, tau);
        c[s * plane + i] = w;
    }
}

// Synthesis (W^H): pixel (y, x) collects c_s[y - my][x - mx] f_{s,y}[my] f_{s,x}[mx] / 2.
// momentum: out = x_new, z = x_new + beta (x_new - x_old).
template <int TAPS>
__global__ void swt_synthesis_kernel(const float2 *__restrict__ c, float2 *__restrict__ out, int ny, int nx,
                                     int momentum, float beta, const float2 *__restrict__ x_old,
                                     float2 *__restrict__ z) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx * ny) return;
    const int y = i / nx, x = i % nx;
    const size_t plane = (size_t)nx * ny;
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int my = 0; my < TAPS; ++my) {
        const size_t r = (size_t)pmod(y - my, ny) * nx;
        float2 lo = make_float2(0.f, 0.f), hi = make_float2(0.f, 0.f);  // summed over s with fy = 0 / 1
#pragma unroll
        for (int mx = 0; mx < TAPS; ++mx) {
            const size_t j = r + pmod(x - mx, nx);
            const Tap hx = tap_h<TAPS>(mx), gx = tap_g<TAPS>(mx);
            lo = tmad(hx, c[j], lo);
            lo = tmad(gx, c[plane + j], lo);
            hi = tmad(hx, c[2 * plane + j], hi);
            hi = tmad(gx, c[3 * plane + j], hi);
        }
        acc = tmad(tap_h<TAPS>(my), lo, acc);
        acc = tmad(tap_g<TAPS>(my), hi, acc);
    }
    acc = make_float2(0.5f * acc.x, 0.5f * acc.y);
    out[i] = acc;
    if (momentum) {
        const float2 o = x_old[i];
        z[i] = make_float2(fmaf(beta, acc.x - o.x, acc.x), fmaf(beta, acc.y - o.y, acc.y));
    }
}

// ---- lambda = sigma / 2 ----
__global__ void aux_reset_kernel(SwtAux *a) {
    for (int i = threadIdx.x; i < kFine; i += blockDim.x) a->fine[i] = 0u;
    for (int i = threadIdx.x; i < kCoarse; i += blockDim.x) a->coarse[i] = 0u;
    if (threadIdx.x == 0) {
        a->mmax_bits = 0u;
        a->n = 0u;
    }
}

__device__ __forceinline__ float cmag(float2 w) { return sqrtf(w.x * w.x + w.y * w.y); }

__global__ void detail_max_kernel(const float2 *__restrict__ d, size_t n, SwtAux *a) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    float m = i < n ? cmag(d[i]) : 0.f;
    const unsigned nz = __popc(__ballot_sync(0xffffffffu, m > 0.f));
    for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) {
        if (m > 0.f) atomicMax(&a->mmax_bits, __float_as_uint(m));
        if (nz) atomicAdd(&a->n, nz);
    }
}

__global__ void fine_hist_kernel(const float2 *__restrict__ d, size_t n, SwtAux *a) {
    __shared__ unsigned h[kFine];
    for (int b = threadIdx.x; b < kFine; b += blockDim.x) h[b] = 0u;
    __syncthreads();
    const float mmax = __uint_as_float(a->mmax_bits);
    const float scale = mmax > 0.f ? (float)kFine / mmax : 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float m = cmag(d[i]);
        if (m > 0.f) atomicAdd(&h[min((int)floorf(m * scale), kFine - 1)], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kFine; b += blockDim.x)
        if (h[b]) atomicAdd(&a->fine[b], h[b]);
}

// one block of 1024 threads: the median bin -> upper = 4 med
__global__ void __launch_bounds__(1024) median_kernel(SwtAux *a) {
    __shared__ unsigned csum[1024];
    // each thread sums 4 consecutive bins; an inclusive scan over threads gives the cumulative
    // count at the end of every group of 4
    unsigned s4 = 0;
    for (int k = 0; k < 4; ++k) s4 += a->fine[4 * threadIdx.x + k];
    csum[threadIdx.x] = s4;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
        const unsigned t = threadIdx.x >= o ? csum[threadIdx.x - o] : 0u;
        __syncthreads();
        csum[threadIdx.x] += t;
        __syncthreads();
    }
    const unsigned half = (a->n + 1) / 2;
    const unsigned before = threadIdx.x ? csum[threadIdx.x - 1] : 0u;
    if (a->n > 0 && before < half && csum[threadIdx.x] >= half) {  // exactly one thread
        unsigned c = before;
        int b = 4 * threadIdx.x;
        for (int k = 0; k < 4; ++k, ++b) {
            c += a->fine[b];
            if (c >= half) break;
        }
        const float mmax = __uint_as_float(a->mmax_bits);
        a->upper = 4.f * ((float)b + 0.5f) * mmax / (float)kFine;
    }
    if (a->n == 0 && threadIdx.x == 0) a->upper = 0.f;
}

__global__ void coarse_hist_kernel(const float2 *__restrict__ d, size_t n, SwtAux *a) {
    __shared__ unsigned h[kCoarse];
    for (int b = threadIdx.x; b < kCoarse; b += blockDim.x) h[b] = 0u;
    __syncthreads();
    const float u = a->upper;
    const float scale = u > 0.f ? (float)kCoarse / u : 0.f;
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
        const float m = cmag(d[i]);
        if (m > 0.f && m < u) atomicAdd(&h[min((int)floorf(m * scale), kCoarse - 1)], 1u);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < kCoarse; b += blockDim.x)
        if (h[b]) atomicAdd(&a->coarse[b], h[b]);
}

__global__ void lambda_kernel(SwtAux *a, double *lam_out) {
    int best = 0;
    for (int b = 1; b < kCoarse; ++b)
        if (a->coarse[b] > a->coarse[best]) best = b;
    const double sigma = a->n ? ((double)best + 0.5) * (double)a->upper / kCoarse : 0.0;
    a->lam = 0.5 * sigma;
    if (lam_out) *lam_out = a->lam;
}

__global__ void lambda_set_kernel(SwtAux *a, double lam, double *lam_out) {
    a->lam = lam;
    if (lam_out) *lam_out = lam;
}

}  // namespace

size_t swt_aux_bytes() { return sizeof(SwtAux); }

double *swt_lambda_slot(char *aux) { return &reinterpret_cast<SwtAux *>(aux)->lam; }

cudaError_t swt_analysis(int wavelet, const float2 *v, float2 *c, int nx, int ny, float tau_host, const double *lam,
                         const double *lip, cudaStream_t st) {
    const int n = nx * ny, T = 256;
    if (wavelet == AEXP_WAVELET_HAAR)
        swt_analysis_kernel<2><<<cdiv(n, T), T, 0, st>>>(v, c, ny, nx, tau_host, lam, lip);
    else
        swt_analysis_kernel<8><<<cdiv(n, T), T, 0, st>>>(v, c, ny, nx, tau_host, lam, lip);
    return cudaGetLastError();
}

cudaError_t swt_synthesis(int wavelet, const float2 *c, float2 *out, int nx, int ny, int momentum, double beta,
                          const float2 *x_old, float2 *z, cudaStream_t st) {
    const int n = nx * ny, T = 256;
    if (wavelet == AEXP_WAVELET_HAAR)
        swt_synthesis_kernel<2><<<cdiv(n, T), T, 0, st>>>(c, out, ny, nx, momentum, (float)beta, x_old, z);
    else
        swt_synthesis_kernel<8><<<cdiv(n, T), T, 0, st>>>(c, out, ny, nx, momentum, (float)beta, x_old, z);
    return cudaGetLastError();
}

// lambda = sigma / 2 from the detail subbands of the coefficients c (of W A^H y) -> aux->lam
cudaError_t swt_rayleigh_lambda(const float2 *c, int nx, int ny, char *aux, double *lam_out, cudaStream_t st) {
    SwtAux *a = reinterpret_cast<SwtAux *>(aux);
    const size_t n = (size_t)3 * nx * ny;
    const float2 *d = c + (size_t)nx * ny;
    const int T = 256;
    aux_reset_kernel<<<1, 1024, 0, st>>>(a);
    detail_max_kernel<<<(unsigned)((n + T - 1) / T), T, 0, st>>>(d, n, a);
    const unsigned blocks = (unsigned)std::min<size_t>((n + T - 1) / T, 152 * 4);
    fine_hist_kernel<<<blocks, T, 0, st>>>(d, n, a);
    median_kernel<<<1, 1024, 0, st>>>(a);
    coarse_hist_kernel<<<blocks, T, 0, st>>>(d, n, a);
    lambda_kernel<<<1, 1, 0, st>>>(a, lam_out);
    return cudaGetLastError();
}

cudaError_t swt_set_lambda(char *aux, double lam, double *lam_out, cudaStream_t st) {
    lambda_set_kernel<<<1, 1, 0, st>>>(reinterpret_cast<SwtAux *>(aux), lam, lam_out);
    return cudaGetLastError();
}

}  // namespace aexp
