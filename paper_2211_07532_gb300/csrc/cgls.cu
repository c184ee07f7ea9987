// Least-squares reconstruction by the conjugate gradient method on the normal equations
// (CGLS), the paper's LS baseline (Sec. 2.1: conjugate gradient with early stopping, 20
// iterations chosen in Supporting Information S2):
//   x_0 = 0, r_0 = y, s_0 = A^H r_0, p_0 = s_0, gamma_0 = ||s_0||^2;
//   per iteration: q = A p, alpha = gamma / ||q||^2, x += alpha p, r -= alpha q,
//                  s = A^H r, gamma' = ||s||^2, p = s + (gamma' / gamma) p.
// The scalars stay on the device in FP64 (two-stage reductions in a fixed order, so runs
// are bitwise repeatable); the update kernels form alpha and beta themselves, so the whole
// loop can be captured in one CUDA graph.  Residual and search directions in k-space use the
// library's sample-major [ntp][CB] layout (padding entries stay zero).
#include <math.h>

#include "aexp_internal.cuh"

namespace aexp {

namespace {

constexpr int kNormThreads = 256;
constexpr int kNormBlocks = 256;  // first-stage partial sums

// partial[b] = sum over this block's grid-stride share of |w_i|^2 (FP64)
__global__ void __launch_bounds__(kNormThreads) norm2_partial_kernel(const float2 *__restrict__ w, size_t n,
                                                                      double *__restrict__ partial) {
    __shared__ double s[kNormThreads / 32];
    double a = 0.0;
    for (size_t i = (size_t)blockIdx.x * kNormThreads + threadIdx.x; i < n; i += (size_t)gridDim.x * kNormThreads) {
        const float2 v = w[i];
        a += (double)v.x * v.x + (double)v.y * v.y;
    }
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x < 32) {
        a = threadIdx.x < kNormThreads / 32 ? s[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (threadIdx.x == 0) partial[blockIdx.x] = a;
    }
}

// *out = sum of the kNormBlocks partial sums (one block, fixed order)
__global__ void __launch_bounds__(kNormBlocks) norm2_final_kernel(const double *__restrict__ partial, double *out) {
    __shared__ double s[kNormBlocks / 32];
    double a = partial[threadIdx.x];
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = a;
    __syncthreads();
    if (threadIdx.x < 32) {
        a = threadIdx.x < kNormBlocks / 32 ? s[threadIdx.x] : 0.0;
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (threadIdx.x == 0) *out = a;
    }
}

// num / den as FP32, 0 when the denominator vanishes (CG has converged exactly)
__device__ __forceinline__ float safe_ratio(const double *num, const double *den) {
    const double d = *den;
    return d > 0.0 ? (float)(*num / d) : 0.f;
}

// y += sign * (num / den) * x
__global__ void axpy_ratio_kernel(float2 *__restrict__ y, const float2 *__restrict__ x, size_t n, const double *num,
                                  const double *den, float sign) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float a = sign * safe_ratio(num, den);
    const float2 xv = x[i], yv = y[i];
    y[i] = make_float2(fmaf(a, xv.x, yv.x), fmaf(a, xv.y, yv.y));
}

// p = s + (num / den) p
__global__ void xpay_ratio_kernel(float2 *__restrict__ p, const float2 *__restrict__ s, size_t n, const double *num,
                                  const double *den) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float b = safe_ratio(num, den);
    const float2 sv = s[i], pv = p[i];
    p[i] = make_float2(fmaf(b, pv.x, sv.x), fmaf(b, pv.y, sv.y));
}

__global__ void copy_kernel(float2 *__restrict__ dst, const float2 *__restrict__ src, size_t n) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) dst[i] = src[i];
}

#define CK(x)                               \
    do {                                    \
        cudaError_t e__ = (x);              \
        if (e__ != cudaSuccess) return e__; \
    } while (0)

unsigned grid_for(size_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

int cgls_layout(const aexp_problem *p, const aexp_recon_opts *o, CglsLayout *C) {
    CglsLayout c{};
    int rc = op_layout(p, o->precision, &c.op, items_target(o->precision, o->items_per_sm), o->tile_variant);
    if (rc) return rc;
    size_t off = c.op.bytes;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = align_up(off + bytes);
        return at;
    };
    const size_t nr = (size_t)c.op.nr, nk = (size_t)c.op.ntp * c.op.CB;
    c.off_x = take(sizeof(float2) * nr);
    c.off_p = take(sizeof(float2) * nr);
    c.off_s = take(sizeof(float2) * nr);
    c.off_r = take(sizeof(float2) * nk);
    c.off_q = take(sizeof(float2) * nk);
    c.off_part = take(sizeof(double) * kNormBlocks);
    c.off_scal = take(sizeof(double) * 4);  // gamma[2] (ping-pong), ||q||^2, spare
    c.bytes = off;
    *C = c;
    return AEXP_OK;
}

cudaError_t norm2_f64(const float2 *w, size_t n, double *partial, double *out, cudaStream_t st) {
    norm2_partial_kernel<<<kNormBlocks, kNormThreads, 0, st>>>(w, n, partial);
    norm2_final_kernel<<<1, kNormBlocks, 0, st>>>(partial, out);
    return cudaGetLastError();
}

cudaError_t cgls_issue(const aexp_problem *p, const CglsLayout &C, const float2 *y, int iters, float2 *x_out,
                       char *ws, cudaStream_t st) {
    const OpLayout &L = C.op;
    const size_t nr = (size_t)L.nr, nk = (size_t)L.ntp * L.CB;
    float2 *x = (float2 *)(ws + C.off_x), *pv = (float2 *)(ws + C.off_p), *s = (float2 *)(ws + C.off_s);
    float2 *r = (float2 *)(ws + C.off_r), *q = (float2 *)(ws + C.off_q);
    double *part = (double *)(ws + C.off_part), *scal = (double *)(ws + C.off_scal);
    double *qq = scal + 2;

    CK(op_prepare(p, L, ws, st));
    CK(cudaMemsetAsync(x, 0, sizeof(float2) * nr, st));
    CK(op_transpose_y(L, y, r, st));  // r_0 = y (sample-major, zero padded)
    CK(op_apply_adjoint(L, r, ws, st));
    CK(op_adjoint_reduce(L, ws, s, st));  // s_0 = A^H y
    copy_kernel<<<grid_for(nr), 256, 0, st>>>(pv, s, nr);
    CK(norm2_f64(s, nr, part, &scal[0], st));
    for (int k = 0; k < iters; ++k) {
        double *g = &scal[k & 1], *g_next = &scal[(k + 1) & 1];
        CK(op_apply_forward(L, pv, ws, st));
        CK(op_reduce_forward_residual(L, ws, nullptr, q, st));  // q = A p
        CK(norm2_f64(q, nk, part, qq, st));
        axpy_ratio_kernel<<<grid_for(nr), 256, 0, st>>>(x, pv, nr, g, qq, 1.f);   // x += alpha p
        axpy_ratio_kernel<<<grid_for(nk), 256, 0, st>>>(r, q, nk, g, qq, -1.f);   // r -= alpha q
        CK(op_apply_adjoint(L, r, ws, st));
        CK(op_adjoint_reduce(L, ws, s, st));  // s = A^H r
        CK(norm2_f64(s, nr, part, g_next, st));
        xpay_ratio_kernel<<<grid_for(nr), 256, 0, st>>>(pv, s, nr, g_next, g);  // p = s + beta p
    }
    CK(cudaMemcpyAsync(x_out, x, sizeof(float2) * nr, cudaMemcpyDeviceToDevice, st));
    return cudaGetLastError();
}

}  // namespace aexp
