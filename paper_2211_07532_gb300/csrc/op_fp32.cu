// A_exp and A_exp^H on FP32 CUDA cores (Eq. 1; Sec. 1 expanded model with B0 and
// spherical-harmonic terms).
//
// Forward (y_c(t) = sum_r exp(-i phi) S_c(r) x(r)):  a block owns 128*MT samples
// (MT per thread, coefficients k_l(t)/2pi held in registers) and a run of 8x8 voxel
// tiles.  Per tile, one bulk (TMA) copy brings the tile's basis offsets dh[64][LP] and
// coil-weighted image b[64][CB] into shared memory (double buffered, mbarrier
// completion).  Every thread then walks the 64 voxels: LP FMAs of local phase on top
// of the tabulated reference phase, reduction to [-1/2, 1/2] turns, one MUFU sincos,
// and 4 FMAs per coil into register accumulators.  Partial sums per run of tiles are
// reduced afterwards in a fixed order (deterministic).
//
// The FMAs are issued as packed FP32x2 (FFMA2: two lanes of one instruction, each rounded
// like fmaf): two coils per instruction in the contractions, even/odd terms per instruction
// in the phase sums (the one-voxel-per-thread adjoint at 32 coils keeps two such pairs of
// partial phase sums, to halve the dependent latency).  This halves the
// instruction count of the FMA work, which otherwise leaves the issue slots, not the FMA
// pipe, as the limit.  The coil-weighted image is stored as coil pairs
// (re c, re c+1, im c, im c+1) so that one 16-byte load yields both packed operands; the
// adjoint permutes each staged block of y into the same order in shared memory.
//
// Adjoint (x(r) = sum_c conj S_c(r) sum_t exp(+i phi) y_c(t)):  a block owns two tiles
// (one voxel per thread, basis offsets in registers) and a run of samples, staged by
// bulk copies of k/2pi [TS][LP], y [TS][CB] and the two tiles' reference phases.
// Per-coil sums stay in registers; the coil combination with conj(S_c) happens once
// per voxel at the end of the run.
#include "aexp_internal.cuh"

namespace aexp {

namespace {

constexpr float kTwoPi = 6.283185307179586f;

__device__ __forceinline__ float2 ffma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 dup2(float v) { return make_float2(v, v); }

// Smallest of the per-voxel work: phase in turns -> (cos, sin) of 2 pi * frac.
__device__ __forceinline__ void turns_sincos(float ph, float &s, float &c) {
    ph = ph - rintf(ph);
    __sincosf(ph * kTwoPi, &s, &c);
}

template <int CB, int LP, int MT>
__global__ void __launch_bounds__(kFwdThreads, MT == 1 ? 4 : 2)
    fwd_fp32_kernel(const float *__restrict__ khi_l, const float *__restrict__ f0, const float *__restrict__ dh,
                    const float2 *__restrict__ b, float2 *__restrict__ part, int ntp, int ntiles,
                    int tiles_per_split, int *status) {
    constexpr unsigned DH_BYTES = kTileVox * LP * sizeof(float);
    constexpr unsigned B_BYTES = kTileVox * CB * sizeof(float2);
    constexpr unsigned STAGE = DH_BYTES + B_BYTES;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar[2];

    const int tid = threadIdx.x;
    const int split = blockIdx.y;
    const int tile0 = split * tiles_per_split;
    const int ntl = min(ntiles, tile0 + tiles_per_split) - tile0;
    const int tbase = blockIdx.x * kFwdThreads * MT + tid;

    float2 kh[MT][LP / 2];  // (even term, odd term)
#pragma unroll
    for (int j = 0; j < MT; ++j)
#pragma unroll
        for (int l = 0; l < LP / 2; ++l)
            kh[j][l] = make_float2(khi_l[(size_t)(2 * l) * ntp + tbase + j * kFwdThreads],
                                   khi_l[(size_t)(2 * l + 1) * ntp + tbase + j * kFwdThreads]);

    float2 are[MT][CB / 2], aim[MT][CB / 2];  // coils (2q, 2q+1)
#pragma unroll
    for (int j = 0; j < MT; ++j)
#pragma unroll
        for (int q = 0; q < CB / 2; ++q) are[j][q] = aim[j][q] = make_float2(0.f, 0.f);

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto issue = [&](int i) {
        int buf = i & 1;
        unsigned char *dst = smem + buf * STAGE;
        size_t tile = (size_t)(tile0 + i);
        mbar_arrive_expect_tx(&bar[buf], STAGE);
        bulk_g2s(dst, dh + tile * kTileVox * LP, DH_BYTES, &bar[buf]);
        bulk_g2s(dst + DH_BYTES, b + tile * kTileVox * CB, B_BYTES, &bar[buf]);
    };
    if (tid == 0) {
        if (ntl > 0) issue(0);
        if (ntl > 1) issue(1);
    }

    for (int i = 0; i < ntl; ++i) {
        const int buf = i & 1;
        bool ok = mbar_wait_bounded(&bar[buf], (i >> 1) & 1, status);
        if (__syncthreads_or(!ok)) {
            // a copy never completed: give in-flight copies a bounded chance to land, then leave
            if (tid == 0)
                for (int k = i; k < min(ntl, i + 2); ++k) mbar_wait_bounded(&bar[k & 1], (k >> 1) & 1, status);
            __syncthreads();
            return;
        }
        const float4 *sdh = reinterpret_cast<const float4 *>(smem + buf * STAGE);
        const float4 *sb = reinterpret_cast<const float4 *>(smem + buf * STAGE + DH_BYTES);
        float f[MT];
#pragma unroll
        for (int j = 0; j < MT; ++j) f[j] = f0[(size_t)(tile0 + i) * ntp + tbase + j * kFwdThreads];

#pragma unroll 2
        for (int v = 0; v < kTileVox; ++v) {
            float2 d[LP / 2];
#pragma unroll
            for (int q = 0; q < LP / 4; ++q) {
                float4 w = sdh[v * (LP / 4) + q];
                d[2 * q] = make_float2(w.x, w.y);
                d[2 * q + 1] = make_float2(w.z, w.w);
            }
            float cr[MT], sr[MT];
#pragma unroll
            for (int j = 0; j < MT; ++j) {
                // even and odd terms in the two lanes: two interleaved chains
                float2 p = make_float2(f[j], 0.f);
#pragma unroll
                for (int l = 0; l < LP / 2; ++l) p = ffma2(kh[j][l], d[l], p);
                turns_sincos(p.x + p.y, sr[j], cr[j]);
            }
            // E = cos - i sin;  acc += E * b
#pragma unroll
            for (int q = 0; q < CB / 2; ++q) {
                const float4 bb = sb[v * (CB / 2) + q];  // (re 2q, re 2q+1, im 2q, im 2q+1)
                const float2 bre = make_float2(bb.x, bb.y), bim = make_float2(bb.z, bb.w);
#pragma unroll
                for (int j = 0; j < MT; ++j) {
                    are[j][q] = ffma2(dup2(cr[j]), bre, are[j][q]);
                    are[j][q] = ffma2(dup2(sr[j]), bim, are[j][q]);
                    aim[j][q] = ffma2(dup2(cr[j]), bim, aim[j][q]);
                    aim[j][q] = ffma2(dup2(-sr[j]), bre, aim[j][q]);
                }
            }
        }
        __syncthreads();
        if (tid == 0 && i + 2 < ntl) issue(i + 2);
    }

#pragma unroll
    for (int j = 0; j < MT; ++j) {
        float4 *dst = reinterpret_cast<float4 *>(part + ((size_t)split * ntp + tbase + j * kFwdThreads) * CB);
#pragma unroll
        for (int q = 0; q < CB / 2; ++q) dst[q] = make_float4(are[j][q].x, aim[j][q].x, are[j][q].y, aim[j][q].y);
    }
}

template <int CB, int LP, int MR>
__global__ void __launch_bounds__(kAdjThreads, MR == 1 ? 4 : 2)
    adj_fp32_kernel(const float *__restrict__ khi_t, const float *__restrict__ f0, const float *__restrict__ dh,
                    const float2 *__restrict__ Sp, const float2 *__restrict__ yt, float2 *__restrict__ part, int ntp,
                    int ntiles, int t_per_split, int *status) {
    constexpr int TS = kAdjStageT;
    constexpr int NT = 2 * MR;  // tiles per block
    constexpr unsigned K_BYTES = TS * LP * sizeof(float);
    constexpr unsigned Y_BYTES = TS * CB * sizeof(float2);
    constexpr unsigned F_BYTES = TS * sizeof(float);
    constexpr unsigned STAGE = K_BYTES + Y_BYTES + NT * F_BYTES;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ uint64_t bar[2];

    const int tid = threadIdx.x;
    const int split = blockIdx.y;
    const int tile_base = NT * blockIdx.x;
    const int t0 = split * t_per_split;
    const int nst = (min(ntp, t0 + t_per_split) - t0) / TS;

    float2 d[MR][LP / 2];  // (even term, odd term)
    bool valid[MR];
    int pv[MR];
#pragma unroll
    for (int m = 0; m < MR; ++m) {
        pv[m] = blockIdx.x * kAdjThreads * MR + m * kAdjThreads + tid;
        valid[m] = pv[m] / kTileVox < ntiles;
        const float4 *src = reinterpret_cast<const float4 *>(dh + (size_t)(valid[m] ? pv[m] : 0) * LP);
#pragma unroll
        for (int q = 0; q < LP / 4; ++q) {
            float4 w = src[q];
            d[m][2 * q] = valid[m] ? make_float2(w.x, w.y) : make_float2(0.f, 0.f);
            d[m][2 * q + 1] = valid[m] ? make_float2(w.z, w.w) : make_float2(0.f, 0.f);
        }
    }
    float2 ure[MR][CB / 2], uim[MR][CB / 2];  // coils (2q, 2q+1)
#pragma unroll
    for (int m = 0; m < MR; ++m)
#pragma unroll
        for (int q = 0; q < CB / 2; ++q) ure[m][q] = uim[m][q] = make_float2(0.f, 0.f);

    if (tid == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        fence_mbar_init();
    }
    __syncthreads();

    auto issue = [&](int i) {
        int buf = i & 1;
        unsigned char *dst = smem + buf * STAGE;
        size_t ts = (size_t)t0 + (size_t)i * TS;
        mbar_arrive_expect_tx(&bar[buf], STAGE);
        bulk_g2s(dst, khi_t + ts * LP, K_BYTES, &bar[buf]);
        bulk_g2s(dst + K_BYTES, yt + ts * CB, Y_BYTES, &bar[buf]);
        for (int q = 0; q < NT; ++q) {
            // tiles past the end (last block) reuse a valid row; their results are discarded
            int tile = min(tile_base + q, ntiles - 1);
            bulk_g2s(dst + K_BYTES + Y_BYTES + q * F_BYTES, f0 + (size_t)tile * ntp + ts, F_BYTES, &bar[buf]);
        }
    };
    if (tid == 0) {
        if (nst > 0) issue(0);
        if (nst > 1) issue(1);
    }

    for (int i = 0; i < nst; ++i) {
        const int buf = i & 1;
        bool ok = mbar_wait_bounded(&bar[buf], (i >> 1) & 1, status);
        if (__syncthreads_or(!ok)) {
            if (tid == 0)
                for (int k = i; k < min(nst, i + 2); ++k) mbar_wait_bounded(&bar[k & 1], (k >> 1) & 1, status);
            __syncthreads();
            return;
        }
        const float4 *sk = reinterpret_cast<const float4 *>(smem + buf * STAGE);
        float4 *sy = reinterpret_cast<float4 *>(smem + buf * STAGE + K_BYTES);
        const float *sf = reinterpret_cast<const float *>(smem + buf * STAGE + K_BYTES + Y_BYTES);
        // the staged y rows to coil-pair planar order (re c, re c+1, im c, im c+1), in place, so that
        // one 16-byte load yields both packed operands (each thread permutes its own 16-byte words)
        for (int k = tid; k < TS * CB / 2; k += kAdjThreads) {
            const float4 w = sy[k];
            sy[k] = make_float4(w.x, w.z, w.y, w.w);
        }
        __syncthreads();

        // phase + sincos of sample s for each of this thread's voxels
        auto encode = [&](int s, float *cs, float *sn) {
#pragma unroll
            for (int m = 0; m < MR; ++m) {
                // the voxel's tile within the block is uniform per warp: 2m + tid/64
                float2 p = make_float2(sf[(2 * m + tid / kTileVox) * TS + s], 0.f);
                if constexpr (MR == 1) {
                    // one voxel per thread: a second pair of chains halves the dependent latency
                    float2 pb = make_float2(0.f, 0.f);
#pragma unroll
                    for (int q = 0; q < LP / 4; ++q) {
                        float4 kk = sk[s * (LP / 4) + q];
                        p = ffma2(make_float2(kk.x, kk.y), d[m][2 * q], p);
                        pb = ffma2(make_float2(kk.z, kk.w), d[m][2 * q + 1], pb);
                    }
                    turns_sincos((p.x + p.y) + (pb.x + pb.y), sn[m], cs[m]);
                } else {
#pragma unroll
                    for (int q = 0; q < LP / 4; ++q) {
                        float4 kk = sk[s * (LP / 4) + q];
                        p = ffma2(make_float2(kk.x, kk.y), d[m][2 * q], p);
                        p = ffma2(make_float2(kk.z, kk.w), d[m][2 * q + 1], p);
                    }
                    turns_sincos(p.x + p.y, sn[m], cs[m]);
                }
            }
        };
        // software pipeline as in the forward kernel: sample s+1 is encoded before the
        // contraction of sample s
        float cnx[MR], snx[MR];
        encode(0, cnx, snx);
#pragma unroll 2
        for (int s = 0; s < TS; ++s) {
            float cs[MR], sn[MR];
#pragma unroll
            for (int m = 0; m < MR; ++m) {
                cs[m] = cnx[m];
                sn[m] = snx[m];
            }
            if (s + 1 < TS) encode(s + 1, cnx, snx);
            // conj(E) = cos + i sin;  u += conj(E) * y
#pragma unroll
            for (int q = 0; q < CB / 2; ++q) {
                const float4 yy = sy[s * (CB / 2) + q];  // (re 2q, re 2q+1, im 2q, im 2q+1)
                const float2 yre = make_float2(yy.x, yy.y), yim = make_float2(yy.z, yy.w);
#pragma unroll
                for (int m = 0; m < MR; ++m) {
                    ure[m][q] = ffma2(dup2(cs[m]), yre, ure[m][q]);
                    ure[m][q] = ffma2(dup2(-sn[m]), yim, ure[m][q]);
                    uim[m][q] = ffma2(dup2(cs[m]), yim, uim[m][q]);
                    uim[m][q] = ffma2(dup2(sn[m]), yre, uim[m][q]);
                }
            }
        }
        // the permuted words were written through the generic proxy; the bulk copy that refills
        // this buffer writes through the async proxy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (tid == 0 && i + 2 < nst) issue(i + 2);
    }

#pragma unroll
    for (int m = 0; m < MR; ++m) {
        if (!valid[m]) continue;
        const float4 *s4 = reinterpret_cast<const float4 *>(Sp + (size_t)pv[m] * CB);
        float xr = 0.f, xi = 0.f;
#pragma unroll
        for (int q = 0; q < CB / 2; ++q) {
            float4 sv = s4[q];
            // conj(S) * u
            xr = fmaf(sv.x, ure[m][q].x, xr);
            xr = fmaf(sv.y, uim[m][q].x, xr);
            xi = fmaf(sv.x, uim[m][q].x, xi);
            xi = fmaf(-sv.y, ure[m][q].x, xi);
            xr = fmaf(sv.z, ure[m][q].y, xr);
            xr = fmaf(sv.w, uim[m][q].y, xr);
            xi = fmaf(sv.z, uim[m][q].y, xi);
            xi = fmaf(-sv.w, ure[m][q].y, xi);
        }
        part[(size_t)split * (size_t)(ntiles * kTileVox) + pv[m]] = make_float2(xr, xi);
    }
}

// ---- reductions of the partial sums (fixed order => deterministic) ----

__global__ void fwd_reduce_public_kernel(const float2 *part, int splits, int ntp, int CB, int nt, int nc, float2 *y) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)nt * CB) return;
    int t = (int)(i / CB), c = (int)(i % CB);
    if (c >= nc) return;
    float2 s = make_float2(0.f, 0.f);
    for (int k = 0; k < splits; ++k) {
        float2 v = part[((size_t)k * ntp + t) * CB + c];
        s.x += v.x;
        s.y += v.y;
    }
    y[(size_t)c * nt + t] = s;
}

__global__ void fwd_reduce_residual_kernel(const float2 *part, int splits, int ntp, int CB, int nt, int nc,
                                           const float2 *ymeas, float2 *rt) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)ntp * CB) return;
    int t = (int)(i / CB), c = (int)(i % CB);
    float2 s = make_float2(0.f, 0.f);
    if (t < nt && c < nc) {
        for (int k = 0; k < splits; ++k) {
            float2 v = part[((size_t)k * ntp + t) * CB + c];
            s.x += v.x;
            s.y += v.y;
        }
        if (ymeas) {
            s.x -= ymeas[i].x;
            s.y -= ymeas[i].y;
        }
    }
    rt[i] = s;
}

__global__ void adj_reduce_kernel(const float2 *part, int splits, int nr_pad, int nx, int ny, int ntx,
                                  const WsHeader *hdr, const float2 *z, float2 *out) {
    int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nx * ny) return;
    int ix = r % nx, iy = r / nx;
    int p = ((iy / kTileSide) * ntx + ix / kTileSide) * kTileVox + (iy % kTileSide) * kTileSide + ix % kTileSide;
    float2 s = make_float2(0.f, 0.f);
    for (int k = 0; k < splits; ++k) {
        float2 v = part[(size_t)k * nr_pad + p];
        s.x += v.x;
        s.y += v.y;
    }
    if (z) {  // gradient step of Eq. (1): v = z - (1/L_f) * 2 A^H (A z - y)
        float step = (float)(2.0 / hdr->lipschitz);
        float2 zv = z[r];
        s.x = zv.x - step * s.x;
        s.y = zv.y - step * s.y;
    }
    out[r] = s;
}

// ---- dispatch over the compile-time coil / term paddings ----

template <int CB, int LP, int MT>
cudaError_t launch_fwd_mt(const OpLayout &L, char *ws, cudaStream_t st) {
    constexpr unsigned STAGE = kTileVox * LP * sizeof(float) + kTileVox * CB * sizeof(float2);
    auto kern = fwd_fp32_kernel<CB, LP, MT>;
    {  // always opted in: the static barriers count against the 48 KB default too
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * STAGE);
        if (e != cudaSuccess) return e;
    }
    WsHeader *hdr = (WsHeader *)(ws + L.off_hdr);
    kern<<<dim3(L.fwd_tblocks, L.fwd_splits), kFwdThreads, 2 * STAGE, st>>>(
        (const float *)(ws + L.off_khi_l), (const float *)(ws + L.off_f0), (const float *)(ws + L.off_dh),
        (const float2 *)(ws + L.off_b), (float2 *)(ws + L.off_fpart), L.ntp, L.ntiles, L.fwd_tiles_per_split,
        &hdr->status);
    return cudaGetLastError();
}

template <int CB, int LP, int MR>
cudaError_t launch_adj_mr(const OpLayout &L, const float2 *yt, char *ws, cudaStream_t st) {
    constexpr unsigned STAGE = kAdjStageT * (LP * sizeof(float) + CB * sizeof(float2) + 2 * MR * sizeof(float));
    auto kern = adj_fp32_kernel<CB, LP, MR>;
    {  // always opted in: the static barriers count against the 48 KB default too
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * STAGE);
        if (e != cudaSuccess) return e;
    }
    WsHeader *hdr = (WsHeader *)(ws + L.off_hdr);
    kern<<<dim3(L.adj_vblocks, L.adj_splits), kAdjThreads, 2 * STAGE, st>>>(
        (const float *)(ws + L.off_khi_t), (const float *)(ws + L.off_f0), (const float *)(ws + L.off_dh),
        (const float2 *)(ws + L.off_S), yt, (float2 *)(ws + L.off_apart), L.ntp, L.ntiles, L.adj_t_per_split,
        &hdr->status);
    return cudaGetLastError();
}

// The layout's register blocking (fwd_mt / adj_mr): the default of the coil padding, or the
// alternative tiling at 32 coils.
template <int CB, int LP>
cudaError_t launch_fwd(const OpLayout &L, char *ws, cudaStream_t st) {
    if constexpr (CB == 32 && fwd_mt_for(32) != kFp32AltBlocking)
        if (L.fwd_mt == kFp32AltBlocking) return launch_fwd_mt<CB, LP, kFp32AltBlocking>(L, ws, st);
    return launch_fwd_mt<CB, LP, fwd_mt_for(CB)>(L, ws, st);
}

template <int CB, int LP>
cudaError_t launch_adj(const OpLayout &L, const float2 *yt, char *ws, cudaStream_t st) {
    if constexpr (CB == 32 && adj_mr_for(32) != kFp32AltBlocking)
        if (L.adj_mr == kFp32AltBlocking) return launch_adj_mr<CB, LP, kFp32AltBlocking>(L, yt, ws, st);
    return launch_adj_mr<CB, LP, adj_mr_for(CB)>(L, yt, ws, st);
}

#define AEXP_DISPATCH_LP(FN, CBV, ...)                   \
    switch (L.LP) {                                      \
        case 4: return FN<CBV, 4>(__VA_ARGS__);          \
        case 8: return FN<CBV, 8>(__VA_ARGS__);          \
        case 12: return FN<CBV, 12>(__VA_ARGS__);        \
        case 20: return FN<CBV, 20>(__VA_ARGS__);        \
        default: return FN<CBV, 32>(__VA_ARGS__);        \
    }

#define AEXP_DISPATCH(FN, ...)                                   \
    switch (L.CB) {                                              \
        case 4: AEXP_DISPATCH_LP(FN, 4, __VA_ARGS__)             \
        case 8: AEXP_DISPATCH_LP(FN, 8, __VA_ARGS__)             \
        case 16: AEXP_DISPATCH_LP(FN, 16, __VA_ARGS__)           \
        case 20: AEXP_DISPATCH_LP(FN, 20, __VA_ARGS__)           \
        default: AEXP_DISPATCH_LP(FN, 32, __VA_ARGS__)           \
    }

}  // namespace

cudaError_t op_forward_core(const OpLayout &L, char *ws, cudaStream_t st) {
    AEXP_DISPATCH(launch_fwd, L, ws, st)
}

cudaError_t op_adjoint_core(const OpLayout &L, const float2 *yt, char *ws, cudaStream_t st) {
    AEXP_DISPATCH(launch_adj, L, yt, ws, st)
}

cudaError_t op_forward_reduce_public(const OpLayout &L, char *ws, float2 *y, cudaStream_t st) {
    size_t n = (size_t)L.nt * L.CB;
    fwd_reduce_public_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        (const float2 *)(ws + L.off_fpart), L.fwd_splits, L.ntp, L.CB, L.nt, L.nc, y);
    return cudaGetLastError();
}

cudaError_t op_forward_reduce_residual(const OpLayout &L, char *ws, const float2 *ymeas_t, float2 *rt,
                                       cudaStream_t st) {
    size_t n = (size_t)L.ntp * L.CB;
    fwd_reduce_residual_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        (const float2 *)(ws + L.off_fpart), L.fwd_splits, L.ntp, L.CB, L.nt, L.nc, ymeas_t, rt);
    return cudaGetLastError();
}

cudaError_t op_adjoint_reduce(const OpLayout &L, char *ws, float2 *out, cudaStream_t st) {
    adj_reduce_kernel<<<cdiv(L.nr, 256), 256, 0, st>>>((const float2 *)(ws + L.off_apart), L.adj_splits, L.nr_pad,
                                                      L.nx, L.ny, L.ntx, (const WsHeader *)(ws + L.off_hdr),
                                                      nullptr, out);
    return cudaGetLastError();
}

cudaError_t op_adjoint_reduce_step(const OpLayout &L, char *ws, const float2 *z, float2 *out, cudaStream_t st) {
    adj_reduce_kernel<<<cdiv(L.nr, 256), 256, 0, st>>>((const float2 *)(ws + L.off_apart), L.adj_splits, L.nr_pad,
                                                      L.nx, L.ny, L.ntx, (const WsHeader *)(ws + L.off_hdr), z,
                                                      out);
    return cudaGetLastError();
}

}  // namespace aexp
