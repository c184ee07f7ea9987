// A_exp and A_exp^H on the tcgen05 tensor cores (BF16 encoding tile, FP32 accumulation).
//
// The complex contraction is embedded in a real GEMM whose A operand is generated on
// the fly and never leaves shared memory:
//   forward   Y[t][n] = sum_k A[t][k] B[n][k],  A[t][2v] = cos phi, A[t][2v+1] = -sin phi,
//             B[c][2v] = Re b_c(v), B[c][2v+1] = -Im b_c(v), B[C+c][2v] = Im b_c, B[C+c][2v+1] = Re b_c
//             so that Y[t][c] = Re y_c(t) and Y[t][C+c] = Im y_c(t) (E = cos - i sin);
//   adjoint   U[r][n] = sum_k A[r][k] B[n][k],  A[r][2s] = cos phi, A[r][2s+1] = sin phi,
//             B[c][2s] = Re y_c, B[c][2s+1] = -Im y_c, B[C+c][2s] = Im y_c, B[C+c][2s+1] = Re y_c,
//             so that U[r][c] + i U[r][C+c] = sum_t conj(E) y_c(t); the coil combination with
//             conj(S_c(r)) runs in the epilogue.
// M = 128 rows per work item, N = 2C (16, 32 or 64), K = 128 per stage (64 voxels or 64
// samples), issued as 8 MMAs of K = 16.
//
// The kernels are persistent: one CTA per SM pulls work items (problem, row block, split)
// from an atomic counter, so one launch covers any ragged batch of problems described by
// a device table of ProbDesc (all with the same padded coil and term counts).  A stage
// counter runs across items, so the mbarrier phases and the staged operands flow from one
// item into the next.
//
// CTA = 16 generator warps + 1 MMA/producer warp.  Generators compute the FP32 phase
// (tabulated reference phase + local offset, as in the CUDA-core kernels), reduce it to
// [-1/2, 1/2] turns, take one MUFU sincos, round to BF16 and store 16-byte chunks straight
// into the 128B-swizzled K-major layout; each thread owns 2 rows x 8 columns.  The producer
// warp brings the packed B tile (plus basis offsets or coefficient rows and reference
// phases) with bulk TMA copies up to kNB - 1 tiles ahead, issues the MMAs from one thread,
// and two tcgen05.commit per tile release the A and B stages.  Every wait is bounded; on a
// timeout the CTA records AEXP_ERR_DEVICE_TIMEOUT, drains its MMAs, frees TMEM and exits.
#include <cuda_bf16.h>

#include <algorithm>

#include "aexp_internal.cuh"
#include "tc_ptx.cuh"

namespace aexp {

namespace {

constexpr int kTcGen = 512;              // generator threads (16 warps)
constexpr int kTcThreads = kTcGen + 32;  // + MMA/producer warp
constexpr int kProdWarp = kTcGen / 32;
constexpr int kRows = 128;               // M
constexpr int kCols = 64;                // voxels (forward) or samples (adjoint) per stage
constexpr int kA_BYTES = kRows * kCols * 2 * 2;  // 128 rows x 128 bf16 = 32 KB
constexpr float kTwoPi = 6.283185307179586f;
constexpr int kSpin = 1 << 22;
constexpr int kNB = 4;  // staged B tiles

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t *>(&v);
}

// Bounded wait that also gives up as soon as another thread of the CTA has aborted.
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, unsigned parity, volatile int *abort_flag,
                                              int *status) {
    for (int i = 0; i < kSpin; ++i) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((i & 255) == 255 && *abort_flag) return false;
    }
    *abort_flag = 1;
    set_status(status, AEXP_ERR_DEVICE_TIMEOUT);
    return false;
}

__device__ __forceinline__ uint32_t align1024(uint32_t a) { return (a + 1023u) & ~1023u; }

__device__ __forceinline__ int find_problem(const int *item_off, int nprob, int item) {
    int lo = 0, hi = nprob - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (item_off[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Shared state of a persistent tensor-core CTA.
struct TcShared {
    uint64_t bfull[kNB], bfree[kNB], afull[2], afree[2];
    uint32_t tmem_base;
    int abort_flag;
    int item[2], stop[2];
};

__device__ __forceinline__ void tc_setup(TcShared &sh, int tid, int warp, uint32_t ncols) {
    if (tid == 0) {
        for (int s = 0; s < kNB; ++s) {
            mbar_init(&sh.bfull[s], 1);
            mbar_init(&sh.bfree[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&sh.afull[s], kTcGen);
            mbar_init(&sh.afree[s], 1);
        }
        sh.abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == kProdWarp) {
        tc::tmem_alloc(&sh.tmem_base, ncols);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

// Next work item, the same for every thread of the CTA (two slots: a thread still reading
// one slot never races the write of the other); false when the queue is empty or aborted.
__device__ __forceinline__ bool tc_next_item(TcShared &sh, int tid, int iter, int *counter, int total, int &item) {
    const int slot = iter & 1;
    if (tid == 0) {
        int it = atomicAdd(counter, 1);
        sh.item[slot] = it;
        sh.stop[slot] = (it >= total) || sh.abort_flag;
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    item = sh.item[slot];
    return !sh.stop[slot];
}

__device__ __forceinline__ void tc_teardown(TcShared &sh, int warp, uint32_t ncols, int last_issued, int *status) {
    if (warp == kProdWarp && (threadIdx.x & 31) == 0 && last_issued >= 0)
        mbar_wait_bounded(&sh.afree[last_issued & 1], (last_issued >> 1) & 1, status);  // drain
    tc::fence_before_sync();
    __syncthreads();
    if (warp == kProdWarp) {
        tc::fence_after_sync();
        tc::tmem_dealloc(sh.tmem_base, ncols);
    }
}

// Issue the 8 MMAs of one stage and commit both stage barriers.
template <int N>
__device__ __forceinline__ void tc_mma_stage(TcShared &sh, uint32_t tmem, const unsigned char *A,
                                             const unsigned char *B, bool first, int sa, int sb) {
    constexpr uint32_t IDESC = tc::idesc_f16(kRows, N, 1);
    const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
        const uint32_t koff = (uint32_t)((kk >> 2) * (kRows * 128) + (kk & 3) * 32);
        const uint32_t kofb = (uint32_t)((kk >> 2) * (N * 128) + (kk & 3) * 32);
        tc::mma_f16(tmem, tc::sdesc_k128(a0 + koff), tc::sdesc_k128(b0 + kofb), IDESC, !(first && kk == 0));
    }
    tc::mma_commit(&sh.afree[sa]);
    tc::mma_commit(&sh.bfree[sb]);
}

// ---------------------------------------------------------------------------
// Forward: item = (problem, block of 128 samples, run of voxel tiles)
// ---------------------------------------------------------------------------
template <int CB, int LP>
__global__ void __launch_bounds__(kTcThreads, 1)
    fwd_tc_kernel(const ProbDesc *__restrict__ pd, const int *__restrict__ item_off, int nprob, int *counter) {
    constexpr int N = 2 * CB;
    constexpr unsigned B_BYTES = N * 256;  // N rows x 128 bf16
    constexpr unsigned DH_BYTES = kTileVox * LP * 4;
    constexpr unsigned F_BYTES = kRows * 4;
    // one staged tile (B | dh | f0 rows): S_DATA bytes arrive per stage; the stride S_BYTES
    // keeps every B tile 1024-byte aligned
    constexpr unsigned S_DATA = B_BYTES + DH_BYTES + F_BYTES;
    constexpr unsigned S_BYTES = (S_DATA + 1023u) & ~1023u;
    constexpr unsigned TMEM_COLS = N <= 32 ? 32 : 64;

    extern __shared__ unsigned char smem_raw[];
    __shared__ TcShared sh;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const uint32_t sbase = align1024(smem_u32(smem_raw));
    unsigned char *gbase = smem_raw + (sbase - smem_u32(smem_raw));
    unsigned char *A[2] = {gbase, gbase + kA_BYTES};
    unsigned char *stage0 = gbase + 2 * kA_BYTES;
    const int total = item_off[nprob];

    tc_setup(sh, tid, warp, TMEM_COLS);
    const uint32_t tmem = sh.tmem_base;
    int gs = 0;            // stages (tiles) this CTA has processed
    int last_issued = -1;  // producer: last stage whose MMAs were committed

    int item;
    for (int iter = 0; tc_next_item(sh, tid, iter, counter, total, item); ++iter) {
        const int q = find_problem(item_off, nprob, item);
        const ProbDesc &P = pd[q];
        int *status = &P.hdr->status;
        const int li = item - item_off[q];
        const int split = li % P.fwd_splits;
        const int tbase = (li / P.fwd_splits) * kRows;
        const int tile0 = split * P.fwd_tps;
        const int ntl = max(0, min(P.ntiles, tile0 + P.fwd_tps) - tile0);
        const int ntp = P.ntp;

        if (warp == kProdWarp) {
            if (tid == kTcGen) {
                auto load = [&](int it) {
                    const int sb = (gs + it) % kNB;
                    unsigned char *dst = stage0 + sb * S_BYTES;
                    const size_t tile = (size_t)(tile0 + it);
                    mbar_arrive_expect_tx(&sh.bfull[sb], S_DATA);
                    bulk_g2s(dst, P.bpk + tile * B_BYTES, B_BYTES, &sh.bfull[sb]);
                    bulk_g2s(dst + B_BYTES, P.dh + tile * kTileVox * LP, DH_BYTES, &sh.bfull[sb]);
                    bulk_g2s(dst + B_BYTES + DH_BYTES, P.f0 + tile * ntp + tbase, F_BYTES, &sh.bfull[sb]);
                };
                for (int j = 0; j < min(kNB, ntl); ++j) load(j);
                for (int it = 0; it < ntl; ++it) {
                    const int g = gs + it, sa = g & 1, sb = g % kNB;
                    if (!wait_or_abort(&sh.afull[sa], (g >> 1) & 1, &sh.abort_flag, status)) break;
                    if (!wait_or_abort(&sh.bfull[sb], (g / kNB) & 1, &sh.abort_flag, status)) break;
                    tc::fence_after_sync();
                    tc_mma_stage<N>(sh, tmem, A[sa], stage0 + sb * S_BYTES, it == 0, sa, sb);
                    last_issued = g;
                    if (it + kNB < ntl) {
                        if (!wait_or_abort(&sh.bfree[sb], (g / kNB) & 1, &sh.abort_flag, status)) break;
                        load(it + kNB);
                    }
                }
            }
        } else {
            // generator: warp w owns chunk columns (w & 7) and (w & 7) + 8, lane g owns rows
            // r0 = 64 (w >> 3) + g and r0 + 32 with their coefficients in registers
            const int jp = warp & 7;
            const int r0 = 64 * (warp >> 3) + (tid & 31);
            float k[2][LP];
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int q4 = 0; q4 < LP / 4; ++q4) {
                    float4 w = reinterpret_cast<const float4 *>(P.khi_t + (size_t)(tbase + r0 + 32 * i) * LP)[q4];
                    k[i][4 * q4] = w.x;
                    k[i][4 * q4 + 1] = w.y;
                    k[i][4 * q4 + 2] = w.z;
                    k[i][4 * q4 + 3] = w.w;
                }
            for (int it = 0; it < ntl; ++it) {
                const int g = gs + it, sa = g & 1, sb = g % kNB;
                if (!wait_or_abort(&sh.bfull[sb], (g / kNB) & 1, &sh.abort_flag, status)) break;
                if (g >= 2 && !wait_or_abort(&sh.afree[sa], ((g - 2) >> 1) & 1, &sh.abort_flag, status)) break;
                const unsigned char *stg = stage0 + sb * S_BYTES;
                const float4 *DH = reinterpret_cast<const float4 *>(stg + B_BYTES);
                const float *F0 = reinterpret_cast<const float *>(stg + B_BYTES + DH_BYTES);
                float f[2];
#pragma unroll
                for (int i = 0; i < 2; ++i) f[i] = F0[r0 + 32 * i];
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const int j = jp + 8 * hh;  // chunk of 4 voxels; atom hh, swizzle column jp
                    uint32_t packed[2][4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        float d[LP];
#pragma unroll
                        for (int q4 = 0; q4 < LP / 4; ++q4) {
                            float4 w = DH[(4 * j + u) * (LP / 4) + q4];
                            d[4 * q4] = w.x;
                            d[4 * q4 + 1] = w.y;
                            d[4 * q4 + 2] = w.z;
                            d[4 * q4 + 3] = w.w;
                        }
#pragma unroll
                        for (int i = 0; i < 2; ++i) {
                            float p0 = f[i], p1 = 0.f;
#pragma unroll
                            for (int l = 0; l < LP; l += 2) {
                                p0 = fmaf(k[i][l], d[l], p0);
                                p1 = fmaf(k[i][l + 1], d[l + 1], p1);
                            }
                            float ph = p0 + p1;
                            ph = ph - rintf(ph);
                            float sn, cs;
                            __sincosf(ph * kTwoPi, &sn, &cs);
                            packed[i][u] = pack_bf16(cs, -sn);  // E = cos - i sin
                        }
                    }
                    unsigned char *atom_base = A[sa] + hh * (kRows * 128);
#pragma unroll
                    for (int i = 0; i < 2; ++i)
                        *reinterpret_cast<uint4 *>(atom_base + tc::swz128(r0 + 32 * i, jp)) =
                            make_uint4(packed[i][0], packed[i][1], packed[i][2], packed[i][3]);
                }
                tc::fence_proxy_async_smem();
                tc::mbar_arrive(&sh.afull[sa]);
            }
            // epilogue (warps 0-7): last stage's MMAs done -> TMEM -> partials (planar re | im)
            bool ok = !sh.abort_flag;
            const int gl = gs + ntl - 1;
            if (ntl > 0 && ok) ok = wait_or_abort(&sh.afree[gl & 1], (gl >> 1) & 1, &sh.abort_flag, status);
            ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-collective
            tc::fence_after_sync();
            if (warp < 8) {
                const int lane_base = 32 * (warp & 3);
                const int half = warp >> 2;
                const int t = tbase + lane_base + (tid & 31);
                float v[N / 2];
                if (ntl > 0 && ok) {
                    tc::tmem_ld<N / 2>(tmem + ((uint32_t)lane_base << 16) + (uint32_t)(half * (N / 2)), v);
                    tc::tmem_ld_wait();
                } else {
#pragma unroll
                    for (int c = 0; c < N / 2; ++c) v[c] = 0.f;
                }
                float4 *dst =
                    reinterpret_cast<float4 *>(P.fpart + ((size_t)split * ntp + t) * N + half * (N / 2));
#pragma unroll
                for (int c = 0; c < N / 8; ++c)
                    dst[c] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
            }
        }
        gs += ntl;
    }
    tc_teardown(sh, warp, TMEM_COLS, last_issued, &pd[0].hdr->status);
}

// ---------------------------------------------------------------------------
// Adjoint: item = (problem, two voxel tiles, run of 64-sample stages)
// ---------------------------------------------------------------------------
template <int CB, int LP>
__global__ void __launch_bounds__(kTcThreads, 1)
    adj_tc_kernel(const ProbDesc *__restrict__ pd, const int *__restrict__ item_off, int nprob, int *counter) {
    constexpr int N = 2 * CB;
    constexpr int TS = kCols;  // samples per stage
    constexpr unsigned B_BYTES = N * 256;
    constexpr unsigned K_BYTES = TS * LP * 4;
    constexpr unsigned F_BYTES = TS * 4;
    // B | k rows | f0 (2 tiles): S_DATA bytes arrive per stage; the stride S_BYTES keeps
    // every B tile 1024-byte aligned
    constexpr unsigned S_DATA = B_BYTES + K_BYTES + 2 * F_BYTES;
    constexpr unsigned S_BYTES = (S_DATA + 1023u) & ~1023u;
    constexpr unsigned TMEM_COLS = N <= 32 ? 32 : 64;

    extern __shared__ unsigned char smem_raw[];
    __shared__ TcShared sh;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const uint32_t sbase = align1024(smem_u32(smem_raw));
    unsigned char *gbase = smem_raw + (sbase - smem_u32(smem_raw));
    unsigned char *A[2] = {gbase, gbase + kA_BYTES};
    unsigned char *stage0 = gbase + 2 * kA_BYTES;
    const int total = item_off[nprob];

    tc_setup(sh, tid, warp, TMEM_COLS);
    const uint32_t tmem = sh.tmem_base;
    int gs = 0;
    int last_issued = -1;

    int item;
    for (int iter = 0; tc_next_item(sh, tid, iter, counter, total, item); ++iter) {
        const int q = find_problem(item_off, nprob, item);
        const ProbDesc &P = pd[q];
        int *status = &P.hdr->status;
        const int li = item - item_off[q];
        const int vb = li / P.adj_splits, split = li % P.adj_splits;
        const int ntiles = P.ntiles, ntp = P.ntp;
        const int tileA = 2 * vb;
        const int tileB = min(tileA + 1, ntiles - 1);  // odd tile count: duplicate row, discarded
        const int t0 = split * P.adj_tps;
        const int nst = max(0, (min(ntp, t0 + P.adj_tps) - t0) / TS);

        if (warp == kProdWarp) {
            if (tid == kTcGen) {
                auto load = [&](int it) {
                    const int sb = (gs + it) % kNB;
                    unsigned char *dst = stage0 + sb * S_BYTES;
                    const size_t ts = (size_t)t0 + (size_t)it * TS;
                    mbar_arrive_expect_tx(&sh.bfull[sb], S_DATA);
                    bulk_g2s(dst, P.ypk + (ts / TS) * B_BYTES, B_BYTES, &sh.bfull[sb]);
                    bulk_g2s(dst + B_BYTES, P.khi_t + ts * LP, K_BYTES, &sh.bfull[sb]);
                    bulk_g2s(dst + B_BYTES + K_BYTES, P.f0 + (size_t)tileA * ntp + ts, F_BYTES, &sh.bfull[sb]);
                    bulk_g2s(dst + B_BYTES + K_BYTES + F_BYTES, P.f0 + (size_t)tileB * ntp + ts, F_BYTES,
                             &sh.bfull[sb]);
                };
                for (int j = 0; j < min(kNB, nst); ++j) load(j);
                for (int it = 0; it < nst; ++it) {
                    const int g = gs + it, sa = g & 1, sb = g % kNB;
                    if (!wait_or_abort(&sh.afull[sa], (g >> 1) & 1, &sh.abort_flag, status)) break;
                    if (!wait_or_abort(&sh.bfull[sb], (g / kNB) & 1, &sh.abort_flag, status)) break;
                    tc::fence_after_sync();
                    tc_mma_stage<N>(sh, tmem, A[sa], stage0 + sb * S_BYTES, it == 0, sa, sb);
                    last_issued = g;
                    if (it + kNB < nst) {
                        if (!wait_or_abort(&sh.bfree[sb], (g / kNB) & 1, &sh.abort_flag, status)) break;
                        load(it + kNB);
                    }
                }
            }
        } else {
            // generator: warp w owns sample chunks (w & 7) and (w & 7) + 8 of each stage; lane g
            // owns voxel rows r0 = 64 (w >> 3) + g and r0 + 32 (both in tile w >> 3 of the item)
            // with their basis offsets in registers
            const int jp = warp & 7;
            const int th = warp >> 3;
            const int r0 = 64 * th + (tid & 31);
            float d[2][LP];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int p = vb * kRows + r0 + 32 * i;
                const bool valid = p < ntiles * kTileVox;
#pragma unroll
                for (int q4 = 0; q4 < LP / 4; ++q4) {
                    float4 w = reinterpret_cast<const float4 *>(P.dh + (size_t)(valid ? p : 0) * LP)[q4];
                    d[i][4 * q4] = valid ? w.x : 0.f;
                    d[i][4 * q4 + 1] = valid ? w.y : 0.f;
                    d[i][4 * q4 + 2] = valid ? w.z : 0.f;
                    d[i][4 * q4 + 3] = valid ? w.w : 0.f;
                }
            }
            for (int it = 0; it < nst; ++it) {
                const int g = gs + it, sa = g & 1, sb = g % kNB;
                if (!wait_or_abort(&sh.bfull[sb], (g / kNB) & 1, &sh.abort_flag, status)) break;
                if (g >= 2 && !wait_or_abort(&sh.afree[sa], ((g - 2) >> 1) & 1, &sh.abort_flag, status)) break;
                const unsigned char *stg = stage0 + sb * S_BYTES;
                const float4 *KS = reinterpret_cast<const float4 *>(stg + B_BYTES);
                const float4 *FS = reinterpret_cast<const float4 *>(stg + B_BYTES + K_BYTES);
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const int j = jp + 8 * hh;  // samples 4j..4j+3 of the stage
                    const float4 fa = FS[th * (TS / 4) + j];
                    const float fA[4] = {fa.x, fa.y, fa.z, fa.w};
                    uint32_t packed[2][4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        float kk[LP];
#pragma unroll
                        for (int q4 = 0; q4 < LP / 4; ++q4) {
                            float4 w = KS[(4 * j + u) * (LP / 4) + q4];
                            kk[4 * q4] = w.x;
                            kk[4 * q4 + 1] = w.y;
                            kk[4 * q4 + 2] = w.z;
                            kk[4 * q4 + 3] = w.w;
                        }
#pragma unroll
                        for (int i = 0; i < 2; ++i) {
                            float p0 = fA[u], p1 = 0.f;
#pragma unroll
                            for (int l = 0; l < LP; l += 2) {
                                p0 = fmaf(kk[l], d[i][l], p0);
                                p1 = fmaf(kk[l + 1], d[i][l + 1], p1);
                            }
                            float ph = p0 + p1;
                            ph = ph - rintf(ph);
                            float sn, cs;
                            __sincosf(ph * kTwoPi, &sn, &cs);
                            packed[i][u] = pack_bf16(cs, sn);  // conj(E) = cos + i sin
                        }
                    }
                    unsigned char *atom_base = A[sa] + hh * (kRows * 128);
#pragma unroll
                    for (int i = 0; i < 2; ++i)
                        *reinterpret_cast<uint4 *>(atom_base + tc::swz128(r0 + 32 * i, jp)) =
                            make_uint4(packed[i][0], packed[i][1], packed[i][2], packed[i][3]);
                }
                tc::fence_proxy_async_smem();
                tc::mbar_arrive(&sh.afull[sa]);
            }
            // epilogue (warps 0-3, one voxel row per thread): conj(S) . u over coils
            bool ok = !sh.abort_flag;
            const int gl = gs + nst - 1;
            if (nst > 0 && ok) ok = wait_or_abort(&sh.afree[gl & 1], (gl >> 1) & 1, &sh.abort_flag, status);
            ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-collective
            tc::fence_after_sync();
            if (warp < 4) {
                const int m = 32 * warp + (tid & 31);
                const int p = vb * kRows + m;
                float u[N];
                if (nst > 0 && ok) {
                    tc::tmem_ld<N / 2>(tmem + ((uint32_t)(32 * warp) << 16), u);
                    tc::tmem_ld<N / 2>(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)(N / 2), u + N / 2);
                    tc::tmem_ld_wait();
                } else {
#pragma unroll
                    for (int c = 0; c < N; ++c) u[c] = 0.f;
                }
                if (p < ntiles * kTileVox) {
                    const float4 *s4 = reinterpret_cast<const float4 *>(P.Sp + (size_t)p * CB);
                    float xr = 0.f, xi = 0.f;
#pragma unroll
                    for (int q4 = 0; q4 < CB / 2; ++q4) {
                        float4 sv = s4[q4];
                        const float ur0 = u[2 * q4], ui0 = u[CB + 2 * q4];
                        const float ur1 = u[2 * q4 + 1], ui1 = u[CB + 2 * q4 + 1];
                        xr = fmaf(sv.x, ur0, xr);
                        xr = fmaf(sv.y, ui0, xr);
                        xi = fmaf(sv.x, ui0, xi);
                        xi = fmaf(-sv.y, ur0, xi);
                        xr = fmaf(sv.z, ur1, xr);
                        xr = fmaf(sv.w, ui1, xr);
                        xi = fmaf(sv.z, ui1, xi);
                        xi = fmaf(-sv.w, ur1, xi);
                    }
                    P.apart[(size_t)split * (size_t)(ntiles * kTileVox) + p] = make_float2(xr, xi);
                }
            }
        }
        gs += nst;
    }
    tc_teardown(sh, warp, TMEM_COLS, last_issued, &pd[0].hdr->status);
}

// ---------------------------------------------------------------------------
// Packing of the B operands into the swizzled K-major smem image, one launch for all
// problems (grid.y = problem; blocks beyond a problem's extent return at once)
// ---------------------------------------------------------------------------

// Forward: coil-weighted image b_c(v) = S_c(v) x(v) of every 8x8 tile, rows n < C carry
// (Re b, -Im b), rows C + c carry (Im b, Re b) at K positions (2v, 2v+1).  The image is
// `x` when given (single problem) or the descriptor's vec[src].
template <int CB>
__global__ void pack_b_fwd_kernel(const ProbDesc *__restrict__ pd, const float2 *__restrict__ x, int src) {
    constexpr int N = 2 * CB;
    const ProbDesc &P = pd[blockIdx.y];
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // (tile, n, chunk)
    if (i >= (size_t)P.ntiles * N * 16) return;
    const float2 *img = x ? x : P.vec[src];
    const int jj = (int)(i % 16);
    const int n = (int)((i / 16) % N);
    const int tile = (int)(i / (16 * N));
    const int c = n < CB ? n : n - CB;
    uint32_t w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const int v = 4 * jj + u;
        const int ix = (tile % P.ntx) * kTileSide + v % kTileSide, iy = (tile / P.ntx) * kTileSide + v / kTileSide;
        float br = 0.f, bi = 0.f;
        if (ix < P.nx && iy < P.ny) {
            float2 s = P.Sp[((size_t)tile * kTileVox + v) * CB + c];
            float2 xv = img[(size_t)iy * P.nx + ix];
            br = s.x * xv.x - s.y * xv.y;
            bi = s.x * xv.y + s.y * xv.x;
        }
        w[u] = n < CB ? pack_bf16(br, -bi) : pack_bf16(bi, br);
    }
    unsigned char *dst = P.bpk + (size_t)tile * (N * 256) + (jj >> 3) * (N * 128) + tc::swz128(n, jj & 7);
    *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
}

// Adjoint: k-space yt[t][c] (or the descriptor's vec[src], or rt when src < 0) per stage of
// 64 samples; rows n < C
// carry (Re y, -Im y), rows C + c carry (Im y, Re y) at K positions (2s, 2s+1).
template <int CB>
__global__ void pack_y_adj_kernel(const ProbDesc *__restrict__ pd, const float2 *__restrict__ yt, int src) {
    constexpr int N = 2 * CB;
    const ProbDesc &P = pd[blockIdx.y];
    const int nstages = P.ntp / kCols;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // (stage, n, chunk)
    if (i >= (size_t)nstages * N * 16) return;
    const float2 *y = yt ? yt : (src >= 0 ? P.vec[src] : P.rt);
    const int jj = (int)(i % 16);
    const int n = (int)((i / 16) % N);
    const int st = (int)(i / (16 * N));
    const int c = n < CB ? n : n - CB;
    uint32_t w[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const size_t t = (size_t)st * kCols + 4 * jj + u;
        float2 v = y[t * CB + c];
        w[u] = n < CB ? pack_bf16(v.x, -v.y) : pack_bf16(v.y, v.x);
    }
    unsigned char *dst = P.ypk + (size_t)st * (N * 256) + (jj >> 3) * (N * 128) + tc::swz128(n, jj & 7);
    *reinterpret_cast<uint4 *>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
}

// Reductions of the planar forward partials [split][t][re(0..C) | im(0..C)].
__global__ void fwd_reduce_planar_public_kernel(const float *part, int splits, int ntp, int CB, int nt, int nc,
                                                float2 *y) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)nt * CB) return;
    int t = (int)(i / CB), c = (int)(i % CB);
    if (c >= nc) return;
    float re = 0.f, im = 0.f;
    for (int k = 0; k < splits; ++k) {
        const float *row = part + ((size_t)k * ntp + t) * 2 * CB;
        re += row[c];
        im += row[CB + c];
    }
    y[(size_t)c * nt + t] = make_float2(re, im);
}

__global__ void fwd_reduce_planar_residual_kernel(const float *part, int splits, int ntp, int CB, int nt, int nc,
                                                  const float2 *ymeas, float2 *rt) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= (size_t)ntp * CB) return;
    int t = (int)(i / CB), c = (int)(i % CB);
    float2 s = make_float2(0.f, 0.f);
    if (t < nt && c < nc) {
        for (int k = 0; k < splits; ++k) {
            const float *row = part + ((size_t)k * ntp + t) * 2 * CB;
            s.x += row[c];
            s.y += row[CB + c];
        }
        if (ymeas) {
            s.x -= ymeas[i].x;
            s.y -= ymeas[i].y;
        }
    }
    rt[i] = s;
}

__global__ void write_desc_kernel(ProbDesc d, ProbDesc *dst) { *dst = d; }

// ---- launch helpers ----
constexpr size_t round1k(size_t v) { return (v + 1023) & ~size_t(1023); }
template <int CB, int LP>
size_t fwd_tc_smem() {
    return 1024 + 2 * kA_BYTES + kNB * round1k(2 * CB * 256 + kTileVox * LP * 4 + kRows * 4);
}
template <int CB, int LP>
size_t adj_tc_smem() {
    return 1024 + 2 * kA_BYTES + kNB * round1k(2 * CB * 256 + kCols * LP * 4 + 2 * kCols * 4);
}

template <int CB, int LP>
cudaError_t launch_fwd_tc(const ProbDesc *pd, int nprob, int max_pack_blocks, const float2 *x, int src,
                          const int *item_off, int total_items, int *counter, cudaStream_t st) {
    pack_b_fwd_kernel<CB><<<dim3(max_pack_blocks, nprob), 256, 0, st>>>(pd, x, src);
    auto kern = fwd_tc_kernel<CB, LP>;
    const size_t smem = fwd_tc_smem<CB, LP>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    kern<<<std::min(total_items, num_sms()), kTcThreads, smem, st>>>(pd, item_off, nprob, counter);
    return cudaGetLastError();
}

template <int CB, int LP>
cudaError_t launch_adj_tc(const ProbDesc *pd, int nprob, int max_pack_blocks, const float2 *yt, int src,
                          const int *item_off, int total_items, int *counter, cudaStream_t st) {
    pack_y_adj_kernel<CB><<<dim3(max_pack_blocks, nprob), 256, 0, st>>>(pd, yt, src);
    auto kern = adj_tc_kernel<CB, LP>;
    const size_t smem = adj_tc_smem<CB, LP>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    kern<<<std::min(total_items, num_sms()), kTcThreads, smem, st>>>(pd, item_off, nprob, counter);
    return cudaGetLastError();
}

#define AEXP_TC_LP(FN, CBV, ...)                         \
    switch (LPv) {                                       \
        case 4: return FN<CBV, 4>(__VA_ARGS__);          \
        case 8: return FN<CBV, 8>(__VA_ARGS__);          \
        case 12: return FN<CBV, 12>(__VA_ARGS__);        \
        default: return FN<CBV, 20>(__VA_ARGS__);        \
    }
#define AEXP_TC_DISPATCH(FN, ...)                                \
    switch (CBv) {                                               \
        case 8: AEXP_TC_LP(FN, 8, __VA_ARGS__)                   \
        case 16: AEXP_TC_LP(FN, 16, __VA_ARGS__)                 \
        default: AEXP_TC_LP(FN, 32, __VA_ARGS__)                 \
    }

}  // namespace

int fwd_pack_blocks(int ntiles, int CB) { return cdiv(ntiles * 2 * CB * 16, 256); }
int adj_pack_blocks(int ntp, int CB) { return cdiv((ntp / kCols) * 2 * CB * 16, 256); }

cudaError_t write_desc(const ProbDesc &d, ProbDesc *dst, cudaStream_t st) {
    write_desc_kernel<<<1, 1, 0, st>>>(d, dst);
    return cudaGetLastError();
}

// Single problem: the descriptor and the item offsets live in the problem's workspace
// (written by op_prepare for the tensor-core precisions).
cudaError_t op_forward_tc(const OpLayout &L, const float2 *x, char *ws, cudaStream_t st) {
    const int CBv = L.CB, LPv = L.LP;
    WsHeader *hdr = (WsHeader *)(ws + L.off_hdr);
    const ProbDesc *pd = (const ProbDesc *)(ws + L.off_desc);
    AEXP_TC_DISPATCH(launch_fwd_tc, pd, 1, fwd_pack_blocks(L.ntiles, L.CB), x, 0, &hdr->item_off[0], L.fwd_items,
                     &hdr->counter[0], st)
}

cudaError_t op_adjoint_tc(const OpLayout &L, const float2 *yt, char *ws, cudaStream_t st) {
    const int CBv = L.CB, LPv = L.LP;
    WsHeader *hdr = (WsHeader *)(ws + L.off_hdr);
    const ProbDesc *pd = (const ProbDesc *)(ws + L.off_desc);
    AEXP_TC_DISPATCH(launch_adj_tc, pd, 1, adj_pack_blocks(L.ntp, L.CB), yt, -1, &hdr->item_off[2], L.adj_items,
                     &hdr->counter[1], st)
}

cudaError_t batch_forward_tc(int CB, int LP, const ProbDesc *pd, int nprob, int max_pack_blocks, int src,
                             const int *item_off, int total_items, int *counter, cudaStream_t st) {
    const int CBv = CB, LPv = LP;
    AEXP_TC_DISPATCH(launch_fwd_tc, pd, nprob, max_pack_blocks, nullptr, src, item_off, total_items, counter, st)
}

cudaError_t batch_adjoint_tc(int CB, int LP, const ProbDesc *pd, int nprob, int max_pack_blocks, int src,
                             const int *item_off, int total_items, int *counter, cudaStream_t st) {
    const int CBv = CB, LPv = LP;
    AEXP_TC_DISPATCH(launch_adj_tc, pd, nprob, max_pack_blocks, nullptr, src, item_off, total_items, counter, st)
}

cudaError_t op_forward_reduce_planar_public(const OpLayout &L, char *ws, float2 *y, cudaStream_t st) {
    size_t n = (size_t)L.nt * L.CB;
    fwd_reduce_planar_public_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        (const float *)(ws + L.off_fpart), L.fwd_splits, L.ntp, L.CB, L.nt, L.nc, y);
    return cudaGetLastError();
}

cudaError_t op_forward_reduce_planar_residual(const OpLayout &L, char *ws, const float2 *ymeas_t, float2 *rt,
                                              cudaStream_t st) {
    size_t n = (size_t)L.ntp * L.CB;
    fwd_reduce_planar_residual_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        (const float *)(ws + L.off_fpart), L.fwd_splits, L.ntp, L.CB, L.nt, L.nc, ymeas_t, rt);
    return cudaGetLastError();
}

}  // namespace aexp
