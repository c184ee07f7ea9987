// A_exp and A_exp^H in the BF16 form with the phase computed on the tensor cores as well.
//
// Inside a work item the phase offsets of a stage are a small matrix product,
//   off(t, v) = sum_l khi(t, l) dh(v, l)        (t: 128 samples or 64 per stage, v: voxels,
//                                                l: field terms incl. B0, padded to 16 or 32)
// with khi = k / 2pi in turns and dh the basis offsets from the tile's reference voxel
// (the same quantities the CUDA-core generators sum with FMAs).  It runs as tcgen05.mma
// kind::f16 with BF16 operands into a TMEM tile, each factor split x = x_hi + x_lo in BF16
// (x_hi rounded to 8 significant bits, x_lo = x - x_hi rounded again) and the products
// hi*hi + hi*lo + lo*hi accumulated in FP32: relative error ~2^-17 of sum_l |khi dh|, about
// 1e-4 rad for the ~12 rad an 8x8 tile spans at the Nyquist edge of k-space, twenty times
// below the BF16 rounding of E (2^-9).  Each K step takes 16 terms, so up to 16 terms cost
// 3 MMAs per stage and up to 32 terms 6 (TF32 operands, 8 terms per step, took 9).
//
// Generators then read their row's phase offsets of the stage with one tcgen05.ld (in
// radians: the k operand carries the factor 2 pi), add 2 pi f0(tile, t) with the tile's
// tabulated reference phase f0 in [-1/2, 1/2) turn, take one MUFU sincos and write their row
// of the BF16 encoding tile into TMEM with one tcgen05.st (no shared-memory stores, no proxy
// fence); the contraction with the coil-weighted image (or the k-space data) is a tcgen05
// kind::f16 GEMM with A read from TMEM and B, the packed BF16 operand, from shared memory.
// The two GEMMs are issued by two threads of their own: the
// contraction thread issues 8 MMAs per stage once the generators have stored A(g); the
// phase thread fills four TMEM phase tiles, each as soon as the generators have read it.
// The generators form two groups of 8 warps that take alternate stages, so that one group
// computes while the other waits for its next stage.
// (A 128-row MMA with N <= 64 occupies the tensor pipe for ~50 cycles, so one thread
// issuing both GEMMs in turn would bound the stage rate.)
// The epilogue waits for the item's last contraction on a barrier of its own (accdone, one
// completion per item with stages, waited for by the same warps every item).  Waiting on the
// A-release barrier of the last stage instead was wrong for the generator group that did not
// produce that stage: it had not followed that barrier's phases, and when the contraction two
// stages back was still running the parity test passed one phase early, so that warp read
// partial accumulators (seen as run-to-run differences in one lane quadrant of one item).
//
// Phase operands, prepared once per problem (BF16 images in the 128B-swizzled K-major
// layout, 64 K slots = 128 bytes per row: slots 0-31 hold the hi parts, 32-63 the lo parts):
//   kph   per block of 128 samples, rows = samples:  forward A_phase; adjoint B_phase
//         (the 64 rows of one stage are one half of a block)
//   dhph  per pair of tiles, rows = 128 voxels:      adjoint A_phase; forward B_phase
//         (the 64 rows of one tile are one half of a pair)
#include <algorithm>

#include "tc_common.cuh"

namespace aexp {
namespace {

constexpr unsigned kHalfImg = 64 * 128;         // the hi | lo image of 64 rows, 8 KB
constexpr unsigned kApBytes = kRows * 128;      // item operand: hi | lo image of 128 rows, 16 KB
constexpr uint32_t kLoBytes = 64;               // the lo parts start 32 slots (64 B) into a row
// TMEM: the contraction accumulates in columns 0..N-1, phase tile b (of 4) sits at 64 + 64 b,
// the generated encoding tile of A buffer a (of 2: 128 rows x 128 BF16, two per column) at
// 320 + 64 a
constexpr uint32_t kPhBase = 64;
constexpr int kPhBufs = 4;
constexpr uint32_t kABase = kPhBase + 64 * kPhBufs;
constexpr uint32_t kTmemCols = 512;
static_assert(kABase + 2 * 64 <= kTmemCols, "TMEM plan");

__device__ __forceinline__ uint32_t phase_col(int g) { return kPhBase + 64u * (uint32_t)(g % kPhBufs); }
__device__ __forceinline__ uint32_t a_col(int sa) { return kABase + 64u * (uint32_t)sa; }

// ---- operand preparation ----

// Eight values -> 16-byte chunks of BF16 hi parts and of BF16 lo parts (lo = x - hi, rounded).
__device__ __forceinline__ void split_bf16_8(const float (&v)[8], uint4 &hi, uint4 &lo) {
    uint32_t h[4], l[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
        const __nv_bfloat162 hb = __floats2bfloat162_rn(v[2 * u], v[2 * u + 1]);
        const float2 hf = __bfloat1622float2(hb);
        const __nv_bfloat162 lb = __floats2bfloat162_rn(v[2 * u] - hf.x, v[2 * u + 1] - hf.y);
        h[u] = *reinterpret_cast<const uint32_t *>(&hb);
        l[u] = *reinterpret_cast<const uint32_t *>(&lb);
    }
    hi = make_uint4(h[0], h[1], h[2], h[3]);
    lo = make_uint4(l[0], l[1], l[2], l[3]);
}

// kph[block][row = sample % 128][hi slots 0-31 | lo slots 0-31] = 2 pi khi_t[sample][slot]
// (0 beyond LP): the phase GEMM yields radians
__global__ void prep_kph_kernel(const float *__restrict__ khi_t, int ntp, int LP, unsigned char *__restrict__ kph) {
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // (sample, chunk of 8 slots)
    if (i >= (size_t)ntp * 4) return;
    const int t = (int)(i / 4), c = (int)(i % 4);
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int l = 8 * c + u;
        v[u] = l < LP ? kTwoPi * khi_t[(size_t)t * LP + l] : 0.f;
    }
    uint4 hi, lo;
    split_bf16_8(v, hi, lo);
    unsigned char *blk = kph + (size_t)(t / kRows) * kPhaseBlockBytes;
    *reinterpret_cast<uint4 *>(blk + tc::swz128(t % kRows, c)) = hi;
    *reinterpret_cast<uint4 *>(blk + tc::swz128(t % kRows, c + 4)) = lo;
}

// dhph[pair][row = 64 (tile & 1) + voxel][hi slots | lo slots] = dh[tile][voxel][slot] (0 beyond
// LP and for the missing second tile of an odd count)
__global__ void prep_dhph_kernel(const float *__restrict__ dh, int ntiles, int LP, unsigned char *__restrict__ dhph) {
    const int npairs = (ntiles + 1) / 2;
    const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;  // (pair, row, chunk)
    if (i >= (size_t)npairs * kRows * 4) return;
    const int c = (int)(i % 4);
    const int r = (int)((i / 4) % kRows);
    const int pair = (int)(i / (4 * kRows));
    const int tile = 2 * pair + r / kTileVox, v = r % kTileVox;
    float x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        const int l = 8 * c + u;
        x[u] = (tile < ntiles && l < LP) ? dh[((size_t)tile * kTileVox + v) * LP + l] : 0.f;
    }
    uint4 hi, lo;
    split_bf16_8(x, hi, lo);
    unsigned char *blk = dhph + (size_t)pair * kPhaseBlockBytes;
    *reinterpret_cast<uint4 *>(blk + tc::swz128(r, c)) = hi;
    *reinterpret_cast<uint4 *>(blk + tc::swz128(r, c + 4)) = lo;
}

// ---- kernels ----

// Warp roles: 16 generator warps; warp 16 issues the contraction MMAs and owns TMEM; warp 17
// loads the contraction operands (+ reference phases); warp 18 issues the phase MMAs; warp 19
// loads the phase operands.  One lane of each non-generator warp works.
constexpr int kMmaWarp = kTcGen / 32;
constexpr int kLoadBWarp = kMmaWarp + 1;
constexpr int kPhaseWarp = kMmaWarp + 2;
constexpr int kLoadPWarp = kMmaWarp + 3;
constexpr int kTcpThreads = kTcGen + 128;
// Ring depths (template parameters NBB, NP of the kernels): per-stage contraction operands +
// reference phases (NBB) and per-stage phase operands (NP, hi | lo image of 8 KB).  Tiling 0:
// 4 and 3; tiling 1 (aexp_recon_opts::tile_variant): 6 and 4.
// A generator group waits only on the stages of its parity, so each B slot and each phase tile
// must belong to one group: with an odd count a slot would alternate between the groups, a
// group would skip every other phase of that slot's barrier and its parity test could pass a
// phase early.  (The MMA thread and the loaders wait on every stage; NP may be anything.)
static_assert(kPhBufs % 2 == 0, "each generator group must own its phase tiles");

// Shared-memory plan of both kernels (byte offsets from the 1024-aligned base; the generated
// encoding tiles live in TMEM):
//   AP item phase operand (hi | lo) | PH ring | B ring
template <int N, int NBB, int NP>
struct TcpPlan {
    static_assert(NBB % 2 == 0, "each generator group must own its B slots");
    static_assert(NBB <= kNBMax && NP <= kNBMax, "ring deeper than the CTA's barriers");
    static constexpr unsigned B_BYTES = N * 256;
    static constexpr unsigned F_BYTES = kRows * 4;  // forward: 128 f0; adjoint: 2 x 64 f0
    static constexpr unsigned BS = (B_BYTES + F_BYTES + 1023u) & ~1023u;  // B ring stride
    static constexpr unsigned PS = kHalfImg;                              // PH ring stride
    static constexpr unsigned OFF_AP = 0;
    static constexpr unsigned OFF_PH = OFF_AP + kApBytes;
    static constexpr unsigned OFF_B = OFF_PH + NP * PS;
    static constexpr unsigned BYTES = OFF_B + NBB * BS;
};

// Contraction of one stage: 8 MMAs of K = 16 (BF16) into columns 0..N-1, A (the encoding
// tile) read from TMEM at `ta` (8 columns per K step), B from shared memory.
template <int N>
__device__ __forceinline__ void contraction_mma(uint32_t tmem, uint32_t ta, uint64_t db, bool first) {
    constexpr uint32_t ID = tc::idesc_f16(kRows, N, 1);
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
        const uint32_t kofb = (uint32_t)((kk >> 2) * (N * 128) + (kk & 3) * 32);
        tc::mma_f16_ts(tmem, ta + 8u * (uint32_t)kk, tc::sdesc_advance(db, kofb), ID, !(first && kk == 0));
    }
}

// Phase GEMM of one stage into the tile at `d`: KS steps of 16 BF16 values, products
// hi*hi + hi*lo + lo*hi (the lo parts sit kLoBytes further along each row).
template <int KS>
__device__ __forceinline__ void phase_mma_ks(uint32_t d, uint64_t a, uint64_t b) {
    constexpr uint32_t ID = tc::idesc_f16(kRows, 64, 1);
#pragma unroll
    for (int k = 0; k < KS; ++k) tc::mma_f16(d, tc::sdesc_advance(a, 32 * k), tc::sdesc_advance(b, 32 * k), ID, k > 0);
#pragma unroll
    for (int k = 0; k < KS; ++k)
        tc::mma_f16(d, tc::sdesc_advance(a, 32 * k), tc::sdesc_advance(b, kLoBytes + 32 * k), ID, 1u);
#pragma unroll
    for (int k = 0; k < KS; ++k)
        tc::mma_f16(d, tc::sdesc_advance(a, kLoBytes + 32 * k), tc::sdesc_advance(b, 32 * k), ID, 1u);
}

__device__ __forceinline__ void phase_mma(int ks, uint32_t d, uint64_t a, uint64_t b) {
    if (ks <= 1) phase_mma_ks<1>(d, a, b);
    else phase_mma_ks<2>(d, a, b);
}

// Contraction thread, one item.
template <int N, int NBB, int NP>
__device__ __forceinline__ void tcp_contraction_item(TcShared &sh, uint32_t tmem, unsigned char *base, int gs, int n,
                                                     int *status) {
    using PL = TcpPlan<N, NBB, NP>;
    for (int it = 0; it < n; ++it) {
        const int g = gs + it, sa = g & 1, sb = g % NBB;
        if (!wait_or_abort(&sh.afull[sa], (g >> 1) & 1, &sh.abort_flag, status)) return;
        if (!wait_or_abort(&sh.bfull[sb], (g / NBB) & 1, &sh.abort_flag, status)) return;
        tc::fence_after_sync();
        contraction_mma<N>(tmem, tmem + a_col(sa), tc::sdesc_k128(smem_u32(base + PL::OFF_B + sb * PL::BS)),
                           it == 0);
        tc::mma_commit(&sh.afree[sa]);
        tc::mma_commit(&sh.bfree[sb]);
    }
    if (n > 0) tc::mma_commit(&sh.accdone);  // the item's accumulators are final
}

// Phase thread, one item: the phases of stage g go into tile g % 4 once the generators have
// read that tile for stage g - 4 and the stage's operand has landed.
template <int N, int NBB, int NP>
__device__ __forceinline__ void tcp_phase_item(TcShared &sh, uint32_t tmem, unsigned char *base, int gs, int n,
                                               int iter, int ks, int *status) {
    using PL = TcpPlan<N, NBB, NP>;
    const uint64_t ad = tc::sdesc_k128(smem_u32(base + PL::OFF_AP));
    if (!wait_or_abort(&sh.apfull, iter & 1, &sh.abort_flag, status)) return;
    for (int it = 0; it < n; ++it) {
        const int g = gs + it, b = g % kPhBufs, sp = g % NP;
        if (g >= kPhBufs && !wait_or_abort(&sh.phfree[b], ((g - kPhBufs) / kPhBufs) & 1, &sh.abort_flag, status))
            return;
        if (!wait_or_abort(&sh.pfull[sp], (g / NP) & 1, &sh.abort_flag, status)) return;
        tc::fence_after_sync();
        phase_mma(ks, tmem + phase_col(g), ad, tc::sdesc_k128(smem_u32(base + PL::OFF_PH + sp * PL::PS)));
        tc::mma_commit(&sh.phfull[b]);
        tc::mma_commit(&sh.pfree[sp]);
    }
}

// Teardown: both MMA threads commit to the drain barrier (count 2); the contraction thread
// waits (bounded) until every MMA has completed; then TMEM is released.
__device__ __forceinline__ void tcp_teardown(TcShared &sh, int tid, int warp, int *status) {
    if (tid == kPhaseWarp * 32) tc::mma_commit(&sh.drain);
    if (tid == kMmaWarp * 32) {
        tc::mma_commit(&sh.drain);
        mbar_wait_bounded(&sh.drain, 0, status);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == kMmaWarp) {
        tc::fence_after_sync();
        tc::tmem_dealloc(sh.tmem_base, kTmemCols);
    }
}

// One generator thread's part of a stage (generators work in two groups of 8 warps that take
// alternate stages; warp w of a group reads TMEM lanes 32 (w & 3) .. + 31 and owns the 32
// columns 32 (w >> 2) .. + 31): its row's 32 phase offsets (TMEM; the tile is released to the
// phase thread right after the read) plus the reference phases -> E (or conj E) as BF16, one
// (re, im) pair per TMEM column of its row of the A tile at `ta`.  Forward: one reference phase
// per row (fsrc[0]); adjoint: one per column (fsrc[0..31]).
template <bool CONJ>
__device__ __forceinline__ bool generate_row(TcShared &sh, int g, uint32_t taddr, const float *fsrc, uint32_t ta,
                                             int *status) {
    float ph[32];
    tc::tmem_ld<32>(taddr, ph);
    tc::tmem_ld_wait();
    tc::tmem_regs_ready<32>(ph);
    tc::fence_before_sync();
    __syncwarp();
    if ((threadIdx.x & 31) == 0) tc::mbar_arrive(&sh.phfree[g % kPhBufs]);
    uint32_t w[32];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
        float f[4];
        if constexpr (CONJ) {
            const float4 fw = reinterpret_cast<const float4 *>(fsrc)[c];
            f[0] = fw.x;
            f[1] = fw.y;
            f[2] = fw.z;
            f[3] = fw.w;
        } else {
            f[0] = f[1] = f[2] = f[3] = fsrc[0];
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            // angle = 2 pi f0 + offset (radians); f0 lies in [-1/2, 1/2) turn and the offset spans
            // a few turns inside a tile, so the hardware sincos needs no further reduction (its
            // error grows like |angle| x 2^-24, ~1e-6 here against 2^-9 for the BF16 rounding)
            const float x = fmaf(f[u], kTwoPi, ph[4 * c + u]);
            float sn, cs;
            __sincosf(x, &sn, &cs);
            w[4 * c + u] = pack_bf16(cs, CONJ ? sn : -sn);  // E = cos - i sin, conj(E) = cos + i sin
        }
    }
    // The A buffer is claimed only now: the contraction of stage g - 2, which frees it,
    // overlaps the sincos work above.  This group waited on the barrier for stage g - 2's
    // previous use (stage g - 4), so the parity is unambiguous.
    bool ok = g < 2 || wait_or_abort(&sh.afree[g & 1], ((g - 2) >> 1) & 1, &sh.abort_flag, status);
    if (!__all_sync(0xffffffffu, ok)) return false;
    tc::fence_after_sync();
    tc::tmem_st32(ta, w);
    tc::tmem_st_wait();
    return true;
}

// Generator waits of stage g before its TMEM read (warp-uniform result): reference phases
// landed, phase tile ready.  The A buffer is waited for inside generate_row.
template <int NBB>
__device__ __forceinline__ bool gen_waits(TcShared &sh, int g, int *status) {
    bool ok = wait_or_abort(&sh.bfull[g % NBB], (g / NBB) & 1, &sh.abort_flag, status);
    if (ok) ok = wait_or_abort(&sh.phfull[g % kPhBufs], (g / kPhBufs) & 1, &sh.abort_flag, status);
    return __all_sync(0xffffffffu, ok);
}

// Forward: item = (problem, block of 128 samples, run of voxel tiles).
template <int CB, int NBB, int NP>
__global__ void __launch_bounds__(kTcpThreads, 1)
    fwd_tcp_kernel(const ProbDesc *__restrict__ pd, const int *__restrict__ item_off, int nprob, int *counter) {
    constexpr int N = 2 * CB;
    using PL = TcpPlan<N, NBB, NP>;

    extern __shared__ unsigned char smem_raw[];
    __shared__ TcShared sh;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const uint32_t sbase = align1024(smem_u32(smem_raw));
    unsigned char *gbase = smem_raw + (sbase - smem_u32(smem_raw));
    const int total = item_off[nprob];

    tc_setup(sh, tid, warp, kTmemCols, 1, kTcGen / 2, kTcGen / 64);  // two generator groups
    const uint32_t tmem = sh.tmem_base;
    int gs = 0;
    int nacc = 0;  // items with stages so far: the accdone phase this CTA waits for next

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

        if (warp >= kMmaWarp) {
            const bool lead = (tid & 31) == 0;
            if (warp == kMmaWarp && lead) {
                tcp_contraction_item<N, NBB, NP>(sh, tmem, gbase, gs, ntl, status);
            } else if (warp == kPhaseWarp && lead) {
                tcp_phase_item<N, NBB, NP>(sh, tmem, gbase, gs, ntl, iter, (P.LP + 15) >> 4, status);
            } else if (warp == kLoadBWarp && lead) {
                ring_load_item(sh.bfree, NBB, gs, ntl, &sh.abort_flag, status, [&](int it, int sb) {
                    const int tile = tile0 + it;  // packed S x of the tile and its reference phases
                    unsigned char *dst = gbase + PL::OFF_B + sb * PL::BS;
                    mbar_arrive_expect_tx(&sh.bfull[sb], PL::B_BYTES + PL::F_BYTES);
                    bulk_g2s(dst, P.bpk + (size_t)tile * PL::B_BYTES, PL::B_BYTES, &sh.bfull[sb]);
                    bulk_g2s(dst + PL::B_BYTES, P.f0 + (size_t)tile * ntp + tbase, PL::F_BYTES, &sh.bfull[sb]);
                });
            } else if (warp == kLoadPWarp && lead) {
                mbar_arrive_expect_tx(&sh.apfull, kApBytes);
                bulk_g2s(gbase + PL::OFF_AP, P.kph + (size_t)(tbase / kRows) * kPhaseBlockBytes, kApBytes, &sh.apfull);
                ring_load_item(sh.pfree, NP, gs, ntl, &sh.abort_flag, status, [&](int it, int sp) {
                    const int tile = tile0 + it;  // the tile's basis offsets, hi | lo
                    const unsigned char *dp =
                        P.dhph + (size_t)(tile >> 1) * kPhaseBlockBytes + (size_t)(tile & 1) * kHalfImg;
                    mbar_arrive_expect_tx(&sh.pfull[sp], kHalfImg);
                    bulk_g2s(gbase + PL::OFF_PH + sp * PL::PS, dp, kHalfImg, &sh.pfull[sp]);
                });
            }
        } else {
            // generator group warp >> 3 takes the stages of its parity; warp w reads TMEM lanes
            // 32 (w & 3) .. + 31 (its rows) and owns voxel columns 32 ((w >> 2) & 1) .. + 31
            const int row = 32 * (warp & 3) + (tid & 31);
            const int ch = (warp >> 2) & 1;
            const int grp = warp >> 3;
            for (int it = 0; it < ntl; ++it) {
                const int g = gs + it, sa = g & 1, sb = g % NBB;
                if ((g & 1) != grp) continue;
                if (!gen_waits<NBB>(sh, g, status)) break;  // warp-uniform exit
                tc::fence_after_sync();
                const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
                if (!generate_row<false>(sh, g, tmem + lanes + phase_col(g) + (uint32_t)(32 * ch),
                                    reinterpret_cast<const float *>(gbase + PL::OFF_B + sb * PL::BS + PL::B_BYTES) + row,
                                    tmem + lanes + a_col(sa) + (uint32_t)(32 * ch), status))
                    break;  // warp-uniform exit
                tc::fence_before_sync();
                tc::mbar_arrive(&sh.afull[sa]);
            }
            // epilogue (warps 0-7): last stage's MMAs done -> TMEM -> partials (planar re | im)
            bool ok = !sh.abort_flag;
            if (ntl > 0 && ok) ok = wait_or_abort(&sh.accdone, nacc & 1, &sh.abort_flag, status);
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
                    tc::tmem_regs_ready<N / 2>(v);
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
        nacc += ntl > 0;
    }
    tcp_teardown(sh, tid, warp, &pd[0].hdr->status);
}

// Adjoint: item = (problem, pair of voxel tiles, run of 64-sample stages).
template <int CB, int NBB, int NP>
__global__ void __launch_bounds__(kTcpThreads, 1)
    adj_tcp_kernel(const ProbDesc *__restrict__ pd, const int *__restrict__ item_off, int nprob, int *counter) {
    constexpr int N = 2 * CB;
    constexpr int TS = kCols;  // samples per stage
    using PL = TcpPlan<N, NBB, NP>;
    constexpr unsigned FT = TS * 4;  // reference phases of one tile for one stage

    extern __shared__ unsigned char smem_raw[];
    __shared__ TcShared sh;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const uint32_t sbase = align1024(smem_u32(smem_raw));
    unsigned char *gbase = smem_raw + (sbase - smem_u32(smem_raw));
    const int total = item_off[nprob];

    tc_setup(sh, tid, warp, kTmemCols, 1, kTcGen / 2, kTcGen / 64);  // two generator groups
    const uint32_t tmem = sh.tmem_base;
    int gs = 0;
    int nacc = 0;  // items with stages so far: the accdone phase this CTA waits for next

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

        if (warp >= kMmaWarp) {
            const bool lead = (tid & 31) == 0;
            if (warp == kMmaWarp && lead) {
                tcp_contraction_item<N, NBB, NP>(sh, tmem, gbase, gs, nst, status);
            } else if (warp == kPhaseWarp && lead) {
                tcp_phase_item<N, NBB, NP>(sh, tmem, gbase, gs, nst, iter, (P.LP + 15) >> 4, status);
            } else if (warp == kLoadBWarp && lead) {
                ring_load_item(sh.bfree, NBB, gs, nst, &sh.abort_flag, status, [&](int it, int sb) {
                    const size_t ts = (size_t)t0 + (size_t)it * TS;  // packed y and both tiles' f0
                    unsigned char *dst = gbase + PL::OFF_B + sb * PL::BS;
                    mbar_arrive_expect_tx(&sh.bfull[sb], PL::B_BYTES + 2 * FT);
                    bulk_g2s(dst, P.ypk + (ts / TS) * PL::B_BYTES, PL::B_BYTES, &sh.bfull[sb]);
                    bulk_g2s(dst + PL::B_BYTES, P.f0 + (size_t)tileA * ntp + ts, FT, &sh.bfull[sb]);
                    bulk_g2s(dst + PL::B_BYTES + FT, P.f0 + (size_t)tileB * ntp + ts, FT, &sh.bfull[sb]);
                });
            } else if (warp == kLoadPWarp && lead) {
                mbar_arrive_expect_tx(&sh.apfull, kApBytes);
                bulk_g2s(gbase + PL::OFF_AP, P.dhph + (size_t)vb * kPhaseBlockBytes, kApBytes, &sh.apfull);
                ring_load_item(sh.pfree, NP, gs, nst, &sh.abort_flag, status, [&](int it, int sp) {
                    const size_t ts = (size_t)t0 + (size_t)it * TS;  // the stage's k rows, hi | lo
                    const unsigned char *kp =
                        P.kph + (ts / kRows) * kPhaseBlockBytes + ((ts / TS) & 1) * (size_t)kHalfImg;
                    mbar_arrive_expect_tx(&sh.pfull[sp], kHalfImg);
                    bulk_g2s(gbase + PL::OFF_PH + sp * PL::PS, kp, kHalfImg, &sh.pfull[sp]);
                });
            }
        } else {
            // generator group warp >> 3 takes the stages of its parity; warp w reads TMEM lanes
            // 32 (w & 3) .. + 31 (voxel rows; rows 0-63 in tile A, 64-127 in tile B) and owns sample
            // columns 32 ((w >> 2) & 1) .. + 31
            const int row = 32 * (warp & 3) + (tid & 31);
            const int th = (warp & 3) >> 1;
            const int ch = (warp >> 2) & 1;
            const int grp = warp >> 3;
            for (int it = 0; it < nst; ++it) {
                const int g = gs + it, sa = g & 1, sb = g % NBB;
                if ((g & 1) != grp) continue;
                if (!gen_waits<NBB>(sh, g, status)) break;  // warp-uniform exit
                tc::fence_after_sync();
                const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
                if (!generate_row<true>(sh, g, tmem + lanes + phase_col(g) + (uint32_t)(32 * ch),
                                   reinterpret_cast<const float *>(gbase + PL::OFF_B + sb * PL::BS + PL::B_BYTES + th * FT) +
                                       32 * ch,
                                   tmem + lanes + a_col(sa) + (uint32_t)(32 * ch), status))
                    break;  // warp-uniform exit
                tc::fence_before_sync();
                tc::mbar_arrive(&sh.afull[sa]);
            }
            // epilogue (warps 0-3, one voxel row per thread): conj(S) . u over coils
            bool ok = !sh.abort_flag;
            if (nst > 0 && ok) ok = wait_or_abort(&sh.accdone, nacc & 1, &sh.abort_flag, status);
            ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-collective
            tc::fence_after_sync();
            if (warp < 4) {
                const int p = vb * kRows + row;
                const bool inside = p < ntiles * kTileVox;
                const bool have = nst > 0 && ok;
                const uint32_t ta0 = tmem + ((uint32_t)(32 * warp) << 16);
                const float4 *s4 = reinterpret_cast<const float4 *>(P.Sp + (size_t)(inside ? p : 0) * CB);
                float xr = 0.f, xi = 0.f;
#pragma unroll 1
                for (int c0 = 0; c0 < CB; c0 += 8) {
                    float ur[8], ui[8];
                    if (have) {
                        tc::tmem_ld<8>(ta0 + (uint32_t)c0, ur);
                        tc::tmem_ld<8>(ta0 + (uint32_t)(CB + c0), ui);
                        tc::tmem_ld_wait();
                        tc::tmem_regs_ready<8>(ur);
                        tc::tmem_regs_ready<8>(ui);
                    } else {
#pragma unroll
                        for (int c = 0; c < 8; ++c) ur[c] = ui[c] = 0.f;
                    }
#pragma unroll
                    for (int q4 = 0; q4 < 4; ++q4) {
                        const float4 sv = s4[c0 / 2 + q4];
                        xr = fmaf(sv.x, ur[2 * q4], xr);
                        xr = fmaf(sv.y, ui[2 * q4], xr);
                        xi = fmaf(sv.x, ui[2 * q4], xi);
                        xi = fmaf(-sv.y, ur[2 * q4], xi);
                        xr = fmaf(sv.z, ur[2 * q4 + 1], xr);
                        xr = fmaf(sv.w, ui[2 * q4 + 1], xr);
                        xi = fmaf(sv.z, ui[2 * q4 + 1], xi);
                        xi = fmaf(-sv.w, ur[2 * q4 + 1], xi);
                    }
                }
                if (inside) P.apart[(size_t)split * (size_t)(ntiles * kTileVox) + p] = make_float2(xr, xi);
            }
        }
        gs += nst;
        nacc += nst > 0;
    }
    tcp_teardown(sh, tid, warp, &pd[0].hdr->status);
}

// ---- launches ----
template <int CB, int NBB, int NP>
size_t tcp_smem() {
    return 1024 + TcpPlan<2 * CB, NBB, NP>::BYTES;
}

template <int CB, int NBB, int NP>
cudaError_t launch_fwd_tcp(const ProbDesc *pd, int nprob, int max_pack_blocks, const float2 *x, int src,
                           const int *item_off, int total_items, int *counter, cudaStream_t st) {
    pack_b_fwd_kernel<CB, false><<<dim3(pack_grid(max_pack_blocks, CB), nprob), 256, 0, st>>>(pd, x, src);
    auto kern = fwd_tcp_kernel<CB, NBB, NP>;
    const size_t smem = tcp_smem<CB, NBB, NP>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    kern<<<std::min(total_items, num_sms()), kTcpThreads, smem, st>>>(pd, item_off, nprob, counter);
    return cudaGetLastError();
}

template <int CB, int NBB, int NP>
cudaError_t launch_adj_tcp(const ProbDesc *pd, int nprob, int max_pack_blocks, const float2 *yt, int src,
                           const int *item_off, int total_items, int *counter, cudaStream_t st) {
    pack_y_adj_kernel<CB, false><<<dim3(pack_grid(max_pack_blocks, CB), nprob), 256, 0, st>>>(pd, yt, src);
    auto kern = adj_tcp_kernel<CB, NBB, NP>;
    const size_t smem = tcp_smem<CB, NBB, NP>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    kern<<<std::min(total_items, num_sms()), kTcpThreads, smem, st>>>(pd, item_off, nprob, counter);
    return cudaGetLastError();
}

template <int CB>
cudaError_t launch_fwd_tcp_variant(int variant, const ProbDesc *pd, int nprob, int max_pack_blocks, const float2 *x,
                                   int src, const int *item_off, int total_items, int *counter, cudaStream_t st) {
    return variant == 1 ? launch_fwd_tcp<CB, 6, 4>(pd, nprob, max_pack_blocks, x, src, item_off, total_items, counter, st)
                        : launch_fwd_tcp<CB, 4, 3>(pd, nprob, max_pack_blocks, x, src, item_off, total_items, counter, st);
}

template <int CB>
cudaError_t launch_adj_tcp_variant(int variant, const ProbDesc *pd, int nprob, int max_pack_blocks, const float2 *yt,
                                   int src, const int *item_off, int total_items, int *counter, cudaStream_t st) {
    return variant == 1 ? launch_adj_tcp<CB, 6, 4>(pd, nprob, max_pack_blocks, yt, src, item_off, total_items, counter, st)
                        : launch_adj_tcp<CB, 4, 3>(pd, nprob, max_pack_blocks, yt, src, item_off, total_items, counter, st);
}

}  // namespace

cudaError_t op_prepare_phase_operands(const OpLayout &L, char *ws, cudaStream_t st) {
    const int T = 256;
    const size_t nk = (size_t)L.ntp * 4;
    prep_kph_kernel<<<(unsigned)((nk + T - 1) / T), T, 0, st>>>((const float *)(ws + L.off_khi_t), L.ntp, L.LP,
                                                               (unsigned char *)(ws + L.off_kph));
    const size_t nd = (size_t)cdiv(L.ntiles, 2) * kRows * 4;
    prep_dhph_kernel<<<(unsigned)((nd + T - 1) / T), T, 0, st>>>((const float *)(ws + L.off_dh), L.ntiles, L.LP,
                                                                (unsigned char *)(ws + L.off_dhph));
    return cudaGetLastError();
}

cudaError_t tcp_forward(int CB, int variant, const ProbDesc *pd, int nprob, int max_pack_blocks, const float2 *x,
                        int src, const int *item_off, int total_items, int *counter, cudaStream_t st) {
    switch (CB) {
        case 8: return launch_fwd_tcp_variant<8>(variant, pd, nprob, max_pack_blocks, x, src, item_off, total_items, counter, st);
        case 16: return launch_fwd_tcp_variant<16>(variant, pd, nprob, max_pack_blocks, x, src, item_off, total_items, counter, st);
        default: return launch_fwd_tcp_variant<32>(variant, pd, nprob, max_pack_blocks, x, src, item_off, total_items, counter, st);
    }
}

cudaError_t tcp_adjoint(int CB, int variant, const ProbDesc *pd, int nprob, int max_pack_blocks, const float2 *yt,
                        int src, const int *item_off, int total_items, int *counter, cudaStream_t st) {
    switch (CB) {
        case 8: return launch_adj_tcp_variant<8>(variant, pd, nprob, max_pack_blocks, yt, src, item_off, total_items, counter, st);
        case 16: return launch_adj_tcp_variant<16>(variant, pd, nprob, max_pack_blocks, yt, src, item_off, total_items, counter, st);
        default: return launch_adj_tcp_variant<32>(variant, pd, nprob, max_pack_blocks, yt, src, item_off, total_items, counter, st);
    }
}

}  // namespace aexp
