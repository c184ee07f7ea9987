// A_exp and A_exp^H on the tcgen05 tensor cores in the FP16 hi+lo form (both operands split
// into FP16 hi and lo parts; FP32 accumulation in TMEM), plus the launches that the BF16 form
// (op_tc_phase.cu) shares: descriptors, dispatch and the planar partial-sum reductions.
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
// CTA = 16 generator warps + an MMA warp + two loader warps (see the warp-role note below).
// Generators compute the FP32 phase in radians (tabulated reference phase + local offset, the
// coefficient or basis operand held in registers pre-multiplied by 2 pi), take one MUFU sincos
// of it (the angle spans a few turns, within the hardware's unreduced range), split E into
// FP16 hi + lo' and store 16-byte chunks straight into the 128B-swizzled K-major layout; each
// thread owns 2 rows x 8 columns.  The A tile is double buffered: the MMAs of stage g - 1 run
// while stage g is generated.  Every wait is bounded; on a timeout the CTA records
// AEXP_ERR_DEVICE_TIMEOUT, drains its MMAs, frees TMEM and exits.
//
// FP16 hi+lo form (HL): every operand value v is split into v_hi = fp16(v) and
// v_lo' = fp16(2^11 (v - v_hi)), so v = v_hi + 2^-11 v_lo' to about 2^-22 relative.  Per
// stage three MMA passes run: A_hi B_hi into accumulator D1 and A_hi B_lo' + A_lo' B_hi into
// D2 (the lo x lo product, ~2^-22, is dropped); the epilogue forms D1 + 2^-11 D2.  |E| <= 1
// needs no scaling; the B operand (S x, or y) is scaled by a power of two 2^e chosen from
// its largest component so that it lies below 2^14 (FP16 tops out at 65504), and the
// epilogue multiplies by 2^-e.  The largest component is found by a reduction kernel before
// the packing (an atomic max on the float bit pattern in the problem's header).  Stages
// carry twice the operand bytes, so two B stages are kept.
// The tensor core's FP32 accumulation loses about 2^-24 of the running sum per MMA, which
// over a long item (hundreds of MMAs) would dominate the hi+lo error; so the accumulator is
// promoted every kPromote stages: two accumulator sets alternate by chunk of stages, the
// epilogue warps add a finished set into FP32 partial sums (forward: the item's rows of
// the partial-sum buffer; adjoint: the coil-combined value in registers) and release the
// set through an mbarrier that the MMA thread waits on before reusing it.
#include <algorithm>

#include "tc_common.cuh"

namespace aexp {

namespace {

// Issue the 24 MMAs of one stage (A_hi B_hi into the first accumulator, the cross products
// A_hi B_lo' and A_lo' B_hi into the second; K = 16 each) and commit both stage barriers.
template <int N>
__device__ __forceinline__ void tc_mma_stage(TcShared &sh, uint32_t tmem, const unsigned char *A,
                                             const unsigned char *B, bool first, int sa, int sb) {
    constexpr uint32_t IDESC = tc::idesc_f16(kRows, N, 0);  // FP16 operands
    // one descriptor per operand image; the K steps advance it
    const uint64_t da = tc::sdesc_k128(smem_u32(A)), db = tc::sdesc_k128(smem_u32(B));
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
        const uint32_t koff = (uint32_t)((kk >> 2) * (kRows * 128) + (kk & 3) * 32);
        const uint32_t kofb = (uint32_t)((kk >> 2) * (N * 128) + (kk & 3) * 32);
        tc::mma_f16(tmem, tc::sdesc_advance(da, koff), tc::sdesc_advance(db, kofb), IDESC, !(first && kk == 0));
    }
    const uint32_t t2 = tmem + tmem_acc_cols(N);
    const uint64_t da1 = tc::sdesc_advance(da, kA_BYTES), db1 = tc::sdesc_advance(db, N * 256);
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
        const uint32_t koff = (uint32_t)((kk >> 2) * (kRows * 128) + (kk & 3) * 32);
        const uint32_t kofb = (uint32_t)((kk >> 2) * (N * 128) + (kk & 3) * 32);
        tc::mma_f16(t2, tc::sdesc_advance(da, koff), tc::sdesc_advance(db1, kofb), IDESC, !(first && kk == 0));
    }
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
        const uint32_t koff = (uint32_t)((kk >> 2) * (kRows * 128) + (kk & 3) * 32);
        const uint32_t kofb = (uint32_t)((kk >> 2) * (N * 128) + (kk & 3) * 32);
        tc::mma_f16(t2, tc::sdesc_advance(da1, koff), tc::sdesc_advance(db, kofb), IDESC, 1u);
    }
    tc::mma_commit(&sh.afree[sa]);
    tc::mma_commit(&sh.bfree[sb]);
}

// (a, b) -> FP16 pairs hi = (fp16 a, fp16 b) and lo' = fp16(2^11 (a - hi.a)), fp16(2^11 (b - hi.b)),
// the low parts from one packed FMA: a - hi.a is exact in FP32 (hi.a is the rounding of a to
// fewer bits), and so is its product with 2^11.
__device__ __forceinline__ void split_hl(float a, float b, uint32_t &hi, uint32_t &lo) {
    const float2 v = make_float2(a, b);
    const __half2 h = __float22half2_rn(v);
    const float2 hf = __half22float2(h);
    const float2 l = __ffma2_rn(v, make_float2(kLoScale, kLoScale), __fmul2_rn(hf, make_float2(-kLoScale, -kLoScale)));
    const __half2 lh = __float22half2_rn(l);
    hi = *reinterpret_cast<const uint32_t *>(&h);
    lo = *reinterpret_cast<const uint32_t *>(&lh);
}

// Store one 16-byte chunk column (4 pairs) of both row slots: FP16 hi into the first A image,
// lo' into the second.
__device__ __forceinline__ void store_hl_chunks(unsigned char *A, int hh, int r0, int jp, const uint32_t (&whi)[2][4],
                                                const uint32_t (&wlo)[2][4]) {
    unsigned char *atom_base = A + hh * (kRows * 128);
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        const uint32_t o = tc::swz128(r0 + 32 * i, jp);
        *reinterpret_cast<uint4 *>(atom_base + o) = make_uint4(whi[i][0], whi[i][1], whi[i][2], whi[i][3]);
        *reinterpret_cast<uint4 *>(atom_base + kA_BYTES + o) = make_uint4(wlo[i][0], wlo[i][1], wlo[i][2], wlo[i][3]);
    }
}

// FP16 hi+lo promotion, forward: (D1 + 2^-11 D2) 2^-e of one accumulator set for this warp's
// 32 rows x N/2 columns (TMEM address `ta`), stored to or added into the partial sums `dst`.
template <int N>
__device__ __forceinline__ void fwd_promote(uint32_t ta, float inv, float4 *dst, bool add) {
    constexpr int CH = 8;
#pragma unroll 1
    for (int c0 = 0; c0 < N / 2; c0 += CH) {
        float v[CH], w[CH];
        tc::tmem_ld<CH>(ta + (uint32_t)c0, v);
        tc::tmem_ld<CH>(ta + tmem_acc_cols(N) + (uint32_t)c0, w);
        tc::tmem_ld_wait();
        tc::tmem_regs_ready<CH>(v);
        tc::tmem_regs_ready<CH>(w);
#pragma unroll
        for (int c = 0; c < CH / 4; ++c) {
            float4 o = make_float4(fmaf(w[4 * c], kLoInv, v[4 * c]) * inv, fmaf(w[4 * c + 1], kLoInv, v[4 * c + 1]) * inv,
                                   fmaf(w[4 * c + 2], kLoInv, v[4 * c + 2]) * inv,
                                   fmaf(w[4 * c + 3], kLoInv, v[4 * c + 3]) * inv);
            if (add) {
                const float4 q = dst[c0 / 4 + c];
                o.x += q.x;
                o.y += q.y;
                o.z += q.z;
                o.w += q.w;
            }
            dst[c0 / 4 + c] = o;
        }
    }
}

// FP16 hi+lo promotion, adjoint: xr + i xi += sum_c conj(S_c) (D1 + 2^-11 D2)_c over the
// coils of one accumulator set for this thread's voxel row (scale 2^-e applied by the caller).
template <int CB>
__device__ __forceinline__ void adj_promote(uint32_t ta, const float4 *s4, float &xr, float &xi) {
    constexpr uint32_t TM = tmem_acc_cols(2 * CB);
#pragma unroll 1
    for (int c0 = 0; c0 < CB; c0 += 8) {
        float ur[8], ui[8], wr[8], wi[8];
        tc::tmem_ld<8>(ta + (uint32_t)c0, ur);
        tc::tmem_ld<8>(ta + (uint32_t)(CB + c0), ui);
        tc::tmem_ld<8>(ta + TM + (uint32_t)c0, wr);
        tc::tmem_ld<8>(ta + TM + (uint32_t)(CB + c0), wi);
        tc::tmem_ld_wait();
        tc::tmem_regs_ready<8>(ur);
        tc::tmem_regs_ready<8>(ui);
        tc::tmem_regs_ready<8>(wr);
        tc::tmem_regs_ready<8>(wi);
#pragma unroll
        for (int q4 = 0; q4 < 4; ++q4) {
            const float4 sv = s4[c0 / 2 + q4];
            const float ar = fmaf(wr[2 * q4], kLoInv, ur[2 * q4]), ai = fmaf(wi[2 * q4], kLoInv, ui[2 * q4]);
            const float br = fmaf(wr[2 * q4 + 1], kLoInv, ur[2 * q4 + 1]);
            const float bi = fmaf(wi[2 * q4 + 1], kLoInv, ui[2 * q4 + 1]);
            xr = fmaf(sv.x, ar, xr);
            xr = fmaf(sv.y, ai, xr);
            xi = fmaf(sv.x, ai, xi);
            xi = fmaf(-sv.y, ar, xi);
            xr = fmaf(sv.z, br, xr);
            xr = fmaf(sv.w, bi, xr);
            xi = fmaf(sv.z, bi, xi);
            xi = fmaf(-sv.w, br, xi);
        }
    }
}

// MMA-thread bookkeeping of the accumulator-set barriers: every chunk but the last of an
// item is promoted once and arrives once on accfree[chunk & 1]; `base` counts the completed
// phases of both barriers over the items already done.
__device__ __forceinline__ void acc_advance(int (&base)[2], int nch) {
    if (nch > 0) {
        base[0] += nch / 2;
        base[1] += (nch - 1) / 2;
    }
}

// ---------------------------------------------------------------------------
// Warp roles and shared-memory plan of the FP16 hi+lo kernels
// ---------------------------------------------------------------------------
// Warps 0-15 generate the encoding tile of every stage (FP32 phases, sincos, hi/lo split);
// warp 16 issues the MMAs and owns TMEM; warp 17 loads the contraction operand B (hi | lo')
// into a 2-deep ring; warp 18 loads the generators' own operands (forward: the tile's basis
// offsets and the 128 rows' reference phases; adjoint: the stage's coefficient rows and both
// tiles' reference phases) into a ring of their own, 2-4 deep, which the generators release
// as soon as they have read it.  Keeping the generators' small operands out of the B ring
// lets them run ahead of the MMAs: a stage's B slot frees only when its 24 MMAs complete,
// its generator slot as soon as the tile has been generated.
constexpr int kHlMmaWarp = kTcGen / 32;
constexpr int kHlLoadBWarp = kHlMmaWarp + 1;
constexpr int kHlLoadGWarp = kHlMmaWarp + 2;
constexpr int kHlThreads = kTcGen + 96;
static_assert(kHlMmaWarp == kProdWarp, "the MMA warp allocates TMEM in tc_setup");

//   A[2] (hi | lo' images of a stage, 64 KB each) | B ring | generator-operand ring
template <int N, int LP, bool FWD>
struct HlPlan {
    static constexpr unsigned A_STAGE = 2 * kA_BYTES;
    static constexpr unsigned B_ALL = 2 * N * 256;                       // hi | lo', N rows x 128 K
    static constexpr unsigned G_OP = (FWD ? kTileVox : kCols) * LP * 4;  // basis offsets or coefficient rows
    static constexpr unsigned G_F0 = kRows * 4;                          // 128 reference phases
    static constexpr unsigned GS = (G_OP + G_F0 + 127u) & ~127u;
    static constexpr int NB = 2;
    static constexpr int NG = LP <= 20 ? 4 : 2;
    static constexpr unsigned OFF_B = 2 * A_STAGE;
    static constexpr unsigned OFF_G = OFF_B + NB * B_ALL;
    static constexpr unsigned BYTES = OFF_G + NG * GS;
    static_assert(NG <= kNBMax && NB <= kNBMax, "ring depths exceed the CTA's barriers");
};

// MMA thread, one item of n stages starting at CTA stage gs.
template <int N, int LP, bool FWD>
__device__ __forceinline__ int hl_mma_item(TcShared &sh, uint32_t tmem, unsigned char *gbase, int gs, int n,
                                           int (&acc_base)[2], int last_issued, int *status) {
    using PL = HlPlan<N, LP, FWD>;
    constexpr uint32_t SET_COLS = 2 * tmem_acc_cols(N);
    for (int it = 0; it < n; ++it) {
        const int g = gs + it, sa = g & 1, sb = g % PL::NB;
        const int m = it / kPromote;
        if (it % kPromote == 0 && m >= 2 &&
            !wait_or_abort(&sh.accfree[m & 1], (acc_base[m & 1] + ((m - 2) >> 1)) & 1, &sh.abort_flag, status))
            break;  // set m & 1 still holds chunk m - 2
        if (!wait_or_abort(&sh.afull[sa], (g >> 1) & 1, &sh.abort_flag, status)) break;
        if (!wait_or_abort(&sh.bfull[sb], (g / PL::NB) & 1, &sh.abort_flag, status)) break;
        tc::fence_after_sync();
        tc_mma_stage<N>(sh, tmem + (uint32_t)(m & 1) * SET_COLS, gbase + sa * PL::A_STAGE,
                        gbase + PL::OFF_B + sb * PL::B_ALL, it % kPromote == 0, sa, sb);
        last_issued = g;
    }
    acc_advance(acc_base, (n + kPromote - 1) / kPromote);
    return last_issued;
}

// ---------------------------------------------------------------------------
// Forward: item = (problem, block of 128 samples, run of voxel tiles)
// ---------------------------------------------------------------------------
template <int CB, int LP>
__global__ void __launch_bounds__(kHlThreads, 1)
    fwd_tc_kernel(const ProbDesc *__restrict__ pd, const int *__restrict__ item_off, int nprob, int *counter) {
    constexpr int N = 2 * CB;
    using PL = HlPlan<N, LP, true>;
    // two accumulator sets of (D1 | D2), alternating by chunk of kPromote stages
    constexpr uint32_t SET_COLS = 2 * tmem_acc_cols(N);
    constexpr unsigned TMEM_COLS = 2 * SET_COLS;

    extern __shared__ unsigned char smem_raw[];
    __shared__ TcShared sh;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const uint32_t sbase = align1024(smem_u32(smem_raw));
    unsigned char *gbase = smem_raw + (sbase - smem_u32(smem_raw));
    const int total = item_off[nprob];

    // accumulator sets are released by warps 0-7; A stages and generator slots by every generator
    tc_setup(sh, tid, warp, TMEM_COLS, 256, kTcGen, kTcGen / 32, kTcGen);
    const uint32_t tmem = sh.tmem_base;
    int gs = 0;            // stages (tiles) this CTA has processed
    int last_issued = -1;  // MMA thread: last stage whose MMAs were committed
    int acc_base[2] = {0, 0};

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

        if (warp >= kHlMmaWarp) {
            const bool lead = (tid & 31) == 0;
            if (warp == kHlMmaWarp && lead) {
                last_issued = hl_mma_item<N, LP, true>(sh, tmem, gbase, gs, ntl, acc_base, last_issued, status);
            } else if (warp == kHlLoadBWarp && lead) {
                ring_load_item(sh.bfree, PL::NB, gs, ntl, &sh.abort_flag, status, [&](int it, int sb) {
                    const size_t tile = (size_t)(tile0 + it);  // packed S x of the tile, hi | lo'
                    mbar_arrive_expect_tx(&sh.bfull[sb], PL::B_ALL);
                    bulk_g2s(gbase + PL::OFF_B + sb * PL::B_ALL, P.bpk + tile * PL::B_ALL, PL::B_ALL, &sh.bfull[sb]);
                });
            } else if (warp == kHlLoadGWarp && lead) {
                ring_load_item(sh.pfree, PL::NG, gs, ntl, &sh.abort_flag, status, [&](int it, int sg) {
                    const size_t tile = (size_t)(tile0 + it);  // basis offsets and the rows' reference phases
                    unsigned char *dst = gbase + PL::OFF_G + sg * PL::GS;
                    mbar_arrive_expect_tx(&sh.pfull[sg], PL::G_OP + PL::G_F0);
                    bulk_g2s(dst, P.dh + tile * kTileVox * LP, PL::G_OP, &sh.pfull[sg]);
                    bulk_g2s(dst + PL::G_OP, P.f0 + tile * ntp + tbase, PL::G_F0, &sh.pfull[sg]);
                });
            }
        } else {
            // generator: warp w owns chunk columns (w & 7) and (w & 7) + 8, lane g owns rows
            // r0 = 64 (w >> 3) + g and r0 + 32 with their coefficients (times 2 pi: phases in
            // radians) in registers
            const int jp = warp & 7;
            const int r0 = 64 * (warp >> 3) + (tid & 31);
            float2 k[2][LP / 2];  // (even term, odd term)
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int q4 = 0; q4 < LP / 4; ++q4) {
                    float4 w = reinterpret_cast<const float4 *>(P.khi_t + (size_t)(tbase + r0 + 32 * i) * LP)[q4];
                    k[i][2 * q4] = make_float2(kTwoPi * w.x, kTwoPi * w.y);
                    k[i][2 * q4 + 1] = make_float2(kTwoPi * w.z, kTwoPi * w.w);
                }
            // epilogue rows and columns (warps 0-7): 32 samples x N/2 columns per warp, computed
            // where used so that they hold no registers during the generation
            auto epi_dst = [&]() {
                return reinterpret_cast<float4 *>(P.fpart +
                                                  ((size_t)split * ntp + tbase + 32 * (warp & 3) + (tid & 31)) * N +
                                                  ((warp >> 2) & 1) * (N / 2));
            };
            auto epi_tmem = [&]() {
                return tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(((warp >> 2) & 1) * (N / 2));
            };
            int next_promo = 0;  // next accumulator chunk to promote
            for (int it = 0; it < ntl; ++it) {
                const int g = gs + it, sa = g & 1, sg = g % PL::NG;
                bool w_ok = wait_or_abort(&sh.pfull[sg], (g / PL::NG) & 1, &sh.abort_flag, status);
                if (w_ok && g >= 2) w_ok = wait_or_abort(&sh.afree[sa], ((g - 2) >> 1) & 1, &sh.abort_flag, status);
                if (!__all_sync(0xffffffffu, w_ok)) break;  // warp-uniform exit
                // stages <= it - 2 are complete: promote a finished chunk and release its set
                if (next_promo < (it - 1) / kPromote) {
                    if (warp < 8) {
                        tc::fence_after_sync();
                        fwd_promote<N>(epi_tmem() + (uint32_t)(next_promo & 1) * SET_COLS,
                                       hl_scale(P.hdr->amax[0], true), epi_dst(), next_promo > 0);
                        tc::fence_before_sync();
                        tc::mbar_arrive(&sh.accfree[next_promo & 1]);
                    }
                    ++next_promo;
                }
                const unsigned char *gsl = gbase + PL::OFF_G + sg * PL::GS;
                const float4 *DH = reinterpret_cast<const float4 *>(gsl);
                const float *F0 = reinterpret_cast<const float *>(gsl + PL::G_OP);
                const float f[2] = {kTwoPi * F0[r0], kTwoPi * F0[r0 + 32]};
                unsigned char *A = gbase + sa * PL::A_STAGE;
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const int j = jp + 8 * hh;  // chunk of 4 voxels; atom hh, swizzle column jp
                    uint32_t whi[2][4], wlo[2][4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        float2 d[LP / 2];
#pragma unroll
                        for (int q4 = 0; q4 < LP / 4; ++q4) {
                            float4 w = DH[(4 * j + u) * (LP / 4) + q4];
                            d[2 * q4] = make_float2(w.x, w.y);
                            d[2 * q4 + 1] = make_float2(w.z, w.w);
                        }
#pragma unroll
                        for (int i = 0; i < 2; ++i) {
                            // even and odd terms in the two lanes of packed FMAs (each lane as fmaf)
                            float2 pp = make_float2(f[i], 0.f);
#pragma unroll
                            for (int l = 0; l < LP / 2; ++l) pp = __ffma2_rn(k[i][l], d[l], pp);
                            // E = cos phi - i sin phi = cos(-phi) + i sin(-phi); the angle spans a few
                            // turns (reference phase in [-pi, pi) plus the tile's offset), within the
                            // range where the hardware sincos needs no reduction of our own
                            float sn, cs;
                            __sincosf(-(pp.x + pp.y), &sn, &cs);
                            split_hl(cs, sn, whi[i][u], wlo[i][u]);
                        }
                    }
                    store_hl_chunks(A, hh, r0, jp, whi, wlo);
                }
                tc::mbar_arrive(&sh.pfree[sg]);  // the generator slot has been read
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
                float4 *dst = epi_dst();
                const uint32_t ta0 = epi_tmem();
                if (ntl > 0 && ok) {
                    // the remaining (at most two) chunks; all but the item's last release their set
                    const int nch = (ntl + kPromote - 1) / kPromote;
                    const float inv = hl_scale(P.hdr->amax[0], true);
                    for (int m = next_promo; m < nch; ++m) {
                        fwd_promote<N>(ta0 + (uint32_t)(m & 1) * SET_COLS, inv, dst, m > 0);
                        if (m < nch - 1) {
                            tc::fence_before_sync();
                            tc::mbar_arrive(&sh.accfree[m & 1]);
                        }
                    }
                } else {
#pragma unroll
                    for (int c = 0; c < N / 8; ++c) dst[c] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
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
__global__ void __launch_bounds__(kHlThreads, 1)
    adj_tc_kernel(const ProbDesc *__restrict__ pd, const int *__restrict__ item_off, int nprob, int *counter) {
    constexpr int N = 2 * CB;
    constexpr int TS = kCols;  // samples per stage
    using PL = HlPlan<N, LP, false>;
    constexpr uint32_t SET_COLS = 2 * tmem_acc_cols(N);
    constexpr unsigned TMEM_COLS = 2 * SET_COLS;

    extern __shared__ unsigned char smem_raw[];
    __shared__ TcShared sh;
    const int tid = threadIdx.x;
    const int warp = tid >> 5;
    const uint32_t sbase = align1024(smem_u32(smem_raw));
    unsigned char *gbase = smem_raw + (sbase - smem_u32(smem_raw));
    const int total = item_off[nprob];

    // accumulator sets are released by warps 0-3; A stages and generator slots by every generator
    tc_setup(sh, tid, warp, TMEM_COLS, 128, kTcGen, kTcGen / 32, kTcGen);
    const uint32_t tmem = sh.tmem_base;
    int gs = 0;
    int last_issued = -1;
    int acc_base[2] = {0, 0};

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

        if (warp >= kHlMmaWarp) {
            const bool lead = (tid & 31) == 0;
            if (warp == kHlMmaWarp && lead) {
                last_issued = hl_mma_item<N, LP, false>(sh, tmem, gbase, gs, nst, acc_base, last_issued, status);
            } else if (warp == kHlLoadBWarp && lead) {
                ring_load_item(sh.bfree, PL::NB, gs, nst, &sh.abort_flag, status, [&](int it, int sb) {
                    const size_t ts = (size_t)t0 + (size_t)it * TS;  // packed k-space of the stage, hi | lo'
                    mbar_arrive_expect_tx(&sh.bfull[sb], PL::B_ALL);
                    bulk_g2s(gbase + PL::OFF_B + sb * PL::B_ALL, P.ypk + (ts / TS) * PL::B_ALL, PL::B_ALL,
                             &sh.bfull[sb]);
                });
            } else if (warp == kHlLoadGWarp && lead) {
                ring_load_item(sh.pfree, PL::NG, gs, nst, &sh.abort_flag, status, [&](int it, int sg) {
                    const size_t ts = (size_t)t0 + (size_t)it * TS;  // coefficient rows, both tiles' f0
                    unsigned char *dst = gbase + PL::OFF_G + sg * PL::GS;
                    mbar_arrive_expect_tx(&sh.pfull[sg], PL::G_OP + 2 * TS * 4);
                    bulk_g2s(dst, P.khi_t + ts * LP, PL::G_OP, &sh.pfull[sg]);
                    bulk_g2s(dst + PL::G_OP, P.f0 + (size_t)tileA * ntp + ts, TS * 4, &sh.pfull[sg]);
                    bulk_g2s(dst + PL::G_OP + TS * 4, P.f0 + (size_t)tileB * ntp + ts, TS * 4, &sh.pfull[sg]);
                });
            }
        } else {
            // generator: warp w owns sample chunks (w & 7) and (w & 7) + 8 of each stage; lane g
            // owns voxel rows r0 = 64 (w >> 3) + g and r0 + 32 (both in tile w >> 3 of the item)
            // with their basis offsets (times 2 pi: phases in radians) in registers
            const int jp = warp & 7;
            const int th = warp >> 3;
            const int r0 = 64 * th + (tid & 31);
            float2 d[2][LP / 2];  // (even term, odd term)
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int p = vb * kRows + r0 + 32 * i;
                const bool valid = p < ntiles * kTileVox;
#pragma unroll
                for (int q4 = 0; q4 < LP / 4; ++q4) {
                    float4 w = reinterpret_cast<const float4 *>(P.dh + (size_t)(valid ? p : 0) * LP)[q4];
                    d[i][2 * q4] = valid ? make_float2(kTwoPi * w.x, kTwoPi * w.y) : make_float2(0.f, 0.f);
                    d[i][2 * q4 + 1] = valid ? make_float2(kTwoPi * w.z, kTwoPi * w.w) : make_float2(0.f, 0.f);
                }
            }
            // epilogue row (warps 0-3): voxel p = vb * 128 + 32 warp + lane; addressing computed
            // where used so that it holds no registers during the generation
            auto epi_row = [&]() { return vb * kRows + 32 * (warp & 3) + (tid & 31); };
            auto epi_s4 = [&]() {
                const int pr = epi_row();
                return reinterpret_cast<const float4 *>(P.Sp + (size_t)(pr < ntiles * kTileVox ? pr : 0) * CB);
            };
            auto epi_tmem = [&]() { return tmem + ((uint32_t)(32 * (warp & 3)) << 16); };
            float xr = 0.f, xi = 0.f;  // promoted, coil-combined partial sum
            int next_promo = 0;
            for (int it = 0; it < nst; ++it) {
                const int g = gs + it, sa = g & 1, sg = g % PL::NG;
                bool w_ok = wait_or_abort(&sh.pfull[sg], (g / PL::NG) & 1, &sh.abort_flag, status);
                if (w_ok && g >= 2) w_ok = wait_or_abort(&sh.afree[sa], ((g - 2) >> 1) & 1, &sh.abort_flag, status);
                if (!__all_sync(0xffffffffu, w_ok)) break;  // warp-uniform exit
                // stages <= it - 2 are complete: promote a finished chunk and release its set
                if (next_promo < (it - 1) / kPromote) {
                    if (warp < 4) {
                        tc::fence_after_sync();
                        adj_promote<CB>(epi_tmem() + (uint32_t)(next_promo & 1) * SET_COLS, epi_s4(), xr, xi);
                        tc::fence_before_sync();
                        tc::mbar_arrive(&sh.accfree[next_promo & 1]);
                    }
                    ++next_promo;
                }
                const unsigned char *gsl = gbase + PL::OFF_G + sg * PL::GS;
                const float4 *KS = reinterpret_cast<const float4 *>(gsl);
                const float4 *FS = reinterpret_cast<const float4 *>(gsl + PL::G_OP);
                unsigned char *A = gbase + sa * PL::A_STAGE;
#pragma unroll
                for (int hh = 0; hh < 2; ++hh) {
                    const int j = jp + 8 * hh;  // samples 4j..4j+3 of the stage
                    const float4 fa = FS[th * (TS / 4) + j];
                    const float fA[4] = {kTwoPi * fa.x, kTwoPi * fa.y, kTwoPi * fa.z, kTwoPi * fa.w};
                    uint32_t whi[2][4], wlo[2][4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        float2 kk[LP / 2];
#pragma unroll
                        for (int q4 = 0; q4 < LP / 4; ++q4) {
                            float4 w = KS[(4 * j + u) * (LP / 4) + q4];
                            kk[2 * q4] = make_float2(w.x, w.y);
                            kk[2 * q4 + 1] = make_float2(w.z, w.w);
                        }
#pragma unroll
                        for (int i = 0; i < 2; ++i) {
                            float2 pp = make_float2(fA[u], 0.f);
#pragma unroll
                            for (int l = 0; l < LP / 2; ++l) pp = __ffma2_rn(kk[l], d[i][l], pp);
                            float sn, cs;
                            __sincosf(pp.x + pp.y, &sn, &cs);  // conj(E) = cos phi + i sin phi
                            split_hl(cs, sn, whi[i][u], wlo[i][u]);
                        }
                    }
                    store_hl_chunks(A, hh, r0, jp, whi, wlo);
                }
                tc::mbar_arrive(&sh.pfree[sg]);  // the generator slot has been read
                tc::fence_proxy_async_smem();
                tc::mbar_arrive(&sh.afull[sa]);
            }
            // epilogue (warps 0-3, one voxel row per thread): conj(S) . u over coils, read
            // from TMEM in chunks of 8 coils (u = (D1 + 2^-11 D2) 2^-e)
            bool ok = !sh.abort_flag;
            const int gl = gs + nst - 1;
            if (nst > 0 && ok) ok = wait_or_abort(&sh.afree[gl & 1], (gl >> 1) & 1, &sh.abort_flag, status);
            ok = __all_sync(0xffffffffu, ok);  // tcgen05.ld is warp-collective
            tc::fence_after_sync();
            if (warp < 4) {
                const bool have = nst > 0 && ok;
                const int p_row = epi_row();
                const bool inside = p_row < ntiles * kTileVox;
                const uint32_t ta0 = epi_tmem();
                const float4 *s4 = epi_s4();
                if (have) {
                    // the remaining (at most two) chunks; all but the item's last release their set
                    const int nch = (nst + kPromote - 1) / kPromote;
                    for (int m = next_promo; m < nch; ++m) {
                        adj_promote<CB>(ta0 + (uint32_t)(m & 1) * SET_COLS, s4, xr, xi);
                        if (m < nch - 1) {
                            tc::fence_before_sync();
                            tc::mbar_arrive(&sh.accfree[m & 1]);
                        }
                    }
                    const float inv = hl_scale(P.hdr->amax[1], true);
                    xr *= inv;
                    xi *= inv;
                } else {
                    xr = xi = 0.f;
                }
                if (inside) P.apart[(size_t)split * (size_t)(ntiles * kTileVox) + p_row] = make_float2(xr, xi);
            }
        }
        gs += nst;
    }
    tc_teardown(sh, warp, TMEM_COLS, last_issued, &pd[0].hdr->status);
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
template <int CB, int LP>
size_t fwd_tc_smem() {
    return 1024 + HlPlan<2 * CB, LP, true>::BYTES;
}
template <int CB, int LP>
size_t adj_tc_smem() {
    return 1024 + HlPlan<2 * CB, LP, false>::BYTES;
}

// max_pack_blocks: the amax grid of the largest problem (see pack_grid for the packing grid).
template <int CB, int LP>
cudaError_t launch_fwd_tc(const ProbDesc *pd, int nprob, int max_pack_blocks, const float2 *x, int src,
                          const int *item_off, int total_items, int *counter, cudaStream_t st) {
    amax_reset_kernel<<<cdiv(nprob, 256), 256, 0, st>>>(pd, nprob, 0);
    amax_b_kernel<CB><<<dim3(max_pack_blocks, nprob), 256, 0, st>>>(pd, x, src);
    pack_b_fwd_kernel<CB, kPackHL><<<dim3(pack_grid(max_pack_blocks, CB), nprob), 256, 0, st>>>(pd, x, src);
    auto kern = fwd_tc_kernel<CB, LP>;
    const size_t smem = fwd_tc_smem<CB, LP>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    kern<<<std::min(total_items, num_sms()), kHlThreads, smem, st>>>(pd, item_off, nprob, counter);
    return cudaGetLastError();
}

template <int CB, int LP>
cudaError_t launch_adj_tc(const ProbDesc *pd, int nprob, int max_pack_blocks, const float2 *yt, int src,
                          const int *item_off, int total_items, int *counter, cudaStream_t st) {
    amax_reset_kernel<<<cdiv(nprob, 256), 256, 0, st>>>(pd, nprob, 1);
    amax_y_kernel<CB><<<dim3(max_pack_blocks, nprob), 256, 0, st>>>(pd, yt, src);
    pack_y_adj_kernel<CB, kPackHL><<<dim3(pack_grid(max_pack_blocks, CB), nprob), 256, 0, st>>>(pd, yt, src);
    auto kern = adj_tc_kernel<CB, LP>;
    const size_t smem = adj_tc_smem<CB, LP>();
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess) e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    kern<<<std::min(total_items, num_sms()), kHlThreads, smem, st>>>(pd, item_off, nprob, counter);
    return cudaGetLastError();
}

#define AEXP_TC_LP(FN, CBV, ...)                         \
    switch (LPv) {                                       \
        case 4: return FN<CBV, 4>(__VA_ARGS__);          \
        case 8: return FN<CBV, 8>(__VA_ARGS__);          \
        case 12: return FN<CBV, 12>(__VA_ARGS__);        \
        case 20: return FN<CBV, 20>(__VA_ARGS__);        \
        default: return FN<CBV, 32>(__VA_ARGS__);        \
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
    if (L.precision == AEXP_BF16_TC || L.variant == 0)
        return tcp_forward(L.precision, L.CB, L.variant, pd, 1, fwd_pack_blocks(L.ntiles, L.CB), x, 0, &hdr->item_off[0], L.fwd_items,
                           &hdr->counter[0], st);
    AEXP_TC_DISPATCH(launch_fwd_tc, pd, 1, fwd_pack_blocks(L.ntiles, L.CB), x, 0, &hdr->item_off[0], L.fwd_items,
                     &hdr->counter[0], st)
}

cudaError_t op_adjoint_tc(const OpLayout &L, const float2 *yt, char *ws, cudaStream_t st) {
    const int CBv = L.CB, LPv = L.LP;
    WsHeader *hdr = (WsHeader *)(ws + L.off_hdr);
    const ProbDesc *pd = (const ProbDesc *)(ws + L.off_desc);
    if (L.precision == AEXP_BF16_TC || L.variant == 0)
        return tcp_adjoint(L.precision, L.CB, L.variant, pd, 1, adj_pack_blocks(L.ntp, L.CB), yt, -1, &hdr->item_off[2], L.adj_items,
                           &hdr->counter[1], st);
    AEXP_TC_DISPATCH(launch_adj_tc, pd, 1, adj_pack_blocks(L.ntp, L.CB), yt, -1, &hdr->item_off[2], L.adj_items,
                     &hdr->counter[1], st)
}

cudaError_t op_residual_adjoint_tc(const OpLayout &L, char *ws, const float2 *ymeas_t, cudaStream_t st) {
    WsHeader *hdr = (WsHeader *)(ws + L.off_hdr);
    const ProbDesc *pd = (const ProbDesc *)(ws + L.off_desc);
    return tcp_residual_adjoint_bf16(L.CB, L.variant, pd, 1, adj_pack_blocks(L.ntp, L.CB), ymeas_t, -1,
                                     &hdr->item_off[2], L.adj_items, &hdr->counter[1], st);
}

cudaError_t batch_forward_tc(int precision, int CB, int LP, int variant, const ProbDesc *pd, int nprob,
                             int max_pack_blocks, int src, const int *item_off, int total_items, int *counter,
                             cudaStream_t st) {
    const int CBv = CB, LPv = LP;
    if (precision == AEXP_BF16_TC || variant == 0)
        return tcp_forward(precision, CB, variant, pd, nprob, max_pack_blocks, nullptr, src, item_off, total_items, counter, st);
    AEXP_TC_DISPATCH(launch_fwd_tc, pd, nprob, max_pack_blocks, nullptr, src, item_off, total_items, counter, st)
}

cudaError_t batch_adjoint_tc(int precision, int CB, int LP, int variant, const ProbDesc *pd, int nprob,
                             int max_pack_blocks, int src, const int *item_off, int total_items, int *counter,
                             cudaStream_t st) {
    const int CBv = CB, LPv = LP;
    if (precision == AEXP_BF16_TC || variant == 0)
        return tcp_adjoint(precision, CB, variant, pd, nprob, max_pack_blocks, nullptr, src, item_off, total_items, counter, st);
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
