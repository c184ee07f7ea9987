// Host-side workspace layouts and launch-shape heuristics.
#include <algorithm>

#include "aexp_internal.cuh"

namespace aexp {

namespace {
int pad_terms(int n) { return n <= 4 ? 4 : n <= 8 ? 8 : n <= 12 ? 12 : n <= 20 ? 20 : 32; }
int pad_coils(int n) { return n <= 4 ? 4 : n <= 8 ? 8 : n <= 16 ? 16 : n <= 20 ? 20 : 32; }
// tensor-core forms: N = 2 * CB must be a multiple of 16 with a power-of-two half for TMEM loads
int pad_coils_tc(int n) { return n <= 8 ? 8 : n <= 16 ? 16 : 32; }
}  // namespace

int op_layout(const aexp_problem *p, int precision, OpLayout *L, int target_items, int variant) {
    if (target_items <= 0) target_items = items_target(precision, 0);
    OpLayout o{};
    o.nx = p->nx;
    o.ny = p->ny;
    o.nr = p->nx * p->ny;
    o.nt = p->nt;
    o.nc = p->nc;
    o.nl = p->nl;
    o.has_b0 = p->omega != nullptr;
    o.nterms = o.nl + o.has_b0;
    o.LP = pad_terms(o.nterms);
    o.CB = precision == AEXP_FP32 ? pad_coils(o.nc) : pad_coils_tc(o.nc);
    o.precision = precision;
    o.variant = variant;
    o.ntx = cdiv(o.nx, kTileSide);
    o.nty = cdiv(o.ny, kTileSide);
    o.ntiles = o.ntx * o.nty;
    o.nr_pad = o.ntiles * kTileVox;
    o.ntp = cdiv(o.nt, kTPad) * kTPad;

    // forward: blocks own 128*mt samples and a contiguous run of tiles
    const bool alt32 = precision == AEXP_FP32 && o.CB == 32 && variant == 1;
    o.fwd_mt = alt32 ? kFp32AltBlocking : fwd_mt_for(o.CB);
    o.fwd_tblocks = o.ntp / (kFwdThreads * o.fwd_mt);
    {
        int by_sum = cdiv(o.ntiles, 32);                       // <= 32 tiles (2048 voxels) per block
        int by_occ = cdiv(target_items, o.fwd_tblocks);
        int s = std::max(by_sum, by_occ);
        s = std::min(s, o.ntiles);
        o.fwd_tiles_per_split = cdiv(o.ntiles, s);
        o.fwd_splits = cdiv(o.ntiles, o.fwd_tiles_per_split);
    }
    // adjoint: blocks own 2*mr tiles (128*mr voxels) and a contiguous run of samples
    o.adj_mr = alt32 ? kFp32AltBlocking : adj_mr_for(o.CB);
    o.adj_vblocks = cdiv(o.ntiles, 2 * o.adj_mr);
    {
        int nstage = o.ntp / kAdjStageT;
        int by_sum = cdiv(o.ntp, 2048);
        int by_occ = cdiv(target_items, o.adj_vblocks);
        int s = std::min(std::max(by_sum, by_occ), nstage);
        int stages_per = cdiv(nstage, s);
        o.adj_t_per_split = stages_per * kAdjStageT;
        o.adj_splits = cdiv(o.ntp, o.adj_t_per_split);
    }

    if (precision != AEXP_FP32) {
        // one CTA (128 samples or 2 tiles) per SM at a time; split the reduction dimension
        // so the grid covers ~8 waves
        const int tblocks = o.ntp / 128;
        int s = std::min(std::max(cdiv(target_items, tblocks), 1), o.ntiles);
        o.fwd_tblocks = tblocks;
        o.fwd_tiles_per_split = cdiv(o.ntiles, s);
        o.fwd_splits = cdiv(o.ntiles, o.fwd_tiles_per_split);
        o.adj_vblocks = cdiv(o.ntiles, 2);
        const int nstage = o.ntp / kAdjStageT;
        s = std::min(std::max(cdiv(target_items, o.adj_vblocks), 1), nstage);
        o.adj_t_per_split = cdiv(nstage, s) * kAdjStageT;
        o.adj_splits = cdiv(o.ntp, o.adj_t_per_split);
    }

    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = align_up(off + bytes);
        return at;
    };
    o.off_hdr = take(sizeof(WsHeader));
    o.off_khi_l = take(sizeof(float) * o.LP * o.ntp);
    o.off_klo_l = take(sizeof(float) * o.LP * o.ntp);
    o.off_khi_t = take(sizeof(float) * o.LP * o.ntp);
    o.off_h0 = take(sizeof(float) * o.LP * o.ntiles);
    o.off_dh = take(sizeof(float) * o.LP * o.nr_pad);
    o.off_f0 = take(sizeof(float) * (size_t)o.ntiles * o.ntp);
    o.off_S = take(sizeof(float2) * (size_t)o.CB * o.nr_pad);
    // FP32: b = S x in tile order; tensor-core forms: the packed B operand (FP16 hi+lo: two images)
    const size_t npk = precision == AEXP_FP16X2_TC ? 2 : 1;
    o.off_b = take(npk * sizeof(float2) * (size_t)o.CB * o.nr_pad);
    o.off_fpart = take(sizeof(float2) * (size_t)o.fwd_splits * o.ntp * o.CB);
    o.off_yt = take(sizeof(float2) * (size_t)o.ntp * o.CB);
    o.off_apart = take(sizeof(float2) * (size_t)o.adj_splits * o.nr_pad);
    o.off_ypk = take(precision == AEXP_FP32 ? 0 : npk * sizeof(float2) * (size_t)o.ntp * o.CB);
    o.off_desc = take(sizeof(ProbDesc));
    o.off_hp = take(sizeof(float) * (size_t)o.LP * o.nr_pad);
    const bool tcp = precision != AEXP_FP32;  // the phase-GEMM operands of both tensor-core forms
    o.off_kph = take(tcp ? (size_t)(o.ntp / 128) * kPhaseBlockBytes : 0);
    o.off_dhph = take(tcp ? (size_t)cdiv(o.ntiles, 2) * kPhaseBlockBytes : 0);
    o.fwd_items = o.fwd_tblocks * o.fwd_splits;
    o.adj_items = o.adj_vblocks * o.adj_splits;
    o.bytes = off;
    *L = o;
    return AEXP_OK;
}

int wave_layout(int nx, int ny, int wavelet, int levels, WaveLayout *W) {
    WaveLayout w{};
    w.nx = nx;
    w.ny = ny;
    w.levels = levels;
    w.wavelet = wavelet;
    int q = 1 << levels;
    w.npx = cdiv(nx, q) * q;
    w.npy = cdiv(ny, q) * q;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = align_up(off + bytes);
        return at;
    };
    w.off_pyr = take(sizeof(float2) * (size_t)w.npx * w.npy);
    for (int j = 1; j < levels; ++j)
        w.off_approx[j] = take(sizeof(float2) * (size_t)(w.npx >> j) * (w.npy >> j));
    w.bytes = off;
    *W = w;
    return AEXP_OK;
}

int rec_layout(const aexp_problem *p, const aexp_recon_opts *opt, RecLayout *R, int target_items,
               int with_grad) {
    RecLayout r{};
    if (target_items < 0) target_items = items_target(opt->precision, opt->items_per_sm);
    int rc = op_layout(p, opt->precision, &r.op, target_items, opt->tile_variant);
    if (rc) return rc;
    rc = wave_layout(p->nx, p->ny, opt->wavelet, opt->levels, &r.wv);
    if (rc) return rc;
    size_t off = r.op.bytes;
    auto take = [&](size_t bytes) {
        size_t at = off;
        off = align_up(off + bytes);
        return at;
    };
    size_t nr = (size_t)r.op.nr;
    // vectors first so that their offsets do not depend on the wavelet options
    r.off_ymeas = take(sizeof(float2) * (size_t)r.op.ntp * r.op.CB);
    r.off_xa = take(sizeof(float2) * nr);
    r.off_xb = take(sizeof(float2) * nr);
    r.off_z = take(sizeof(float2) * nr);
    r.off_v = take(sizeof(float2) * nr);
    r.off_w = take(sizeof(float2) * nr);
    r.off_wave = take(r.wv.bytes);
    if (opt->undecimated) {
        r.off_swt = take(4 * sizeof(float2) * nr);
        r.off_swtaux = take(swt_aux_bytes());
    }
    if (with_grad) {
        const OpLayout &L = r.op;
        const int tblocks = L.ntp / 128;
        int s = std::max(cdiv(L.ntiles, 32), cdiv(152 * 8, tblocks));
        s = std::min(s, L.ntiles);
        r.grad_tiles_per_split = cdiv(L.ntiles, s);
        r.grad_splits = cdiv(L.ntiles, r.grad_tiles_per_split);
        r.off_rk = take(sizeof(float2) * (size_t)L.ntp * L.CB);
        r.off_xbar = take(sizeof(float2) * nr);
        r.off_vbar = take(sizeof(float2) * nr);
        r.off_wave2 = take(r.wv.bytes);
        r.off_zq = take(sizeof(float2) * (size_t)L.nr_pad);
        r.off_gq = take(sizeof(float2) * (size_t)L.nr_pad);
        r.off_gpart = take(sizeof(float) * (size_t)r.grad_splits * L.LP * L.ntp);
    }
    r.bytes = off;
    *R = r;
    return AEXP_OK;
}

}  // namespace aexp

namespace aexp {

ProbDesc make_op_desc(const OpLayout &L, char *ws) {
    ProbDesc d{};
    d.nx = L.nx;
    d.ny = L.ny;
    d.nr = L.nr;
    d.nt = L.nt;
    d.nc = L.nc;
    d.ntp = L.ntp;
    d.ntiles = L.ntiles;
    d.ntx = L.ntx;
    d.nr_pad = L.nr_pad;
    d.CB = L.CB;
    d.LP = L.LP;
    d.fwd_splits = L.fwd_splits;
    d.fwd_tps = L.fwd_tiles_per_split;
    d.adj_splits = L.adj_splits;
    d.adj_tps = L.adj_t_per_split;
    d.adj_vblocks = L.adj_vblocks;
    d.khi_t = (const float *)(ws + L.off_khi_t);
    d.f0 = (const float *)(ws + L.off_f0);
    d.dh = (const float *)(ws + L.off_dh);
    d.Sp = (const float2 *)(ws + L.off_S);
    d.bpk = (unsigned char *)(ws + L.off_b);
    d.ypk = (unsigned char *)(ws + L.off_ypk);
    d.kph = (const unsigned char *)(ws + L.off_kph);
    d.dhph = (const unsigned char *)(ws + L.off_dhph);
    d.fpart = (float *)(ws + L.off_fpart);
    d.apart = (float2 *)(ws + L.off_apart);
    d.rt = (float2 *)(ws + L.off_yt);
    d.hdr = (WsHeader *)(ws + L.off_hdr);
    return d;
}

int num_sms() {
    static int n = 0;
    if (n == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
            n = 152;
    }
    return n;
}

}  // namespace aexp
