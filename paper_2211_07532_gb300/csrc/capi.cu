// The C ABI (include/aexp.h): argument validation, workspace sizing, the host-side
// record of prepared workspaces, CUDA-graph capture of cs_recon, status strings.
#include <string.h>

#include <mutex>
#include <unordered_map>
#include <vector>

#include "aexp_internal.cuh"
#include "batch_internal.h"

using namespace aexp;

namespace {

thread_local int g_last_cuda_error = 0;

int cuda_fail(cudaError_t e) {
    g_last_cuda_error = (int)e;
    return AEXP_ERR_CUDA;
}

bool aligned(const void *p, size_t a) { return ((uintptr_t)p % a) == 0; }

int check_problem(const aexp_problem *p) {
    if (!p) return AEXP_ERR_INVALID_ARG;
    if (p->nx < 1 || p->ny < 1 || p->nt < 1 || p->nc < 1 || p->nl < 0) return AEXP_ERR_INVALID_ARG;
    if ((long long)p->nx * p->ny > (1LL << 28) || p->nt > (1 << 28)) return AEXP_ERR_UNSUPPORTED;
    int nterms = p->nl + (p->omega != nullptr);
    if (nterms < 1) return AEXP_ERR_INVALID_ARG;
    if (nterms > kMaxTerms || p->nc > kMaxCoils) return AEXP_ERR_UNSUPPORTED;
    // grid.y limits: one row of blocks per tile (reference phases) and per sample stage
    if ((long long)cdiv(p->nx, kTileSide) * cdiv(p->ny, kTileSide) > 65535) return AEXP_ERR_UNSUPPORTED;
    if ((long long)p->nt > 65535LL * kAdjStageT - kTPad) return AEXP_ERR_UNSUPPORTED;
    if ((p->nl > 0 && (!p->k || !p->h)) || !p->S) return AEXP_ERR_INVALID_ARG;
    if (p->omega && !p->t) return AEXP_ERR_INVALID_ARG;
    if (!aligned(p->k, 4) || !aligned(p->h, 4) || !aligned(p->omega, 4) || !aligned(p->t, 4) ||
        !aligned(p->S, 8))
        return AEXP_ERR_MISALIGNED;
    return AEXP_OK;
}

int check_precision(int precision) {
    if (precision != AEXP_FP32 && precision != AEXP_BF16_TC && precision != AEXP_FP16X2_TC)
        return AEXP_ERR_INVALID_ARG;
    return AEXP_OK;
}

int check_ws(const void *ws, size_t have, size_t need) {
    if (!ws) return AEXP_ERR_INVALID_ARG;
    if (!aligned(ws, kAlign)) return AEXP_ERR_MISALIGNED;
    if (have < need) return AEXP_ERR_WORKSPACE;
    return AEXP_OK;
}

// Host-side record of which problem a workspace was last prepared for.
struct PrepRecord {
    aexp_problem prob;
    int precision;
    int items_per_sm;  // layout granularity the workspace was prepared with (0 = default)
    int tile_variant;  // kernel tiling of that layout
};
std::mutex g_mu;
std::unordered_map<const void *, PrepRecord> g_prepared;

bool same_problem(const aexp_problem &a, const aexp_problem &b) { return memcmp(&a, &b, sizeof(a)) == 0; }

// the granularity a layout actually uses (0 stands for the precision's default)
int effective_items(int precision, int items_per_sm) {
    return items_per_sm > 0 ? items_per_sm : default_items_per_sm(precision);
}

void record_prepared(const void *ws, const aexp_problem *p, int precision, int items_per_sm = 0, int variant = 0) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_prepared[ws] = PrepRecord{*p, precision, effective_items(precision, items_per_sm), variant};
}

// The layout granularity and tiling `ws` was last prepared with for (p, precision), if any.
bool prepared_tiling(const void *ws, const aexp_problem *p, int precision, int *items_per_sm, int *variant) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_prepared.find(ws);
    if (it == g_prepared.end() || !same_problem(it->second.prob, *p) || it->second.precision != precision) return false;
    *items_per_sm = it->second.items_per_sm;
    *variant = it->second.tile_variant;
    return true;
}

bool is_prepared(const void *ws, const aexp_problem *p, int precision, int items_per_sm = 0, int variant = 0) {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_prepared.find(ws);
    return it != g_prepared.end() && same_problem(it->second.prob, *p) && it->second.precision == precision &&
           it->second.items_per_sm == effective_items(precision, items_per_sm) && it->second.tile_variant == variant;
}

// One captured cs_recon per workspace, relaunched while every argument is identical.
struct GraphEntry {
    std::vector<unsigned char> key;
    cudaGraphExec_t exec = nullptr;
};
std::unordered_map<const void *, GraphEntry> g_graphs;

template <class T>
void put(std::vector<unsigned char> &v, const T &x) {
    const unsigned char *b = reinterpret_cast<const unsigned char *>(&x);
    v.insert(v.end(), b, b + sizeof(T));
}

// Capture `issue` on st once per (workspace, key) and replay the instantiated graph on every
// later call with the same key.
template <class Issue>
cudaError_t launch_captured(const void *ws, const std::vector<unsigned char> &key, cudaStream_t st, Issue issue) {
    std::lock_guard<std::mutex> lk(g_mu);
    GraphEntry &ge = g_graphs[ws];
    if (ge.exec == nullptr || ge.key != key) {
        if (ge.exec) {
            cudaGraphExecDestroy(ge.exec);
            ge.exec = nullptr;
        }
        cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        cudaError_t ei = issue();
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(st, &g);
        if (ei != cudaSuccess || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return ei != cudaSuccess ? ei : e;
        }
        e = cudaGraphInstantiate(&ge.exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            ge.exec = nullptr;
            return e;
        }
        ge.key = key;
    }
    return cudaGraphLaunch(ge.exec, st);
}

int check_tiling(int items_per_sm, int tile_variant) {
    if (items_per_sm < 0 || items_per_sm > 256) return AEXP_ERR_INVALID_ARG;
    if (tile_variant < 0 || tile_variant >= kTileVariants) return AEXP_ERR_INVALID_ARG;
    return AEXP_OK;
}

int check_opts(const aexp_recon_opts *o) {
    if (!o) return AEXP_ERR_INVALID_ARG;
    int rc = check_precision(o->precision);
    if (rc) return rc;
    if (o->wavelet != AEXP_WAVELET_HAAR && o->wavelet != AEXP_WAVELET_DB4) return AEXP_ERR_INVALID_ARG;
    if (o->levels < 1 || o->levels > 12) return AEXP_ERR_INVALID_ARG;
    if (!(o->lipschitz > 0.0) && o->n_power < 1) return AEXP_ERR_INVALID_ARG;
    if ((rc = check_tiling(o->items_per_sm, o->tile_variant))) return rc;
    if (o->lambda_rule != AEXP_LAMBDA_GIVEN && o->lambda_rule != AEXP_LAMBDA_RAYLEIGH) return AEXP_ERR_INVALID_ARG;
    if (o->lambda_rule == AEXP_LAMBDA_RAYLEIGH && !o->undecimated) return AEXP_ERR_UNSUPPORTED;
    if (!aligned(o->x0, 8) || !aligned(o->power_init, 8) || !aligned(o->lambda_out, 8)) return AEXP_ERR_MISALIGNED;
    return AEXP_OK;
}

}  // namespace

void aexp::aexp_set_last_cuda_error(int e) { g_last_cuda_error = e; }

void aexp::forget_prepared(const void *ws) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_prepared.erase(ws);
}

extern "C" {

int aexp_version(void) { return 100; }

int aexp_last_cuda_error(void) { return g_last_cuda_error; }

const char *aexp_status_string(int status) {
    switch (status) {
        case AEXP_OK: return "ok";
        case AEXP_ERR_INVALID_ARG: return "invalid argument";
        case AEXP_ERR_MISALIGNED: return "misaligned pointer";
        case AEXP_ERR_UNSUPPORTED: return "unsupported size or option";
        case AEXP_ERR_WORKSPACE: return "workspace too small";
        case AEXP_ERR_CUDA: return "CUDA runtime error";
        case AEXP_ERR_DEVICE_TIMEOUT: return "bounded device wait timed out";
        case AEXP_ERR_NONFINITE: return "non-finite device scalar";
        case AEXP_ERR_NOT_PREPARED: return "workspace not prepared for this problem";
        default: return "unknown status";
    }
}

int aexp_workspace_size(const aexp_problem *prob, int precision, size_t *bytes) {
    int rc = check_problem(prob);
    if (rc) return rc;
    if ((rc = check_precision(precision))) return rc;
    if (!bytes) return AEXP_ERR_INVALID_ARG;
    OpLayout L;
    op_layout(prob, precision, &L);
    *bytes = L.bytes;
    return AEXP_OK;
}

int aexp_prepare(const aexp_problem *prob, int precision, void *ws, size_t ws_bytes, void *stream) {
    return aexp_prepare_tiled(prob, precision, 0, 0, ws, ws_bytes, stream);
}

int aexp_workspace_size_tiled(const aexp_problem *prob, int precision, int items_per_sm, int tile_variant,
                              size_t *bytes) {
    int rc = check_problem(prob);
    if (rc) return rc;
    if ((rc = check_precision(precision))) return rc;
    if ((rc = check_tiling(items_per_sm, tile_variant))) return rc;
    if (!bytes) return AEXP_ERR_INVALID_ARG;
    OpLayout L;
    op_layout(prob, precision, &L, items_target(precision, items_per_sm), tile_variant);
    *bytes = L.bytes;
    return AEXP_OK;
}

int aexp_prepare_tiled(const aexp_problem *prob, int precision, int items_per_sm, int tile_variant, void *ws,
                       size_t ws_bytes, void *stream) {
    int rc = check_problem(prob);
    if (rc) return rc;
    if ((rc = check_precision(precision))) return rc;
    if ((rc = check_tiling(items_per_sm, tile_variant))) return rc;
    OpLayout L;
    op_layout(prob, precision, &L, items_target(precision, items_per_sm), tile_variant);
    if ((rc = check_ws(ws, ws_bytes, L.bytes))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemsetAsync((char *)ws + L.off_hdr, 0, sizeof(WsHeader), st);
    if (e == cudaSuccess) e = op_prepare(prob, L, (char *)ws, st);
    if (e != cudaSuccess) return cuda_fail(e);
    record_prepared(ws, prob, precision, items_per_sm, tile_variant);
    return AEXP_OK;
}

int a_exp_forward(const aexp_problem *prob, int precision, const void *x, void *y, void *ws, size_t ws_bytes,
                  void *stream) {
    int rc = check_problem(prob);
    if (rc) return rc;
    if ((rc = check_precision(precision))) return rc;
    if (!x || !y) return AEXP_ERR_INVALID_ARG;
    if (!aligned(x, 8) || !aligned(y, 8)) return AEXP_ERR_MISALIGNED;
    int items = 0, variant = 0;
    const bool prepared = prepared_tiling(ws, prob, precision, &items, &variant);
    OpLayout L;
    op_layout(prob, precision, &L, items_target(precision, items), variant);
    if ((rc = check_ws(ws, ws_bytes, L.bytes))) return rc;
    if (!prepared) return AEXP_ERR_NOT_PREPARED;
    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)ws;
    cudaError_t e = op_apply_forward(L, (const float2 *)x, w, st);
    if (e == cudaSuccess) e = op_reduce_forward_public(L, w, (float2 *)y, st);
    return e == cudaSuccess ? AEXP_OK : cuda_fail(e);
}

int a_exp_adjoint(const aexp_problem *prob, int precision, const void *y, void *x, void *ws, size_t ws_bytes,
                  void *stream) {
    int rc = check_problem(prob);
    if (rc) return rc;
    if ((rc = check_precision(precision))) return rc;
    if (!x || !y) return AEXP_ERR_INVALID_ARG;
    if (!aligned(x, 8) || !aligned(y, 8)) return AEXP_ERR_MISALIGNED;
    int items = 0, variant = 0;
    const bool prepared = prepared_tiling(ws, prob, precision, &items, &variant);
    OpLayout L;
    op_layout(prob, precision, &L, items_target(precision, items), variant);
    if ((rc = check_ws(ws, ws_bytes, L.bytes))) return rc;
    if (!prepared) return AEXP_ERR_NOT_PREPARED;
    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)ws;
    float2 *yt = (float2 *)(w + L.off_yt);
    cudaError_t e = op_transpose_y(L, (const float2 *)y, yt, st);
    if (e == cudaSuccess) e = op_apply_adjoint(L, yt, w, st);
    if (e == cudaSuccess) e = op_adjoint_reduce(L, w, (float2 *)x, st);
    return e == cudaSuccess ? AEXP_OK : cuda_fail(e);
}

void aexp_recon_opts_default(aexp_recon_opts *o) {
    if (!o) return;
    memset(o, 0, sizeof(*o));
    o->precision = AEXP_FP32;
    o->wavelet = AEXP_WAVELET_HAAR;
    o->levels = 3;
    o->n_power = 30;
    o->lipschitz = 0.0;
    o->x0 = nullptr;
    o->power_init = nullptr;
    o->use_graph = 1;
    o->undecimated = 0;
    o->lambda_rule = AEXP_LAMBDA_GIVEN;
    o->lambda_out = nullptr;
    o->items_per_sm = 0;
    o->tile_variant = 0;
}

int aexp_recon_workspace_size(const aexp_problem *prob, const aexp_recon_opts *opts, size_t *bytes) {
    int rc = check_problem(prob);
    if (rc) return rc;
    if ((rc = check_opts(opts))) return rc;
    if (!bytes) return AEXP_ERR_INVALID_ARG;
    RecLayout R;
    rec_layout(prob, opts, &R);
    *bytes = R.bytes;
    return AEXP_OK;
}

int cs_recon(const aexp_problem *prob, const void *y, float lambda, int iters, const aexp_recon_opts *opts,
             void *x_out, double *lipschitz_out, void *ws, size_t ws_bytes, void *stream) {
    int rc = check_problem(prob);
    if (rc) return rc;
    if ((rc = check_opts(opts))) return rc;
    if (!y || !x_out || iters < 0 || !(lambda >= 0.f)) return AEXP_ERR_INVALID_ARG;
    if (!aligned(y, 8) || !aligned(x_out, 8) || !aligned(lipschitz_out, 8)) return AEXP_ERR_MISALIGNED;
    RecLayout R;
    rec_layout(prob, opts, &R);
    if ((rc = check_ws(ws, ws_bytes, R.bytes))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)ws;

    cudaError_t e = cudaMemsetAsync(w + R.op.off_hdr, 0, sizeof(WsHeader), st);
    if (e != cudaSuccess) return cuda_fail(e);
    if (!opts->use_graph || st == nullptr) {
        e = recon_issue(prob, R, opts, (const float2 *)y, lambda, iters, (float2 *)x_out,
                        lipschitz_out, w, st);
        if (e != cudaSuccess) return cuda_fail(e);
        record_prepared(ws, prob, opts->precision, opts->items_per_sm, opts->tile_variant);
        return AEXP_OK;
    }

    std::vector<unsigned char> key;
    put(key, *prob);
    put(key, *opts);
    put(key, y);
    put(key, lambda);
    put(key, iters);
    put(key, x_out);
    put(key, lipschitz_out);
    put(key, ws_bytes);
    std::lock_guard<std::mutex> lk(g_mu);
    GraphEntry &ge = g_graphs[ws];
    if (ge.exec == nullptr || ge.key != key) {
        if (ge.exec) {
            cudaGraphExecDestroy(ge.exec);
            ge.exec = nullptr;
        }
        e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e);
        cudaError_t ei = recon_issue(prob, R, opts, (const float2 *)y, lambda, iters, (float2 *)x_out,
                                     lipschitz_out, w, st);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(st, &g);
        if (ei != cudaSuccess || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_fail(ei != cudaSuccess ? ei : e);
        }
        e = cudaGraphInstantiate(&ge.exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            ge.exec = nullptr;
            return cuda_fail(e);
        }
        ge.key = key;
    }
    e = cudaGraphLaunch(ge.exec, st);
    if (e != cudaSuccess) return cuda_fail(e);
    g_prepared[ws] = PrepRecord{*prob, opts->precision, effective_items(opts->precision, opts->items_per_sm),
                                opts->tile_variant};
    return AEXP_OK;
}

int aexp_cgls_workspace_size(const aexp_problem *prob, const aexp_recon_opts *opts, size_t *bytes) {
    int rc = check_problem(prob);
    if (rc) return rc;
    if ((rc = check_opts(opts))) return rc;
    if (!bytes) return AEXP_ERR_INVALID_ARG;
    CglsLayout C;
    if ((rc = cgls_layout(prob, opts, &C))) return rc;
    *bytes = C.bytes;
    return AEXP_OK;
}

int cgls_recon(const aexp_problem *prob, const void *y, int iters, const aexp_recon_opts *opts, void *x_out,
               void *ws, size_t ws_bytes, void *stream) {
    int rc = check_problem(prob);
    if (rc) return rc;
    if ((rc = check_opts(opts))) return rc;
    if (!y || !x_out || iters < 0) return AEXP_ERR_INVALID_ARG;
    if (!aligned(y, 8) || !aligned(x_out, 8)) return AEXP_ERR_MISALIGNED;
    CglsLayout C;
    if ((rc = cgls_layout(prob, opts, &C))) return rc;
    if ((rc = check_ws(ws, ws_bytes, C.bytes))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)ws;
    cudaError_t e = cudaMemsetAsync(w + C.op.off_hdr, 0, sizeof(WsHeader), st);
    if (e != cudaSuccess) return cuda_fail(e);
    auto issue = [&]() { return cgls_issue(prob, C, (const float2 *)y, iters, (float2 *)x_out, w, st); };
    if (!opts->use_graph || st == nullptr) {
        e = issue();
    } else {
        std::vector<unsigned char> key;
        put(key, 'L');  // distinguishes this solver's graphs from cs_recon's on the same workspace
        put(key, *prob);
        put(key, *opts);
        put(key, y);
        put(key, iters);
        put(key, x_out);
        put(key, ws_bytes);
        e = launch_captured(ws, key, st, issue);
    }
    if (e != cudaSuccess) return cuda_fail(e);
    record_prepared(ws, prob, opts->precision, opts->items_per_sm, opts->tile_variant);
    return AEXP_OK;
}

int aexp_batch_workspace_size(const aexp_problem *probs, int nprob, const aexp_recon_opts *opts, size_t *bytes) {
    if (!probs || nprob < 1 || nprob > kMaxBatchProblems || !bytes) return AEXP_ERR_INVALID_ARG;
    int rc = check_opts(opts);
    if (rc) return rc;
    if (opts->precision == AEXP_FP32 || opts->undecimated) return AEXP_ERR_UNSUPPORTED;
    for (int q = 0; q < nprob; ++q)
        if ((rc = check_problem(&probs[q]))) return rc;
    BatchLayout B;
    if ((rc = batch_layout(probs, nprob, opts, &B))) return rc;
    *bytes = B.bytes;
    return AEXP_OK;
}

int cs_recon_batched(const aexp_problem *probs, int nprob, const void *const *y, const float *lambda, int iters,
                     const aexp_recon_opts *opts, void *const *x_out, double *lipschitz_out, void *ws,
                     size_t ws_bytes, void *stream) {
    if (!probs || nprob < 1 || nprob > kMaxBatchProblems || !y || !lambda || !x_out || iters < 0)
        return AEXP_ERR_INVALID_ARG;
    int rc = check_opts(opts);
    if (rc) return rc;
    if (opts->precision == AEXP_FP32 || opts->undecimated) return AEXP_ERR_UNSUPPORTED;
    if (opts->x0 || opts->power_init) return AEXP_ERR_UNSUPPORTED;
    if (!aligned(lipschitz_out, 8)) return AEXP_ERR_MISALIGNED;
    for (int q = 0; q < nprob; ++q) {
        if ((rc = check_problem(&probs[q]))) return rc;
        if (!y[q] || !x_out[q] || !(lambda[q] >= 0.f)) return AEXP_ERR_INVALID_ARG;
        if (!aligned(y[q], 8) || !aligned(x_out[q], 8)) return AEXP_ERR_MISALIGNED;
    }
    BatchLayout B;
    if ((rc = batch_layout(probs, nprob, opts, &B))) return rc;
    if ((rc = check_ws(ws, ws_bytes, B.bytes))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)ws;
    cudaError_t e = cudaMemsetAsync(w + B.off_hdr, 0, sizeof(WsHeader), st);
    if (e != cudaSuccess) return cuda_fail(e);
    if (!opts->use_graph || st == nullptr) {
        e = batch_recon_issue(probs, B, opts, y, lambda, iters, x_out, lipschitz_out, w, st);
        return e == cudaSuccess ? AEXP_OK : cuda_fail(e);
    }
    std::vector<unsigned char> key;
    for (int q = 0; q < nprob; ++q) {
        put(key, probs[q]);
        put(key, y[q]);
        put(key, lambda[q]);
        put(key, x_out[q]);
    }
    put(key, *opts);
    put(key, iters);
    put(key, lipschitz_out);
    put(key, ws_bytes);
    std::lock_guard<std::mutex> lk(g_mu);
    GraphEntry &ge = g_graphs[ws];
    if (ge.exec == nullptr || ge.key != key) {
        if (ge.exec) {
            cudaGraphExecDestroy(ge.exec);
            ge.exec = nullptr;
        }
        e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(e);
        cudaError_t ei = batch_recon_issue(probs, B, opts, y, lambda, iters, x_out, lipschitz_out, w, st);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(st, &g);
        if (ei != cudaSuccess || e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_fail(ei != cudaSuccess ? ei : e);
        }
        e = cudaGraphInstantiate(&ge.exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            ge.exec = nullptr;
            return cuda_fail(e);
        }
        ge.key = key;
    }
    e = cudaGraphLaunch(ge.exec, st);
    return e == cudaSuccess ? AEXP_OK : cuda_fail(e);
}

int aexp_power_lipschitz(const aexp_problem *prob, int precision, const void *v0, int n_power,
                         double *lipschitz_out, void *ws, size_t ws_bytes, void *stream) {
    int rc = check_problem(prob);
    if (rc) return rc;
    if ((rc = check_precision(precision))) return rc;
    if (!v0 || !lipschitz_out || n_power < 1) return AEXP_ERR_INVALID_ARG;
    if (!aligned(v0, 8) || !aligned(lipschitz_out, 8)) return AEXP_ERR_MISALIGNED;
    aexp_recon_opts o;
    aexp_recon_opts_default(&o);
    o.precision = precision;
    o.levels = 1;
    RecLayout R;
    rec_layout(prob, &o, &R);
    if ((rc = check_ws(ws, ws_bytes, R.off_wave))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)ws;
    cudaError_t e = cudaMemsetAsync(w + R.op.off_hdr, 0, sizeof(WsHeader), st);
    if (e == cudaSuccess) e = op_prepare(prob, R.op, w, st);
    if (e == cudaSuccess)
        e = power_iteration(R.op, w, (const float2 *)v0, (float2 *)(w + R.off_v), (float2 *)(w + R.off_w), n_power,
                            lipschitz_out, st);
    if (e != cudaSuccess) return cuda_fail(e);
    record_prepared(ws, prob, precision);
    return AEXP_OK;
}

int aexp_unroll_workspace_size(const aexp_problem *prob, const aexp_recon_opts *opts, size_t *bytes) {
    int rc = check_problem(prob);
    if (rc) return rc;
    if ((rc = check_opts(opts))) return rc;
    if (!bytes) return AEXP_ERR_INVALID_ARG;
    RecLayout R;
    rec_layout(prob, opts, &R, -1, 1);
    *bytes = R.bytes;
    return AEXP_OK;
}

static int unroll_common(const aexp_problem *prob, const aexp_recon_opts *opts, const void *y, double lipschitz,
                         void *ws, size_t ws_bytes, RecLayout *R) {
    int rc = check_problem(prob);
    if (rc) return rc;
    if ((rc = check_opts(opts))) return rc;
    if (opts->undecimated) return AEXP_ERR_UNSUPPORTED;  // the unrolled step uses the orthogonal W
    if (!y || !(lipschitz > 0.0)) return AEXP_ERR_INVALID_ARG;
    if (!aligned(y, 8)) return AEXP_ERR_MISALIGNED;
    rec_layout(prob, opts, R, -1, 1);
    if ((rc = check_ws(ws, ws_bytes, R->bytes))) return rc;
    if (!is_prepared(ws, prob, opts->precision, opts->items_per_sm, opts->tile_variant)) return AEXP_ERR_NOT_PREPARED;
    return AEXP_OK;
}

int aexp_fista_step(const aexp_problem *prob, const aexp_recon_opts *opts, const void *y, float lambda,
                    double lipschitz, const void *z, const void *x_prev, double beta, void *x_out, void *z_out,
                    void *ws, size_t ws_bytes, void *stream) {
    RecLayout R;
    int rc = unroll_common(prob, opts, y, lipschitz, ws, ws_bytes, &R);
    if (rc) return rc;
    if (!z || !x_prev || !x_out || !z_out || !(lambda >= 0.f)) return AEXP_ERR_INVALID_ARG;
    if (!aligned(z, 8) || !aligned(x_prev, 8) || !aligned(x_out, 8) || !aligned(z_out, 8)) return AEXP_ERR_MISALIGNED;
    cudaError_t e = unroll_step(R, (const float2 *)y, lambda, lipschitz, (const float2 *)z, (const float2 *)x_prev,
                                beta, (float2 *)x_out, (float2 *)z_out, (char *)ws, (cudaStream_t)stream);
    return e == cudaSuccess ? AEXP_OK : cuda_fail(e);
}

int aexp_fista_step_vjp(const aexp_problem *prob, const aexp_recon_opts *opts, const void *y, float lambda,
                        double lipschitz, const void *z, double beta, double beta_next, const void *xbar_in,
                        const void *zbar_next, const void *zbar_next2, void *zbar_out, float *kbar, double *lambar,
                        void *ws, size_t ws_bytes, void *stream) {
    RecLayout R;
    int rc = unroll_common(prob, opts, y, lipschitz, ws, ws_bytes, &R);
    if (rc) return rc;
    if (!z || !zbar_out || !(lambda >= 0.f)) return AEXP_ERR_INVALID_ARG;
    if (!aligned(z, 8) || !aligned(xbar_in, 8) || !aligned(zbar_next, 8) || !aligned(zbar_next2, 8) ||
        !aligned(zbar_out, 8) || !aligned(kbar, 4) || !aligned(lambar, 8))
        return AEXP_ERR_MISALIGNED;
    cudaError_t e = unroll_step_vjp(R, (const float2 *)y, lambda, lipschitz, (const float2 *)z, beta, beta_next,
                                    (const float2 *)xbar_in, (const float2 *)zbar_next, (const float2 *)zbar_next2,
                                    (float2 *)zbar_out, kbar, lambar, (char *)ws, (cudaStream_t)stream);
    return e == cudaSuccess ? AEXP_OK : cuda_fail(e);
}

int aexp_coil_compress_workspace_size(int nc, size_t *bytes) {
    if (nc < 1 || nc > kMaxCoils || !bytes) return AEXP_ERR_INVALID_ARG;
    *bytes = coil_compress_bytes(nc);
    return AEXP_OK;
}

int aexp_coil_compress_sweeps(const aexp_problem *prob, const void *y, int nv, int max_sweeps, void *y_out,
                              void *S_out, double *eig_out, void *ws, size_t ws_bytes, void *stream) {
    int rc = check_problem(prob);
    if (rc) return rc;
    if (!y || !y_out || !S_out || nv < 1 || nv > prob->nc) return AEXP_ERR_INVALID_ARG;
    if (max_sweeps < 1 || max_sweeps > kJacobiMaxSweeps) return AEXP_ERR_INVALID_ARG;
    if (!aligned(y, 8) || !aligned(y_out, 8) || !aligned(S_out, 8) || !aligned(eig_out, 8)) return AEXP_ERR_MISALIGNED;
    if ((rc = check_ws(ws, ws_bytes, coil_compress_bytes(prob->nc)))) return rc;
    cudaError_t e = coil_compress((const float2 *)y, (const float2 *)prob->S, prob->nc, prob->nt, prob->nx * prob->ny,
                                  nv, (float2 *)y_out, (float2 *)S_out, eig_out, (char *)ws, (cudaStream_t)stream,
                                  max_sweeps);
    return e == cudaSuccess ? AEXP_OK : cuda_fail(e);
}

int aexp_coil_compress(const aexp_problem *prob, const void *y, int nv, void *y_out, void *S_out, double *eig_out,
                       void *ws, size_t ws_bytes, void *stream) {
    return aexp_coil_compress_sweeps(prob, y, nv, kJacobiMaxSweeps, y_out, S_out, eig_out, ws, ws_bytes, stream);
}

int aexp_probe_bounded_wait(int polls, int *result, void *ws, size_t ws_bytes, void *stream) {
    if (polls < 1 || polls > kWaitPolls || !result) return AEXP_ERR_INVALID_ARG;
    if (!aligned(result, 4)) return AEXP_ERR_MISALIGNED;
    int rc = check_ws(ws, ws_bytes, sizeof(WsHeader));
    if (rc) return rc;
    cudaError_t e = bounded_wait_probe(polls, &((WsHeader *)ws)->status, result, (cudaStream_t)stream);
    return e == cudaSuccess ? AEXP_OK : cuda_fail(e);
}

size_t aexp_header_bytes(void) { return sizeof(WsHeader); }

int aexp_coil_compress_status(const void *ws, int nc, void *stream, int *status) {
    if (!ws || !status || nc < 1 || nc > kMaxCoils) return AEXP_ERR_INVALID_ARG;
    const char *p = (const char *)ws + coil_compress_bytes(nc) - align_up(sizeof(int));
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(status, p, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e == cudaSuccess ? AEXP_OK : cuda_fail(e);
}

int aexp_swt_workspace_size(int nx, int ny, size_t *bytes) {
    if (nx < 1 || ny < 1 || !bytes) return AEXP_ERR_INVALID_ARG;
    if ((long long)nx * ny > (1LL << 26)) return AEXP_ERR_UNSUPPORTED;
    *bytes = align_up(4 * sizeof(float2) * (size_t)nx * ny) + swt_aux_bytes();
    return AEXP_OK;
}

int aexp_swt_forward(int nx, int ny, int wavelet, const void *in, void *coef, void *stream) {
    if (nx < 1 || ny < 1 || !in || !coef) return AEXP_ERR_INVALID_ARG;
    if (wavelet != AEXP_WAVELET_HAAR && wavelet != AEXP_WAVELET_DB4) return AEXP_ERR_INVALID_ARG;
    if ((long long)nx * ny > (1LL << 26)) return AEXP_ERR_UNSUPPORTED;
    if (!aligned(in, 8) || !aligned(coef, 8)) return AEXP_ERR_MISALIGNED;
    cudaError_t e = swt_analysis(wavelet, (const float2 *)in, (float2 *)coef, nx, ny, -1.f, nullptr, nullptr,
                                 (cudaStream_t)stream);
    return e == cudaSuccess ? AEXP_OK : cuda_fail(e);
}

int aexp_swt_prox(int nx, int ny, int wavelet, float tau, const void *in, void *out, void *ws, size_t ws_bytes,
                  void *stream) {
    size_t need;
    int rc = aexp_swt_workspace_size(nx, ny, &need);
    if (rc) return rc;
    if (!in || !out || !(tau >= 0.f)) return AEXP_ERR_INVALID_ARG;
    if (wavelet != AEXP_WAVELET_HAAR && wavelet != AEXP_WAVELET_DB4) return AEXP_ERR_INVALID_ARG;
    if (!aligned(in, 8) || !aligned(out, 8)) return AEXP_ERR_MISALIGNED;
    if ((rc = check_ws(ws, ws_bytes, need))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    float2 *c = (float2 *)ws;
    cudaError_t e = swt_analysis(wavelet, (const float2 *)in, c, nx, ny, tau, nullptr, nullptr, st);
    if (e == cudaSuccess) e = swt_synthesis(wavelet, c, (float2 *)out, nx, ny, 0, 0.0, nullptr, nullptr, st);
    return e == cudaSuccess ? AEXP_OK : cuda_fail(e);
}

int aexp_swt_lambda(int nx, int ny, int wavelet, const void *img, double *lambda_out, void *ws, size_t ws_bytes,
                    void *stream) {
    size_t need;
    int rc = aexp_swt_workspace_size(nx, ny, &need);
    if (rc) return rc;
    if (!img || !lambda_out) return AEXP_ERR_INVALID_ARG;
    if (wavelet != AEXP_WAVELET_HAAR && wavelet != AEXP_WAVELET_DB4) return AEXP_ERR_INVALID_ARG;
    if (!aligned(img, 8) || !aligned(lambda_out, 8)) return AEXP_ERR_MISALIGNED;
    if ((rc = check_ws(ws, ws_bytes, need))) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    char *w = (char *)ws;
    float2 *c = (float2 *)w;
    char *aux = w + align_up(4 * sizeof(float2) * (size_t)nx * ny);
    cudaError_t e = swt_analysis(wavelet, (const float2 *)img, c, nx, ny, -1.f, nullptr, nullptr, st);
    if (e == cudaSuccess) e = swt_rayleigh_lambda(c, nx, ny, aux, lambda_out, st);
    return e == cudaSuccess ? AEXP_OK : cuda_fail(e);
}

int aexp_wavelet_workspace_size(int nx, int ny, int wavelet, int levels, size_t *bytes) {
    if (nx < 1 || ny < 1 || levels < 1 || levels > 12 || !bytes) return AEXP_ERR_INVALID_ARG;
    if (wavelet != AEXP_WAVELET_HAAR && wavelet != AEXP_WAVELET_DB4) return AEXP_ERR_INVALID_ARG;
    WaveLayout W;
    wave_layout(nx, ny, wavelet, levels, &W);
    *bytes = W.bytes;
    return AEXP_OK;
}

int aexp_wavelet_prox(int nx, int ny, int wavelet, int levels, float tau, const void *in, void *out, void *ws,
                      size_t ws_bytes, void *stream) {
    size_t need;
    int rc = aexp_wavelet_workspace_size(nx, ny, wavelet, levels, &need);
    if (rc) return rc;
    if (!in || !out || !(tau >= 0.f)) return AEXP_ERR_INVALID_ARG;
    if (!aligned(in, 8) || !aligned(out, 8)) return AEXP_ERR_MISALIGNED;
    if ((rc = check_ws(ws, ws_bytes, need))) return rc;
    WaveLayout W;
    wave_layout(nx, ny, wavelet, levels, &W);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = wave_prox(W, (const float2 *)in, (char *)ws, tau, nullptr, (float2 *)out, 0, 0.0, nullptr, nullptr, st);
    return e == cudaSuccess ? AEXP_OK : cuda_fail(e);
}

int aexp_wavelet_forward(int nx, int ny, int wavelet, int levels, const void *in, void *coef, void *ws,
                         size_t ws_bytes, void *stream) {
    size_t need;
    int rc = aexp_wavelet_workspace_size(nx, ny, wavelet, levels, &need);
    if (rc) return rc;
    if (!in || !coef) return AEXP_ERR_INVALID_ARG;
    if (!aligned(in, 8) || !aligned(coef, 8)) return AEXP_ERR_MISALIGNED;
    if ((rc = check_ws(ws, ws_bytes, need))) return rc;
    WaveLayout W;
    wave_layout(nx, ny, wavelet, levels, &W);
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = wave_forward(W, (const float2 *)in, (char *)ws, 0.f, nullptr, 0, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(coef, (char *)ws + W.off_pyr, sizeof(float2) * (size_t)W.npx * W.npy,
                            cudaMemcpyDeviceToDevice, st);
    return e == cudaSuccess ? AEXP_OK : cuda_fail(e);
}

int aexp_read_status(void *ws, void *stream, int *status) {
    if (!ws || !status) return AEXP_ERR_INVALID_ARG;
    if (!aligned(ws, kAlign)) return AEXP_ERR_MISALIGNED;
    cudaStream_t st = (cudaStream_t)stream;
    int s = 0;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaMemcpy(&s, ws, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(ws, 0, sizeof(int));
    if (e != cudaSuccess) return cuda_fail(e);
    *status = s;
    return AEXP_OK;
}

}  // extern "C"
