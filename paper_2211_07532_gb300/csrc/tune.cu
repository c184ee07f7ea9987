// Autotuning of the work-item granularity of the operator launches.
//
// The split of the sample (forward) and voxel (adjoint) reductions trades load balance
// (more, smaller blocks or persistent work items) against partial-sum traffic and the
// per-item pipeline start-up.  The best point depends on the problem sizes, the batch
// size and the precision, so it is measured: each candidate granularity lays out the
// caller's workspace, prepares the problem(s) and times one A^H A application with CUDA
// events on the caller's stream (one warm-up, best of three).
#include <algorithm>
#include <vector>

#include "aexp_internal.cuh"
#include "batch_internal.h"

namespace aexp {
namespace {

constexpr int kCandidates[] = {2, 4, 8, 16, 32};
constexpr int kReps = 3;

#define TK(x)                                      \
    do {                                           \
        cudaError_t e__ = (x);                     \
        if (e__ != cudaSuccess) {                  \
            aexp_set_last_cuda_error((int)e__);    \
            return AEXP_ERR_CUDA;                  \
        }                                          \
    } while (0)

int layout_bytes(const aexp_problem *probs, int nprob, const aexp_recon_opts *o, size_t *bytes) {
    if (nprob == 1) {
        RecLayout R;
        int rc = rec_layout(probs, o, &R);
        *bytes = R.bytes;
        return rc;
    }
    BatchLayout B;
    int rc = batch_layout(probs, nprob, o, &B);
    *bytes = B.bytes;
    return rc;
}

// Issue one timed unit (A^H A on a zero image) for the layout of `o`; the preparation is
// issued by `setup`.
struct Unit {
    const aexp_problem *probs;
    int nprob;
    aexp_recon_opts o;
    RecLayout R;
    BatchLayout B;
    char *ws;

    int layout() { return nprob == 1 ? rec_layout(probs, &o, &R) : batch_layout(probs, nprob, &o, &B); }

    cudaError_t setup(cudaStream_t st) {
        if (nprob == 1) {
            cudaError_t e = cudaMemsetAsync(ws + R.op.off_hdr, 0, sizeof(WsHeader), st);
            if (e == cudaSuccess) e = op_prepare(probs, R.op, ws, st);
            if (e == cudaSuccess) e = cudaMemsetAsync(ws + R.off_v, 0, sizeof(float2) * (size_t)R.op.nr, st);
            return e;
        }
        cudaError_t e = cudaMemsetAsync(ws + B.off_hdr, 0, sizeof(WsHeader), st);
        return e == cudaSuccess ? batch_setup(probs, B, nullptr, nullptr, nullptr, nullptr, ws, st) : e;
    }

    cudaError_t run(cudaStream_t st) {
        if (nprob == 1)
            return normal_apply(R.op, ws, (const float2 *)(ws + R.off_v), (float2 *)(ws + R.off_w), st);
        return batch_normal_once(B, &o, ws, st);
    }
};

}  // namespace
}  // namespace aexp

using namespace aexp;

extern "C" {

int aexp_autotune_workspace_size(const aexp_problem *probs, int nprob, const aexp_recon_opts *opts, size_t *bytes) {
    if (!probs || nprob < 1 || nprob > kMaxBatchProblems || !opts || !bytes) return AEXP_ERR_INVALID_ARG;
    size_t one = 0, need = 0;
    int rc = nprob == 1 ? aexp_recon_workspace_size(probs, opts, &one) : aexp_batch_workspace_size(probs, nprob, opts, &one);
    if (rc) return rc;  // validates the problems and options
    for (int c : kCandidates) {
        aexp_recon_opts o = *opts;
        o.items_per_sm = c;
        if ((rc = layout_bytes(probs, nprob, &o, &one))) return rc;
        need = std::max(need, one);
    }
    *bytes = need;
    return AEXP_OK;
}

int aexp_autotune(const aexp_problem *probs, int nprob, const aexp_recon_opts *opts, void *ws, size_t ws_bytes,
                  void *stream, int *best_items_per_sm, float *best_ms) {
    size_t need = 0;
    int rc = aexp_autotune_workspace_size(probs, nprob, opts, &need);
    if (rc) return rc;
    if (!best_items_per_sm) return AEXP_ERR_INVALID_ARG;
    if (!ws) return AEXP_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(ws) % kAlign) return AEXP_ERR_MISALIGNED;
    if (ws_bytes < need) return AEXP_ERR_WORKSPACE;
    cudaStream_t st = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    TK(cudaStreamIsCapturing(st, &cap));
    if (cap != cudaStreamCaptureStatusNone) return AEXP_ERR_INVALID_ARG;  // timing needs real execution
    forget_prepared(ws);

    cudaEvent_t ev[2];
    TK(cudaEventCreate(&ev[0]));
    if (cudaEventCreate(&ev[1]) != cudaSuccess) {
        cudaEventDestroy(ev[0]);
        return AEXP_ERR_CUDA;
    }
    int best = 0, status = 0;
    float best_t = 0.f;
    cudaError_t e = cudaSuccess;
    for (int c : kCandidates) {
        Unit u{probs, nprob, *opts, {}, {}, (char *)ws};
        u.o.items_per_sm = c;
        if ((rc = u.layout())) break;
        e = u.setup(st);
        if (e == cudaSuccess) e = u.run(st);  // warm-up
        float t_min = 0.f;
        for (int r = 0; r < kReps && e == cudaSuccess; ++r) {
            e = cudaEventRecord(ev[0], st);
            if (e == cudaSuccess) e = u.run(st);
            if (e == cudaSuccess) e = cudaEventRecord(ev[1], st);
            if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
            float t = 0.f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&t, ev[0], ev[1]);
            if (r == 0 || t < t_min) t_min = t;
        }
        if (e != cudaSuccess) break;
        // a device-side error (bounded wait) disqualifies the whole call
        const char *hdr = (const char *)ws + (nprob == 1 ? u.R.op.off_hdr : u.B.off_hdr);
        if (nprob > 1) {
            // the batch header collects nothing here; read every problem's status word
            for (int q = 0; q < nprob && status == 0 && e == cudaSuccess; ++q)
                e = cudaMemcpy(&status, (const char *)ws + u.B.base[q] + u.B.R[q].op.off_hdr, sizeof(int),
                               cudaMemcpyDeviceToHost);
        } else {
            e = cudaMemcpy(&status, hdr, sizeof(int), cudaMemcpyDeviceToHost);
        }
        if (e != cudaSuccess || status != 0) break;
        if (best == 0 || t_min < best_t) {
            best = c;
            best_t = t_min;
        }
    }
    cudaEventDestroy(ev[0]);
    cudaEventDestroy(ev[1]);
    if (rc) return rc;
    if (e != cudaSuccess) {
        aexp_set_last_cuda_error((int)e);
        return AEXP_ERR_CUDA;
    }
    if (status != 0) return status;
    *best_items_per_sm = best;
    if (best_ms) *best_ms = best_t;
    return AEXP_OK;
}

}  // extern "C"
