// Host-side layout of a ragged-batch workspace (batch.cu, capi.cu).
#pragma once

#include <vector>

#include "aexp_internal.cuh"

namespace aexp {

constexpr int kMaxBatchProblems = 4095;

struct BatchLayout {
    int nprob = 0;
    int CB = 0, LP = 0;
    std::vector<RecLayout> R;      // one reconstruction workspace per problem
    std::vector<size_t> base;      // its byte offset inside the batch workspace
    std::vector<int> items_fwd;    // prefix offsets of the persistent kernels' work items
    std::vector<int> items_adj;
    size_t off_hdr = 0, off_desc = 0, off_items_fwd = 0, off_items_adj = 0;
    int max_nr = 0, max_ntpcb = 0, max_fwd_pack = 0, max_adj_pack = 0, max_npx = 0, max_npy = 0;
    size_t bytes = 0;
};

int batch_layout(const aexp_problem *probs, int nprob, const aexp_recon_opts *opts, BatchLayout *B);
// Per-problem preparation, descriptors, item offsets and header reset (y, lambda, x_out
// and lip_out may be null when only operator applications follow).
cudaError_t batch_setup(const aexp_problem *probs, const BatchLayout &B, const void *const *y, const float *lambda,
                        void *const *x_out, double *lip_out, char *ws, cudaStream_t st);
cudaError_t batch_normal_once(const BatchLayout &B, const aexp_recon_opts *o, char *ws, cudaStream_t st);
cudaError_t batch_recon_issue(const aexp_problem *probs, const BatchLayout &B, const aexp_recon_opts *o,
                              const void *const *y, const float *lambda, int iters, void *const *x_out,
                              double *lip_out, char *ws, cudaStream_t st);

}  // namespace aexp
