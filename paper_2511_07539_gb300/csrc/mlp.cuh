// The population surrogate's network state in a context (mlp.cu: init,
// weights, prediction, the training loop; mlp_train.cu: the fused training
// kernel).
#pragma once
#include <cuda_bf16.h>

#include <vector>

#include "xt_internal.cuh"

struct xt_mlp {
  std::vector<int> sizes;             // n_in, h, ..., n_out
  int64_t nparam = 0;
  std::vector<int64_t> woff, boff;    // offsets of W_k [s_(k-1)][s_k] and b_k in the flat vector
  float* w = nullptr;                 // FP32 master
  float* m = nullptr;                 // Adam moments
  float* v = nullptr;
  float* g = nullptr;                 // gradients (flat, like w)
  __nv_bfloat16* wb = nullptr;        // BF16 copy, flat (prediction)
  // BF16 copies in the tensor cores' operand rows, padded to 16 elements:
  // wp_k [s_(k-1)][P(s_k)] (row i = the weights out of input i) and
  // wt_k [s_k][P(s_(k-1))] (row o = the weights into output o)
  __nv_bfloat16* wp = nullptr;
  __nv_bfloat16* wt = nullptr;
  std::vector<int64_t> wpo, wto;      // offsets of wp_k, wt_k
  // prediction buffers (batch capacity cap)
  int64_t cap = 0;
  std::vector<float*> Z;              // [B][s_k] pre-activations (k = 1..L)
  std::vector<__nv_bfloat16*> H;      // [B][s_k] bf16 activations (H[0] = input)
  float* X = nullptr;                 // [B][s_0] input (host copy)
  // training buffers (batch capacity tcap), rows padded to P(s)
  int64_t tcap = 0;
  std::vector<__nv_bfloat16*> hp;     // [B][P(s_k)] activations, k = 0..L-1
  std::vector<float*> zp;             // [B][P(s_k)] pre-activations, k = 1..L-1 (index k)
  __nv_bfloat16* dz[2] = {nullptr, nullptr};   // [B][P(max s)] output gradients, alternating
  // the same transposed, rows of P(B): hT_k [s_k + 1][P(B)] (the last row all
  // ones over the batch, for the bias gradients), dzT [max s][P(B)]
  std::vector<__nv_bfloat16*> hT;
  __nv_bfloat16* dzT[2] = {nullptr, nullptr};
  float* T = nullptr;                 // [B][s_L] targets and mask of the batch
  float* M = nullptr;
  double* loss = nullptr;             // one step's loss and mask sum (surrogate_train_step)
  double* msum1 = nullptr;
  int64_t* st = nullptr;              // Adam steps taken
  unsigned* bar = nullptr;            // grid barrier: arrivals, generation; error flag
};

namespace xt {

__host__ __device__ inline int pad16(int s) { return (s + 15) & ~15; }

// Rows X/T/M of a batch and where they come from (idx = nullptr: rows 0..B-1
// of X, with T and M already the batch's).
struct TrainSrc {
  const float* X; const float* T; const float* M; const int* idx;
};

// Fused training: steps t = 0..nsteps-1 of one launch, step t on batch rows
// idx[t B .. t B + B); mask sums to msumv[t], losses to lossv[t] (zeroed by
// the caller); Adam after each step with a non-empty mask when update.
int mlp_train_run(xt_ctx* c, xt_mlp* n, int64_t B, const TrainSrc& src, int64_t nsteps, double* msumv,
                  double* lossv, double lr, bool update);
// (Re)allocate the training buffers for batch B.
int mlp_train_buffers(xt_ctx* c, xt_mlp* n, int64_t B);
// Offsets and buffers of the operand-layout copies wp, wt (after sizes,
// woff, boff are set); XT_EINVAL for more layers than the fused kernel takes.
int mlp_layout_copies(xt_ctx* c, xt_mlp* n);
// Refresh every BF16 copy (wb, wp, wt) from the FP32 master weights.
void mlp_sync_copies(xt_ctx* c, xt_mlp* n);

}  // namespace xt
