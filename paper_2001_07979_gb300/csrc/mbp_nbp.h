// Internal declarations of the unrolled normalised BP (mbp_nbp_forward and
// mbp_nbp_backward; kernels in mbp_nbp.cu).
#pragma once

#include "mbp_multi.h"

namespace mbp {

// Workspace of one unrolled decode of F frames over T iterations, after the
// single-decode state (channel LLRs, syndrome words): every iteration's
// messages and posteriors (the checkpoints the backward pass reads), the edge
// adjoint, the posterior adjoints and the per-block partial sums of the
// parameter gradients.
struct NbpState {
  int32_t F, T, n_tiles;
  float* lp;          // [n_tiles][n][kLanes] L_P (internal unit)
  uint32_t* zt;       // [n_tiles][m_tot] syndrome words
  float* ck;          // [T] x ck_stride: C^t, [n_tiles][s_tot][kLanes]
  size_t ck_stride;   // floats between consecutive iterations' messages
  float* lk;          // [T] x lk_stride: L^t, [n_tiles][n][kLanes]
  size_t lk_stride;
  float* w;           // [n_tiles][s_tot][kLanes] dJ/dV of the current backward iteration
  float* lbar;        // [n_tiles][n][kLanes] dJ/dL^t
  float* lpbar;       // [n_tiles][n][kLanes] dJ/dL_P
  float* partial;     // [T][blocks][2u] partial sums of dJ/dalpha, dJ/dbeta
};

size_t nbp_workspace_bytes(const DevCode& c, int F, int T);
void nbp_carve(const DevCode& c, int F, int T, void* ws, DevState* st, NbpState* ns);
int nbp_forward(const DevCode& c, DevState& st, const NbpState& ns, const float* llr, const uint32_t* z_bits,
                const float* alpha, const float* beta, double l_max, float* lv_out, cudaStream_t s);
int nbp_backward(const DevCode& c, const NbpState& ns, const float* alpha, const float* beta, double l_max,
                 const float* grad_lv, float* grad_alpha, float* grad_beta, float* grad_llr, cudaStream_t s);

}  // namespace mbp
