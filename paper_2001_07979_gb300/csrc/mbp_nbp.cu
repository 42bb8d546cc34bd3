// Unrolled normalised BP with learnable per-iteration, per-matrix scale and
// offset, forward and hand-written adjoint (mbp_nbp_forward / mbp_nbp_backward).
//
// Forward, iterations t = 1..T (flooding over all u matrices, no early exit):
//   V_e   = clip(L^{t-1}[i(e)] - C_e^{t-1})                 (L^0 = L_P, C^0 = 0)
//   c_e   = eq. (6) on the row's V (clipped magnitude, sign of the others and z_j)
//   C_e^t = alpha[t][l] * sgn(c_e) * max(|c_e| - beta[t][l], 0)       (l = the row's matrix)
//   L^t   = L_P + sum over the node's edges of C^t                   (eq. 2)
// with the same FP32 arithmetic and summation order as the plain decoder, so
// alpha = 1, beta = 0 reproduces it bit for bit. Every C^t and L^t is kept
// (per-iteration checkpoints) for the backward pass.
//
// Backward, t = T..1, given dJ/dL^t for every t:
//   Lbar^t = dJ/dL^t + sum over the node's edges of W^{t+1}          (total adjoint of L^t)
//   per check row, recomputing V, c and the masks from the checkpoints:
//     Cbar_e = Lbar^t[i(e)] - W_e^{t+1}                             (dJ/dC_e^t)
//     cbar_e = alpha Cbar_e where |c_e| > beta;  dalpha += Cbar_e sgn(c) (|c| - beta);
//     dbeta -= alpha Cbar_e sgn(c)
//     W_e^t  = dJ/dV_e^t (through the V clip) = m_e sgn(V_e) delta_e (1 - delta_e) S_e, with
//       S_e = sum_{k != e} u_k prod_{r != k, e} t_r,  u_k = cbar_k d_k sgn(c_k) / (D_k (1 - D_k)),
//       t_r = tanh(|V_r| / 2) = 1 - 2 delta_r, D_k the (+)-combination of the deltas of r != k,
//       d_k = 1 where |c_k| is below the clip. S comes from prefix and suffix sums of leave-one-out
//       products (O(d) per row, no division by an edge's own term).
//   dJ/dL_P = sum_t Lbar^t + sum over the node's edges of W^1.
// The per-block partial sums of dalpha and dbeta are reduced in a fixed order
// (deterministic). Units: the decoder runs in log2 units (LLR x log2 e), in
// which the Jacobian of eq. (6) is the same as in natural units; beta and the
// LLR gradients are converted at the boundary.
#include <cmath>

#include "mbp_device.cuh"
#include "mbp_nbp.h"

namespace mbp {
namespace {

using namespace dev;

inline unsigned blocks_for(int64_t n, int per) { return unsigned((n + per - 1) / per); }

constexpr float kLog2e = 1.4426950408889634f;
constexpr float kLn2 = 0.69314718055994531f;

// ---------------------------------------------------------------- layouts

// [F][n] frame-major (natural units) <-> [tile][n][lane] (internal units), 32 x 32 blocks through shared memory.
__global__ void to_tiles_kernel(const float* __restrict__ src, int F, int n, float scale, float* __restrict__ dst) {
  __shared__ float sm[32][33];
  const int tile = blockIdx.y, c0 = blockIdx.x * 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int r = w; r < 32; r += 8) {
    const int f = tile * kLanes + r, i = c0 + lane;
    sm[r][lane] = (f < F && i < n) ? src[int64_t(f) * n + i] * scale : 0.f;
  }
  __syncthreads();
  for (int r = w; r < 32; r += 8) {
    const int i = c0 + r;
    if (i < n) dst[(int64_t(tile) * n + i) * kLanes + lane] = sm[lane][r];
  }
}

__global__ void from_tiles_kernel(const float* __restrict__ src, int F, int n, float scale, float* __restrict__ dst) {
  __shared__ float sm[32][33];
  const int tile = blockIdx.y, c0 = blockIdx.x * 32;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int r = w; r < 32; r += 8) {
    const int i = c0 + r;
    sm[r][lane] = i < n ? src[(int64_t(tile) * n + i) * kLanes + lane] : 0.f;
  }
  __syncthreads();
  for (int r = w; r < 32; r += 8) {
    const int f = tile * kLanes + r, i = c0 + lane;
    if (f < F && i < n) dst[int64_t(f) * n + i] = sm[lane][r] * scale;
  }
}

// ---------------------------------------------------------------- forward

// One check row of one tile (warp, lane = frame): eq. (6) as in the plain
// decoder, then the normalisation of the row's matrix and iteration.
template <int D, bool CHECKED>
__device__ __forceinline__ void nbp_row_fwd(int deg, const int* __restrict__ cols, const float* __restrict__ gsrc,
                                            const float* __restrict__ cprev, float* __restrict__ cout, uint32_t par,
                                            float l_max, float d_lmax, float a, float b) {
  using A = Arith<float>;
  using B = Bits<float>;
  int col[D];
#pragma unroll
  for (int k = 0; k < D; ++k) col[k] = (!CHECKED || k < deg) ? __ldg(cols + k) : -1;
  float v[D];
#pragma unroll
  for (int k = 0; k < D; ++k) v[k] = (!CHECKED || col[k] >= 0) ? __ldg(gsrc + col[k] * kLanes) : 0.f;
  if (cprev) {
#pragma unroll
    for (int k = 0; k < D; ++k) v[k] -= (!CHECKED || col[k] >= 0) ? __ldcs(cprev + k * kLanes) : 0.f;
  }
  float pre[D];
  float P = 0.f;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const uint32_t sx = B::sign_word(v[k]);
    par ^= sx;
    float d = A::clipped_delta(v[k], l_max, d_lmax);
    if (CHECKED) d = col[k] >= 0 ? d : 0.f;
    v[k] = B::with_sign(d, sx & kSign);
    pre[k] = P;
    P = A::oplus(P, d);
  }
  float suf = 0.f;
#pragma unroll
  for (int k = D - 1; k >= 0; --k) {
    if (!CHECKED || col[k] >= 0) {
      const float mag = A::clipped_mag(A::oplus(pre[k], suf), l_max);
      const float nmag = a * fmaxf(mag - b, 0.f);
      __stcs(cout + k * kLanes, B::copy_sign(nmag, par ^ B::sign_word(v[k])));
    }
    suf = A::oplus(suf, fabsf(v[k]));
  }
}

template <int DMAX>
__global__ void __launch_bounds__(256) nbp_cn_fwd_kernel(const DevCode c, int t, int u, const float* __restrict__ lsrc,
                                                         const float* __restrict__ cprev_all, float* __restrict__ cout_all,
                                                         const uint32_t* __restrict__ zt, const float* __restrict__ alpha,
                                                         const float* __restrict__ beta, float l_max) {
  const int tile = blockIdx.y;
  const int p = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (p >= c.m_tot) return;
  const int lane = threadIdx.x & 31;
  const int base = c.slice_base[p];
  const int deg = c.slice_base[p + 1] - base;
  const int l = c.row_mat[p];
  const float a = alpha[(t - 1) * u + l], b = beta[(t - 1) * u + l] * kLog2e;
  const int64_t off = (int64_t(tile) * c.s_tot + base) * kLanes + lane;
  const float* cprev = cprev_all ? cprev_all + off : nullptr;
  float* cout = cout_all + off;
  const float* gsrc = lsrc + int64_t(tile) * c.n * kLanes + lane;
  const int* cols = c.slot_col + base;
  const uint32_t par = ((zt[int64_t(tile) * c.m_tot + p] >> lane) & 1u) << 31;
  const float inv = Arith<float>::delta(l_max);  // d_lmax
  if (deg == DMAX) nbp_row_fwd<DMAX, false>(deg, cols, gsrc, cprev, cout, par, l_max, inv, a, b);
  else if (DMAX > 1 && deg == DMAX - 1)
    nbp_row_fwd<(DMAX > 1 ? DMAX - 1 : 1), false>(deg, cols, gsrc, cprev, cout, par, l_max, inv, a, b);
  else nbp_row_fwd<DMAX, true>(deg, cols, gsrc, cprev, cout, par, l_max, inv, a, b);
}

// L^t = L_P + sum of the node's C^t in stacked-row order (the plain decoder's order).
__global__ void __launch_bounds__(256) nbp_vn_fwd_kernel(const DevCode c, const float* __restrict__ cin,
                                                         const float* __restrict__ lp, float* __restrict__ lout) {
  const int tile = blockIdx.y;
  const int col = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (col >= c.n) return;
  const int lane = threadIdx.x & 31;
  const int64_t at = (int64_t(tile) * c.n + col) * kLanes + lane;
  const float* msg = cin + int64_t(tile) * c.s_tot * kLanes + lane;
  const int a0 = c.col_ptr[col];
  const int d = c.col_ptr[col + 1] - a0;
  const int* slots = c.col_slot + a0;
  float sum = lp[at];
  if (d <= 4) sum = vn_sum<float, float, 4, kPolStream, kLanes>(slots, d, msg, sum);
  else if (d <= 8) sum = vn_sum<float, float, 8, kPolStream, kLanes>(slots, d, msg, sum);
  else
    for (int q = 0; q < d; q += 16) sum = vn_sum<float, float, 16, kPolStream, kLanes>(slots + q, d - q, msg, sum);
  lout[at] = sum;
}

// ---------------------------------------------------------------- backward

// Lbar <- Lbar + sum of the node's W (if w); LPbar <- LPbar + (that sum, or Lbar) as asked.
__global__ void __launch_bounds__(256) nbp_vn_bwd_kernel(const DevCode c, const float* __restrict__ w,
                                                         float* __restrict__ lbar, float* __restrict__ lpbar,
                                                         int lpbar_init) {
  const int tile = blockIdx.y;
  const int col = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (col >= c.n) return;
  const int lane = threadIdx.x & 31;
  const int64_t at = (int64_t(tile) * c.n + col) * kLanes + lane;
  float sum = lbar ? lbar[at] : 0.f;
  if (w) {
    const float* msg = w + int64_t(tile) * c.s_tot * kLanes + lane;
    const int a0 = c.col_ptr[col];
    const int d = c.col_ptr[col + 1] - a0;
    const int* slots = c.col_slot + a0;
    for (int q = 0; q < d; q += 16) sum = vn_sum<float, float, 16, kPolStream, kLanes>(slots + q, d - q, msg, sum);
  }
  if (lbar) lbar[at] = sum;
  if (lpbar) lpbar[at] = lpbar_init ? sum : lpbar[at] + sum;
}

// Adjoint of one check row (see the file header). Returns this lane's dalpha, dbeta contributions.
template <int D, bool CHECKED>
__device__ __forceinline__ void nbp_row_bwd(int deg, const int* __restrict__ cols, const float* __restrict__ gsrc,
                                            const float* __restrict__ cprev, const float* __restrict__ lbar,
                                            float* __restrict__ w, bool has_next, uint32_t par, float l_max,
                                            float d_lmax, float a, float b, float& ga, float& gb) {
  using A = Arith<float>;
  using B = Bits<float>;
  int col[D];
#pragma unroll
  for (int k = 0; k < D; ++k) col[k] = (!CHECKED || k < deg) ? __ldg(cols + k) : -1;
  float v[D], cb[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const bool on = !CHECKED || col[k] >= 0;
    v[k] = on ? __ldg(gsrc + col[k] * kLanes) : 0.f;
    cb[k] = on ? __ldg(lbar + col[k] * kLanes) : 0.f;
  }
  if (cprev) {
#pragma unroll
    for (int k = 0; k < D; ++k) v[k] -= (!CHECKED || col[k] >= 0) ? __ldcs(cprev + k * kLanes) : 0.f;
  }
  if (has_next) {
#pragma unroll
    for (int k = 0; k < D; ++k) cb[k] -= (!CHECKED || col[k] >= 0) ? w[k * kLanes] : 0.f;
  }
  // forward recomputation: deltas (sign of V in the sign bit), clip masks, prefix combinations
  uint32_t clipped_in = 0;  // bit k: |V_k| above the clip (no gradient through V_k)
  float pre[D];
  float P = 0.f;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const uint32_t sx = B::sign_word(v[k]);
    par ^= sx;
    if (fabsf(v[k]) > l_max) clipped_in |= 1u << k;
    float d = A::clipped_delta(v[k], l_max, d_lmax);
    if (CHECKED) d = col[k] >= 0 ? d : 0.f;
    v[k] = B::with_sign(d, sx & kSign);
    pre[k] = P;
    P = A::oplus(P, d);
  }
  // descending: D_k, c_k, the normalisation's adjoint, u_k, and the suffix sums A'_k, B'_k
  float Ap[D], Bp[D];
  float suf = 0.f, As = 1.f, Bs = 0.f;
#pragma unroll
  for (int k = D - 1; k >= 0; --k) {
    const float dk = fabsf(v[k]);
    float uk = 0.f;
    if (!CHECKED || col[k] >= 0) {
      const float Dk = A::oplus(pre[k], suf);
      const float g = A::mag(Dk);
      const float cm = A::clipped_mag(Dk, l_max);
      const float s = ((par ^ B::sign_word(v[k])) & kSign) ? -1.f : 1.f;
      if (cm > b) {
        ga += cb[k] * s * (cm - b);
        gb -= a * cb[k] * s;
        if (g < l_max) uk = a * cb[k] * s / (Dk * (1.f - Dk));
      }
    }
    Ap[k] = As;
    Bp[k] = Bs;
    const float tk = 1.f - 2.f * dk;
    Bs = Bs * tk + uk * As;
    As = As * tk;
    pre[k] = uk;
    suf = A::oplus(suf, dk);
  }
  // ascending: prefix sums A_k, B_k, S_k and W_k
  float Aq = 1.f, Bq = 0.f;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    if (!CHECKED || col[k] >= 0) {
      const float dk = fabsf(v[k]);
      const float S = Bq * Ap[k] + Aq * Bp[k];
      float wk = 0.f;
      if (!((clipped_in >> k) & 1u)) {
        const float sv = (B::sign_word(v[k]) & kSign) ? -1.f : 1.f;
        wk = sv * dk * (1.f - dk) * S;
      }
      w[k * kLanes] = wk;
    }
    const float tk = 1.f - 2.f * fabsf(v[k]);
    Bq = Bq * tk + pre[k] * Aq;
    Aq = Aq * tk;
  }
}

template <int DMAX>
__global__ void __launch_bounds__(256) nbp_cn_bwd_kernel(const DevCode c, int t, int u, int has_next,
                                                         const float* __restrict__ lsrc,
                                                         const float* __restrict__ cprev_all,
                                                         const float* __restrict__ lbar, float* __restrict__ w_all,
                                                         const uint32_t* __restrict__ zt,
                                                         const float* __restrict__ alpha,
                                                         const float* __restrict__ beta, float l_max,
                                                         float* __restrict__ partial) {
  __shared__ float s_ga[8], s_gb[8];
  __shared__ int s_l[8];
  const int tile = blockIdx.y;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = blockIdx.x * 8 + warp;
  float ga = 0.f, gb = 0.f;
  int l = -1;
  if (p < c.m_tot) {
    const int base = c.slice_base[p];
    const int deg = c.slice_base[p + 1] - base;
    l = c.row_mat[p];
    const float a = alpha[(t - 1) * u + l], b = beta[(t - 1) * u + l] * kLog2e;
    const int64_t off = (int64_t(tile) * c.s_tot + base) * kLanes + lane;
    const float* cprev = cprev_all ? cprev_all + off : nullptr;
    float* w = w_all + off;
    const int64_t node0 = int64_t(tile) * c.n * kLanes + lane;
    const int* cols = c.slot_col + base;
    const uint32_t par = ((zt[int64_t(tile) * c.m_tot + p] >> lane) & 1u) << 31;
    const float inv = Arith<float>::delta(l_max);  // d_lmax
    if (deg == DMAX)
      nbp_row_bwd<DMAX, false>(deg, cols, lsrc + node0, cprev, lbar + node0, w, has_next, par, l_max, inv, a, b, ga,
                               gb);
    else if (DMAX > 1 && deg == DMAX - 1)
      nbp_row_bwd<(DMAX > 1 ? DMAX - 1 : 1), false>(deg, cols, lsrc + node0, cprev, lbar + node0, w, has_next, par,
                                                    l_max, inv, a, b, ga, gb);
    else
      nbp_row_bwd<DMAX, true>(deg, cols, lsrc + node0, cprev, lbar + node0, w, has_next, par, l_max, inv, a, b, ga,
                              gb);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    ga += __shfl_xor_sync(kFull, ga, o);
    gb += __shfl_xor_sync(kFull, gb, o);
  }
  if (lane == 0) {
    s_ga[warp] = ga;
    s_gb[warp] = gb;
    s_l[warp] = l;
  }
  __syncthreads();
  // block partials [2u] in warp order (deterministic): dalpha of matrix l at [l], dbeta at [u + l]
  const int64_t blk = int64_t(blockIdx.y) * gridDim.x + blockIdx.x;
  if (threadIdx.x < 2 * u) {
    const int q = threadIdx.x % u;
    const bool is_b = threadIdx.x >= u;
    float acc = 0.f;
    for (int k = 0; k < 8; ++k)
      if (s_l[k] == q) acc += is_b ? s_gb[k] : s_ga[k];
    partial[blk * 2 * u + threadIdx.x] = acc;
  }
}

// grad[t][q] = scale_q * sum over blocks of partial[t][block][q], in block order with a double accumulator.
__global__ void nbp_reduce_kernel(const float* __restrict__ partial, int64_t n_blocks, int u,
                                  float* __restrict__ grad_alpha, float* __restrict__ grad_beta) {
  __shared__ double sm[256];
  const int t = blockIdx.y, q = blockIdx.x;  // q < 2u
  const float* p = partial + int64_t(t) * n_blocks * 2 * u + q;
  double acc = 0.0;
  for (int64_t b = threadIdx.x; b < n_blocks; b += blockDim.x) acc += double(p[b * 2 * u]);
  sm[threadIdx.x] = acc;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) sm[threadIdx.x] += sm[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (q < u) grad_alpha[t * u + q] = float(sm[0]);
    else grad_beta[t * u + (q - u)] = float(sm[0] * double(kLog2e));  // beta is an LLR offset: internal unit
  }
}

// launch helpers over the unroll bound of the code's largest check degree
#define MBP_NBP_DISPATCH(NAME, d, ...)            \
  do {                                            \
    if (d <= 4) NAME<4>(__VA_ARGS__);             \
    else if (d <= 6) NAME<6>(__VA_ARGS__);        \
    else if (d <= 8) NAME<8>(__VA_ARGS__);        \
    else if (d <= 10) NAME<10>(__VA_ARGS__);      \
    else if (d <= 12) NAME<12>(__VA_ARGS__);      \
    else if (d <= 14) NAME<14>(__VA_ARGS__);      \
    else if (d <= 16) NAME<16>(__VA_ARGS__);      \
    else if (d <= 20) NAME<20>(__VA_ARGS__);      \
    else if (d <= 24) NAME<24>(__VA_ARGS__);      \
    else NAME<32>(__VA_ARGS__);                   \
  } while (0)

template <int DMAX>
void launch_cn_fwd(const DevCode& c, const NbpState& ns, int t, const float* lsrc, const float* cprev, float* cout,
                   const float* alpha, const float* beta, float l_max, cudaStream_t s) {
  nbp_cn_fwd_kernel<DMAX><<<dim3(blocks_for(c.m_tot, 8), ns.n_tiles), 256, 0, s>>>(c, t, c.u, lsrc, cprev, cout,
                                                                                 ns.zt, alpha, beta, l_max);
}

template <int DMAX>
void launch_cn_bwd(const DevCode& c, const NbpState& ns, int t, int has_next, const float* lsrc, const float* cprev,
                   const float* alpha, const float* beta, float l_max, cudaStream_t s) {
  const int64_t nb = int64_t(blocks_for(c.m_tot, 8)) * ns.n_tiles;
  nbp_cn_bwd_kernel<DMAX><<<dim3(blocks_for(c.m_tot, 8), ns.n_tiles), 256, 0, s>>>(
      c, t, c.u, has_next, lsrc, cprev, ns.lbar, ns.w, ns.zt, alpha, beta, l_max,
      ns.partial + int64_t(t - 1) * nb * 2 * c.u);
}

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

size_t nbp_workspace_bytes(const DevCode& c, int F, int T) {
  const size_t NT = (size_t(F) + kLanes - 1) / kLanes;
  const size_t msgs = NT * size_t(c.s_tot) * kLanes * 4, nodes = NT * size_t(c.n) * kLanes * 4;
  const size_t nb = size_t(blocks_for(c.m_tot, 8)) * NT;
  return align256(workspace_bytes(c, F, MBP_MSG_F32, false)) + size_t(T) * align256(msgs) +
         size_t(T) * align256(nodes) + align256(msgs) + 2 * align256(nodes) + align256(size_t(T) * nb * 2 * c.u * 4);
}

void nbp_carve(const DevCode& c, int F, int T, void* ws, DevState* st, NbpState* ns) {
  const size_t NT = (size_t(F) + kLanes - 1) / kLanes;
  const size_t msgs = NT * size_t(c.s_tot) * kLanes * 4, nodes = NT * size_t(c.n) * kLanes * 4;
  char* b = static_cast<char*>(ws);
  carve_workspace(c, F, MBP_MSG_F32, false, b, st);
  b += align256(workspace_bytes(c, F, MBP_MSG_F32, false));
  ns->F = F;
  ns->T = T;
  ns->n_tiles = int(NT);
  ns->lp = static_cast<float*>(st->lp);
  ns->zt = st->zt;
  ns->ck = reinterpret_cast<float*>(b);
  ns->ck_stride = align256(msgs) / 4;
  b += size_t(T) * align256(msgs);
  ns->lk = reinterpret_cast<float*>(b);
  ns->lk_stride = align256(nodes) / 4;
  b += size_t(T) * align256(nodes);
  ns->w = reinterpret_cast<float*>(b);
  b += align256(msgs);
  ns->lbar = reinterpret_cast<float*>(b);
  b += align256(nodes);
  ns->lpbar = reinterpret_cast<float*>(b);
  b += align256(nodes);
  ns->partial = reinterpret_cast<float*>(b);
}

int nbp_forward(const DevCode& c, DevState& st, const NbpState& ns, const float* llr, const uint32_t* z_bits,
                const float* alpha, const float* beta, double l_max_nat, float* lv_out, cudaStream_t s) {
  cudaError_t e;
  DecodeArgs a{};
  a.llr = llr;
  a.z_bits = z_bits;
  a.max_iter = ns.T;
  a.l_max = l_max_nat;
  int rc = group_setup(c, st, MBP_MSG_F32, a, s);  // L_P (internal unit) and the syndrome words
  if (rc) return rc;
  const float l_max = float(l_max_nat * Arith<float>::kToInternal);  // as the plain decoder forms it
  const dim3 node_grid(blocks_for(c.n, 8), ns.n_tiles);
  const dim3 tr_grid(blocks_for(c.n, 32), ns.n_tiles);
  for (int t = 1; t <= ns.T; ++t) {
    const float* lsrc = t == 1 ? ns.lp : ns.lk + size_t(t - 2) * ns.lk_stride;
    const float* cprev = t == 1 ? nullptr : ns.ck + size_t(t - 2) * ns.ck_stride;
    float* cout = ns.ck + size_t(t - 1) * ns.ck_stride;
    float* lout = ns.lk + size_t(t - 1) * ns.lk_stride;
    MBP_NBP_DISPATCH(launch_cn_fwd, c.max_row_deg, c, ns, t, lsrc, cprev, cout, alpha, beta, l_max, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "nbp_cn_fwd_kernel");
    nbp_vn_fwd_kernel<<<node_grid, 256, 0, s>>>(c, cout, ns.lp, lout);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "nbp_vn_fwd_kernel");
    if (lv_out) {
      from_tiles_kernel<<<tr_grid, 256, 0, s>>>(lout, ns.F, c.n, kLn2, lv_out + size_t(t - 1) * ns.F * c.n);
      if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "from_tiles_kernel");
    }
  }
  return MBP_OK;
}

int nbp_backward(const DevCode& c, const NbpState& ns, const float* alpha, const float* beta, double l_max_nat,
                 const float* grad_lv, float* grad_alpha, float* grad_beta, float* grad_llr, cudaStream_t s) {
  cudaError_t e;
  const float l_max = float(l_max_nat * Arith<float>::kToInternal);  // as the plain decoder forms it
  const dim3 node_grid(blocks_for(c.n, 8), ns.n_tiles);
  const dim3 tr_grid(blocks_for(c.n, 32), ns.n_tiles);
  for (int t = ns.T; t >= 1; --t) {
    // Lbar^t = dJ/dL^t (internal unit: times ln 2) + sum of the node's W^{t+1}; dJ/dL_P collects every Lbar^t
    to_tiles_kernel<<<tr_grid, 256, 0, s>>>(grad_lv + size_t(t - 1) * ns.F * c.n, ns.F, c.n, kLn2, ns.lbar);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "to_tiles_kernel");
    nbp_vn_bwd_kernel<<<node_grid, 256, 0, s>>>(c, t < ns.T ? ns.w : nullptr, ns.lbar, grad_llr ? ns.lpbar : nullptr,
                                                t == ns.T);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "nbp_vn_bwd_kernel");
    const float* lsrc = t == 1 ? ns.lp : ns.lk + size_t(t - 2) * ns.lk_stride;
    const float* cprev = t == 1 ? nullptr : ns.ck + size_t(t - 2) * ns.ck_stride;
    MBP_NBP_DISPATCH(launch_cn_bwd, c.max_row_deg, c, ns, t, t < ns.T, lsrc, cprev, alpha, beta, l_max, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "nbp_cn_bwd_kernel");
  }
  const int64_t nb = int64_t(blocks_for(c.m_tot, 8)) * ns.n_tiles;
  nbp_reduce_kernel<<<dim3(2 * c.u, ns.T), 256, 0, s>>>(ns.partial, nb, c.u, grad_alpha, grad_beta);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "nbp_reduce_kernel");
  if (grad_llr) {
    nbp_vn_bwd_kernel<<<node_grid, 256, 0, s>>>(c, ns.w, nullptr, ns.lpbar, 0);  // + sum of the node's W^1
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "nbp_vn_bwd_kernel");
    from_tiles_kernel<<<tr_grid, 256, 0, s>>>(ns.lpbar, ns.F, c.n, kLog2e, grad_llr);  // L_P = llr x log2 e
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_error(e, "from_tiles_kernel");
  }
  return MBP_OK;
}

}  // namespace mbp
