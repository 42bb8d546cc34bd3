// Device building blocks of libmbp (sm_103a), shared by the streaming and the
// resident schedules.
//
// Data layout (per decode, inside the caller's workspace): kLanes = 32 frames
// form a tile; every per-edge or per-node array stores the tile's 32 frames of
// one edge or node contiguously, so each random access moves one 128-byte line
// (FP32) and one warp (lane = frame) handles one check row or one variable
// node of one tile. Message slots are shared by tile pairs (msg_at: FP32 in two
// adjacent lines, 2-byte messages interleaved in one line), and the fast
// kernels (mbp_pair.cuh) give each lane the frame of both tiles.
//
// Check-node arithmetic. For a check with incoming V2C values v_k, eq. (6) gives
//   |C2V_k| = 2 atanh( prod_{r != k} tanh(|v_r| / 2) ),
//   sign(C2V_k) = (-1)^{z_j} prod_{r != k} sign(v_r).
// With delta_r = (1 - tanh(|v_r| / 2)) / 2 = 1 / (1 + e^{|v_r|}) the product
// becomes 1 - 2 D_k with D_k = (+)_{r != k} delta_r under x (+) y = x + y - 2 x y
// (the complement of a product, halved), and 2 atanh(1 - 2 D) = ln((1 - D) / D).
// Working with delta keeps full relative precision for reliable messages
// (delta ~ e^{-|v|}) where tanh rounds to 1 in FP32. The exclusion r != k uses
// prefix and suffix (+)-combinations, never a division. Per edge this is two
// MUFU operations in, two out (exp + reciprocal, reciprocal + log).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "mbp_internal.h"

namespace mbp {
namespace dev {

constexpr uint32_t kFull = 0xffffffffu;
constexpr uint32_t kSign = 0x80000000u;

// Approximate MUFU forms with denormals flushed (the decoder's values stay normal
// or are meant to vanish), straight from the PTX ISA.
__device__ __forceinline__ float ex2_ftz(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float rcp_ftz(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float lg2_ftz(float x) {
  float y;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Check-node arithmetic in the halved complement form (see the file header).
// FP32 messages are kept in log2 units inside the decoder (LLR * log2 e), so
// e^{|v|} is one ex2 and the natural log is one lg2: delta = rcp(1 + ex2(a)),
// magnitude = lg2((1 - D) / D) = lg2(rcp(D) - 1). FP64 keeps natural units and
// the libm exp/log. kToInternal / kToLLR convert at the boundary (set-up and
// outputs).
//
// The clip of eq. (6)'s inputs and outputs to L = l_max: delta falls with |v|,
// so delta(min(|v|, L)) = max(delta(|v|), delta(L)), one FMNMX with the row's
// d_lmax = delta(L); the output clip is one more. In FP32 a rounding-level
// negative magnitude (D a hair below 1/2) is taken as its absolute value.
template <typename M>
struct Arith;

template <>
struct Arith<float> {
  static constexpr double kToInternal = 1.4426950408889634074;  // log2(e)
  static constexpr float kToLLR = 0.69314718055994530942f;      // ln(2)
  static __device__ __forceinline__ float delta(float a) { return rcp_ftz(1.0f + ex2_ftz(a)); }
  static __device__ __forceinline__ float oplus(float p, float d) { return fmaf(d, fmaf(-2.0f, p, 1.0f), p); }
  static __device__ __forceinline__ float mag(float D) { return lg2_ftz(rcp_ftz(D) - 1.0f); }
  // delta(min(|v|, L)); d_lmax = delta(L)
  static __device__ __forceinline__ float clipped_delta(float v, float, float d_lmax) {
    return fmaxf(delta(fabsf(v)), d_lmax);
  }
  // min(|mag(D)|, L)
  static __device__ __forceinline__ float clipped_mag(float D, float L) { return fminf(fabsf(mag(D)), L); }
};

template <>
struct Arith<double> {
  static constexpr double kToInternal = 1.0;
  static constexpr double kToLLR = 1.0;
  static __device__ __forceinline__ double delta(double a) { return 1.0 / (1.0 + exp(a)); }
  static __device__ __forceinline__ double oplus(double p, double d) { return fma(d, fma(-2.0, p, 1.0), p); }
  static __device__ __forceinline__ double mag(double D) { return log((1.0 - D) / D); }
  static __device__ __forceinline__ double clipped_delta(double v, double L, double) { return delta(fmin(fabs(v), L)); }
  static __device__ __forceinline__ double clipped_mag(double D, double L) { return fmax(fmin(mag(D), L), 0.0); }
};

// Sign-bit access: sign_word returns a 32-bit word whose top bit is the sign.
template <typename M>
struct Bits;

template <>
struct Bits<float> {
  static __device__ __forceinline__ uint32_t sign_word(float x) { return __float_as_uint(x); }
  static __device__ __forceinline__ float with_sign(float m, uint32_t sign) {
    return __uint_as_float(__float_as_uint(m) | sign);
  }
  // |m| with the top bit of `word` as sign
  static __device__ __forceinline__ float copy_sign(float m, uint32_t word) {
    return __uint_as_float((__float_as_uint(m) & ~kSign) | (word & kSign));
  }
};

template <>
struct Bits<double> {
  static __device__ __forceinline__ uint32_t sign_word(double x) { return uint32_t(__double2hiint(x)); }
  static __device__ __forceinline__ double with_sign(double m, uint32_t sign) {
    return __hiloint2double(int(uint32_t(__double2hiint(m)) | sign), __double2loint(m));
  }
  static __device__ __forceinline__ double copy_sign(double m, uint32_t word) {
    const uint32_t hi = (uint32_t(__double2hiint(m)) & ~kSign) | (word & kSign);
    return __hiloint2double(int(hi), __double2loint(m));
  }
};

// Stored message type S and arithmetic type M: FP32 and FP64 store what they
// compute; FP16 and BF16 store rounded copies of FP32 messages (round to
// nearest even) and widen them on load.
template <typename S>
struct Store;

template <>
struct Store<float> {
  static __device__ __forceinline__ float widen(float v) { return v; }
  static __device__ __forceinline__ float narrow(float v) { return v; }
};

template <>
struct Store<double> {
  static __device__ __forceinline__ double widen(double v) { return v; }
  static __device__ __forceinline__ double narrow(double v) { return v; }
};

template <>
struct Store<__half> {
  static __device__ __forceinline__ float widen(__half v) { return __half2float(v); }
  static __device__ __forceinline__ __half narrow(float v) { return __float2half_rn(v); }
};

template <>
struct Store<__nv_bfloat16> {
  static __device__ __forceinline__ float widen(__nv_bfloat16 v) { return __bfloat162float(v); }
  static __device__ __forceinline__ __nv_bfloat16 narrow(float v) { return __float2bfloat16_rn(v); }
};

// Message addressing (the layout of mbp_internal.h): slot k of a tile's row is
// kMsgStride<S> elements after slot k - 1. Tiles 2q and 2q + 1 share each
// slot: 2-byte messages interleave them lane by lane (one 128-byte line), 4-byte
// messages put them in two adjacent 128-byte lines, so a kernel of one tile
// still reads whole lines and a kernel of the pair gathers 256 contiguous bytes
// per edge (random 256-byte units run at the copy bandwidth on GB300, random
// 128-byte lines at about two thirds of it).
template <typename S>
constexpr int kMsgTiles = sizeof(S) <= 4 ? 2 : 1;
template <typename S>
constexpr int kMsgStride = kLanes * kMsgTiles<S>;
// Element of (tile, slot 0, lane).
template <typename S>
__device__ __forceinline__ int64_t msg_at(int tile, int s_tot, int lane) {
  constexpr int P = kMsgTiles<S>;
  const int64_t q = int64_t(tile / P) * s_tot * kMsgStride<S>;
  if constexpr (sizeof(S) == 2) return q + lane * P + tile % P;
  else return q + (tile % P) * kLanes + lane;
}

// Memory policies.
//  kPolStream:   streaming kernels, which only read data written by earlier
//                launches: posterior through the read-only path, messages
//                loaded and stored evict-first (touched once per iteration).
//  kPolCoherent: the persistent resident schedule, whose phases read data
//                written by other blocks of the same launch: every such load
//                goes to L2 (.cg, no stale L1 line) and messages stay in L2.
constexpr int kPolStream = 0, kPolCoherent = 1;
template <int POL, typename T>
__device__ __forceinline__ T ld_state(const T* p) {
  if constexpr (POL == kPolCoherent) return __ldcg(p);
  else return __ldg(p);
}
template <int POL, typename T>
__device__ __forceinline__ T ld_msg(const T* p) {
  if constexpr (POL == kPolCoherent) return __ldcg(p);
  else return __ldcs(p);
}
template <int POL, typename T>
__device__ __forceinline__ void st_msg(T* p, T v) {
  if constexpr (POL == kPolCoherent) __stcg(p, v);
  else __stcs(p, v);
}

// Channel LLR L_P of one node for this lane. BSC inputs keep Bob's bits as one
// word per node (bit = lane) and ln((1 - e)/e) per lane, so L_P = (1 - 2y) mag
// (eq. 5) costs a 4-byte broadcast load instead of a 128-byte vector; general
// inputs keep the LLR array (yt == NULL). tn = tile * n + node.
template <typename M, int POL>
__device__ __forceinline__ M channel_llr(const M* __restrict__ lp, const uint32_t* __restrict__ yt,
                                         const M* __restrict__ ymag, int64_t tn, int tile, int lane) {
  if (yt) {
    const M m = ld_state<POL>(ymag + tile * kLanes + lane);
    return ((ld_state<POL>(yt + tn) >> lane) & 1u) ? -m : m;
  }
  return ld_state<POL>(lp + tn * kLanes + lane);
}

// ------------------------------------------------------------- eq. (6)

// The check-node update of eq. (6) for one row and one lane (frame).
// Every load of the row is issued before the first use: the row's columns, then
// the posterior gathers and the old messages, so a warp waits for two memory
// round trips per row rather than two per edge. CHECKED = false is the body for
// rows of exactly D edges (no per-edge tests).
//
// Signs travel in IEEE sign bits: the row's sign parity (with z_j) is the XOR
// of the V2C words' top bits, and each edge's own sign is kept in the sign bit
// of its delta, whose magnitude the (+) operations read through |.|.
//
// ysrc != NULL: the first iteration of BSC inputs, where V2C = L_P comes from
// the sign words ysrc (bit = lane) and this lane's magnitude ymag instead of
// gsrc (a warp-uniform branch): all of the frame's V2C then share one
// magnitude, and the row's output magnitude is formed once.
//
// FIXED: also add each edge's change of message, q(C2V_new) - q(C2V_old) with
// q(x) = round(x * qscale), to the posterior accumulator lacc of its variable
// node (a 32-bit red.global.add in L2). Integer addition is associative, so
// the accumulated sum sum_e q(C2V_e) is exact and independent of the order of
// the atomics; finalize_kernel turns it into L_V.
// First iteration of BSC inputs: every V2C of a frame has the magnitude ymag,
// so the combination of a row's other edges is the same deg - 1 fold for every
// edge; its output magnitude is formed once per row.
template <typename M, int D, bool CHECKED>
__device__ __forceinline__ M cn_first_mag(int deg, M ymag, M l_max, M d_lmax) {
  const M d = Arith<M>::clipped_delta(ymag, l_max, d_lmax);
  M P = M(0);
#pragma unroll
  for (int k = 0; k < D - 1; ++k)
    if (!CHECKED || k + 1 < deg) P = Arith<M>::oplus(P, d);
  return Arith<M>::clipped_mag(P, l_max);
}

// cn_first_mag for a row of any degree (the same operations in the same order).
template <typename M>
__device__ __forceinline__ M cn_first_mag_any(int deg, M ymag, M l_max, M d_lmax) {
  const M d = Arith<M>::clipped_delta(ymag, l_max, d_lmax);
  M P = M(0);
  for (int k = 0; k + 1 < deg; ++k) P = Arith<M>::oplus(P, d);
  return Arith<M>::clipped_mag(P, l_max);
}

// The stored value of a first-iteration magnitude in row form: rounded to the
// message type, so that a message rebuilt from it equals the stored one.
template <typename M, typename S>
__device__ __forceinline__ M row_mag(M mag) {
  return M(Store<S>::widen(Store<S>::narrow(mag)));
}

// A first-iteration C2V in row form (DevState::fmag): the magnitude of its row's
// degree with sign bit `lane` of rs ^ y (rs the row's sign word, y the node's
// sign word).
template <typename M>
__device__ __forceinline__ M row_msg(M rm, uint32_t rs, uint32_t y, int lane) {
  return Bits<M>::copy_sign(rm, (rs ^ y) << (31 - lane));
}

// 32 x 32 bit-matrix transpose across a warp: lane i holds row i (bit j =
// A[i][j]); afterwards lane j holds column j (bit i = A[i][j]). Five exchange
// rounds of block sizes 16, 8, 4, 2, 1, each swapping the off-diagonal blocks:
// a lane whose bit s is clear keeps the low halves of its 2s-bit blocks and
// takes its partner's low halves into the high halves (partner word rotated
// left by s), a lane whose bit s is set keeps the high halves and takes the
// partner's high halves into the low halves (rotated right by s). One shuffle,
// one funnel rotate and one bitwise select per round; the per-lane masks and
// rotate amounts depend on the lane only.
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t a) {
  const uint32_t lane = threadIdx.x & 31;
  constexpr uint32_t kMask[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
  for (int r = 0; r < 5; ++r) {
    const uint32_t s = 16u >> r;
    const uint32_t hi = uint32_t(int32_t(lane << (27 + r)) >> 31);  // all ones where lane bit s is set
    const uint32_t keep = kMask[r] ^ hi;
    const uint32_t amt = s ^ (hi & (s ^ (32u - s)));  // s, or 32 - s (a right rotation by s)
    const uint32_t o = __shfl_xor_sync(kFull, a, int(s));
    a = (a & keep) | (__funnelshift_l(o, o, amt) & ~keep);
  }
  return a;
}

// The first-iteration row of BSC inputs (see cn_first_mag): each edge takes the
// shared magnitude with the sign of the other edges' bits and z_j. The row's
// bits are kept as one mask (D <= 32), edges k >= deg are padding.
template <typename M, typename S, int D, bool CHECKED, int POL>
__device__ __forceinline__ void cn_row_signs(int deg, const int* __restrict__ cols, const uint32_t* __restrict__ ysrc,
                                             M ymag, S* __restrict__ msg, uint32_t par, bool store, M l_max,
                                             M d_lmax) {
  static_assert(D <= 32, "one bit per edge");
  const int lane = threadIdx.x & 31;
  uint32_t bits = 0;
#pragma unroll
  for (int k = 0; k < D; ++k)
    if (!CHECKED || k < deg) bits |= ((ld_state<POL>(ysrc + __ldg(cols + k)) >> lane) & 1u) << k;
  if (!store) return;
  par ^= uint32_t(__popc(bits) & 1) << 31;
  const M mag = cn_first_mag<M, D, CHECKED>(deg, ymag, l_max, d_lmax);
#pragma unroll
  for (int k = 0; k < D; ++k)
    if (!CHECKED || k < deg)
      st_msg<POL>(msg + k * kMsgStride<S>, Store<S>::narrow(Bits<M>::copy_sign(mag, par ^ (((bits >> k) & 1u) << 31))));
}

template <typename M, typename S, int D, bool FIXED, bool CHECKED, int POL, bool RIN = false>
__device__ __forceinline__ void cn_row(int deg, const int* __restrict__ cols, const M* __restrict__ gsrc,
                                       const uint32_t* __restrict__ ysrc, M ymag, S* __restrict__ msg,
                                       int first_iter, uint32_t par, bool store, M l_max, M d_lmax,
                                       int32_t* __restrict__ lacc, float qscale, const M* __restrict__ rm_p,
                                       const uint32_t* __restrict__ rs_p, const uint32_t* __restrict__ yprev) {
  int col[D];
#pragma unroll
  for (int k = 0; k < D; ++k) col[k] = (!CHECKED || k < deg) ? __ldg(cols + k) : -1;
  M v[D];
  if (ysrc) {
    if constexpr (!FIXED && D <= 32) {
      cn_row_signs<M, S, D, CHECKED, POL>(deg, cols, ysrc, ymag, msg, par, store, l_max, d_lmax);
      return;
    } else {
      const int lane = threadIdx.x & 31;
      uint32_t sgn[D];
#pragma unroll
      for (int k = 0; k < D; ++k) {
        sgn[k] = (!CHECKED || col[k] >= 0) ? ((ld_state<POL>(ysrc + col[k]) >> lane) & 1u) << 31 : 0u;
        par ^= sgn[k];
      }
      if (!store) return;
      const M mag = cn_first_mag<M, D, CHECKED>(deg, ymag, l_max, d_lmax);
#pragma unroll
      for (int k = 0; k < D; ++k)
        if (!CHECKED || col[k] >= 0) {
          const M nv = Bits<M>::copy_sign(mag, par ^ sgn[k]);
          st_msg<POL>(msg + k * kMsgStride<S>, Store<S>::narrow(nv));
          if constexpr (FIXED) {
            const int32_t dq = __float2int_rn(float(nv) * qscale);
            if (dq != 0) atomicAdd(lacc + col[k] * kLanes, dq);
          }
        }
      return;
    }
  } else {
#pragma unroll
    for (int k = 0; k < D; ++k) v[k] = (!CHECKED || col[k] >= 0) ? ld_state<POL>(gsrc + col[k] * kLanes) : M(0);
  }
  [[maybe_unused]] M old[FIXED ? D : 1];
  if constexpr (RIN) {  // iteration 2 after a row-form iteration 1: C2V^1 rebuilt from the row
    const int lane = threadIdx.x & 31;
    const M rm = ld_state<POL>(rm_p);
    const uint32_t rs = ld_state<POL>(rs_p);
    // lane k fetches edge k's sign word (one gather for the row; rows of up to 32
    // edges), then each edge's word is broadcast
    const uint32_t ymine = lane < deg ? ld_state<POL>(yprev + __ldg(cols + lane)) : 0u;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const uint32_t yk = __shfl_sync(kFull, ymine, k & 31);
      if (!CHECKED || col[k] >= 0) v[k] -= row_msg(rm, rs, yk, lane);
    }
  } else if (!first_iter) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const M o = (!CHECKED || col[k] >= 0) ? M(Store<S>::widen(ld_msg<POL>(msg + k * kMsgStride<S>))) : M(0);
      if constexpr (FIXED) old[k] = o;
      v[k] -= o;
    }
  } else if constexpr (FIXED) {
#pragma unroll
    for (int k = 0; k < D; ++k) old[k] = M(0);
  }
  M pre[D];
  M P = M(0);
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const uint32_t sx = Bits<M>::sign_word(v[k]);
    par ^= sx;
    M d = Arith<M>::clipped_delta(v[k], l_max, d_lmax);
    if constexpr (CHECKED) d = col[k] >= 0 ? d : M(0);
    v[k] = Bits<M>::with_sign(d, sx & kSign);
    pre[k] = P;
    P = Arith<M>::oplus(P, d);
  }
  if (!store) return;
  M suf = M(0);
#pragma unroll
  for (int k = D - 1; k >= 0; --k) {
    if (!CHECKED || col[k] >= 0) {
      const M Dk = Arith<M>::oplus(pre[k], suf);
      const M mag = Arith<M>::clipped_mag(Dk, l_max);
      const M nv = Bits<M>::copy_sign(mag, par ^ Bits<M>::sign_word(v[k]));
      st_msg<POL>(msg + k * kMsgStride<S>, Store<S>::narrow(nv));
      if constexpr (FIXED) {
        const int32_t dq = __float2int_rn(float(nv) * qscale) - __float2int_rn(float(old[k]) * qscale);
        if (dq != 0) atomicAdd(lacc + col[k] * kLanes, dq);
      }
    }
    suf = Arith<M>::oplus(suf, fabs(v[k]));
  }
}

// Check row p (degree order) of one tile, by one warp. Rows of exactly DMAX or
// DMAX - 1 edges take an unchecked body. lsrc is the posterior (L_P in the
// first iteration of general inputs); the first iteration of BSC inputs reads
// the sign words yt and magnitudes ymag instead.
// RIN: the old messages are the row's first-iteration messages in row form
// (iteration 2): rm_p / rs_p / yprev.
template <typename M, typename S, int DMAX, bool FIXED, int POL, bool RIN = false>
__device__ __forceinline__ void cn_tile_row_src(int deg, const int* __restrict__ cols,
                                                const M* __restrict__ gsrc, const uint32_t* __restrict__ ysrc,
                                                M ym, S* __restrict__ msg, int first_iter, uint32_t par,
                                                bool store, M l_max, M d_lmax, int32_t* __restrict__ lacc,
                                                float qscale, const M* __restrict__ rm_p = nullptr,
                                                const uint32_t* __restrict__ rs_p = nullptr,
                                                const uint32_t* __restrict__ yprev = nullptr) {
  if (deg == DMAX)
    cn_row<M, S, DMAX, FIXED, false, POL, RIN>(deg, cols, gsrc, ysrc, ym, msg, first_iter, par, store, l_max, d_lmax,
                                            lacc, qscale, rm_p, rs_p, yprev);
  else if (DMAX > 1 && deg == DMAX - 1)
    cn_row<M, S, (DMAX > 1 ? DMAX - 1 : 1), FIXED, false, POL, RIN>(deg, cols, gsrc, ysrc, ym, msg, first_iter, par,
                                                                  store, l_max, d_lmax, lacc, qscale, rm_p, rs_p,
                                                                  yprev);
  else
    cn_row<M, S, DMAX, FIXED, true, POL, RIN>(deg, cols, gsrc, ysrc, ym, msg, first_iter, par, store, l_max, d_lmax,
                                           lacc, qscale, rm_p, rs_p, yprev);
}

// The min-sum check rule (an algorithm variant) for one row and one lane, FP32
// arithmetic: V2C clipped to l_max as for eq. (6), then every edge gets the sign
// of the others (and z_j) and the smallest magnitude among the others, found
// from the row's two smallest magnitudes. Padding edges take no part.
template <typename S, int D, bool CHECKED, int POL>
__device__ __forceinline__ void cn_row_minsum(int deg, const int* __restrict__ cols, const float* __restrict__ gsrc,
                                              const uint32_t* __restrict__ ysrc, float ymag, S* __restrict__ msg,
                                              int first_iter, uint32_t par, bool store, float l_max) {
  int col[D];
#pragma unroll
  for (int k = 0; k < D; ++k) col[k] = (!CHECKED || k < deg) ? __ldg(cols + k) : -1;
  float v[D];
  if (ysrc) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < D; ++k)
      v[k] = (!CHECKED || col[k] >= 0) ? (((ld_state<POL>(ysrc + col[k]) >> lane) & 1u) ? -ymag : ymag) : 0.f;
  } else {
#pragma unroll
    for (int k = 0; k < D; ++k) v[k] = (!CHECKED || col[k] >= 0) ? ld_state<POL>(gsrc + col[k] * kLanes) : 0.f;
  }
  if (!first_iter) {
#pragma unroll
    for (int k = 0; k < D; ++k)
      v[k] -= (!CHECKED || col[k] >= 0) ? float(Store<S>::widen(ld_msg<POL>(msg + k * kMsgStride<S>))) : 0.f;
  }
  float m1 = __int_as_float(0x7f800000), m2 = m1;  // +inf
  int i1 = -1;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    par ^= Bits<float>::sign_word(v[k]);
    const float a = (!CHECKED || col[k] >= 0) ? fminf(fabsf(v[k]), l_max) : __int_as_float(0x7f800000);
    if (a < m1) {
      m2 = m1;
      m1 = a;
      i1 = k;
    } else if (a < m2) {
      m2 = a;
    }
  }
  if (!store) return;
#pragma unroll
  for (int k = 0; k < D; ++k)
    if (!CHECKED || col[k] >= 0) {
      const float mag = fminf(k == i1 ? m2 : m1, l_max);
      st_msg<POL>(msg + k * kMsgStride<S>, Store<S>::narrow(Bits<float>::copy_sign(mag, par ^ Bits<float>::sign_word(v[k]))));
    }
}

// One tile's arrays for the check-node update of its rows: pointers offset to
// the tile (and to this lane where the data is per frame).
template <typename M, typename S>
struct CnView {
  const int32_t* slice_base;
  const int32_t* slot_col;
  S* msg;                // the tile's messages, lane
  const M* gsrc;         // the tile's posterior (or L_P), lane
  const uint32_t* ysrc;  // the tile's sign words in the first iteration of BSC inputs, else NULL
  M ym;                  // this lane's ln((1 - e)/e) with ysrc
  const uint32_t* zt;    // the tile's syndrome words
  int32_t* lacc;         // the tile's fixed-point sums, lane (FIXED) or NULL
  uint32_t act;          // lanes still decoding
  // iteration 2 after a row-form iteration 1 (else NULL): the tile's magnitude table (by row degree, lane),
  // row sign words (row p at rs[p * rs_nt]) and Bob's sign words
  const M* rm;
  const uint32_t* rs;
  int rs_nt;
  const uint32_t* yprev;
};

template <typename M, typename S, int POL>
__device__ __forceinline__ CnView<M, S> cn_view(const DevCode& c, int tile, uint32_t act, int first_iter,
                                                S* __restrict__ c2v, const M* __restrict__ lsrc,
                                                const uint32_t* __restrict__ yt, const M* __restrict__ ymag,
                                                const uint32_t* __restrict__ zt, int32_t* __restrict__ lacc) {
  const int lane = threadIdx.x & 31;
  const int64_t node0 = int64_t(tile) * c.n * kLanes + lane;
  const bool signs = first_iter && yt;
  CnView<M, S> v;
  v.slice_base = c.slice_base;
  v.slot_col = c.slot_col;
  v.msg = c2v + msg_at<S>(tile, c.s_tot, lane);
  v.gsrc = lsrc + node0;
  v.ysrc = signs ? yt + int64_t(tile) * c.n : nullptr;
  v.ym = signs ? ld_state<POL>(ymag + tile * kLanes + lane) : M(0);
  v.zt = zt + int64_t(tile) * c.m_tot;
  v.lacc = lacc ? lacc + node0 : nullptr;
  v.act = act;
  v.rm = nullptr;
  v.rs = nullptr;
  v.rs_nt = 0;
  v.yprev = nullptr;
  return v;
}

// Check row p (degree order) of the view's tile, by one warp.
template <typename M, typename S, int DMAX, bool FIXED, int POL, bool RIN = false>
__device__ __forceinline__ void cn_view_row(const CnView<M, S>& v, int p, int first_iter, M l_max, M d_lmax,
                                            float qscale) {
  const int lane = threadIdx.x & 31;
  const int base = v.slice_base[p];
  const int deg = v.slice_base[p + 1] - base;
  const uint32_t par = ((v.zt[p] >> lane) & 1u) << 31;
  const bool store = (v.act >> lane) & 1u;
  cn_tile_row_src<M, S, DMAX, FIXED, POL, RIN>(deg, v.slot_col + base, v.gsrc, v.ysrc, v.ym,
                                               v.msg + int64_t(base) * kMsgStride<S>, first_iter, par, store, l_max,
                                               d_lmax, v.lacc, qscale, RIN ? v.rm + (deg - 1) * kLanes : nullptr,
                                               RIN ? v.rs + int64_t(p) * v.rs_nt : nullptr, v.yprev);
}

// Min-sum rule for check row p of the view's tile (FP32 arithmetic).
template <typename S, int DMAX, int POL>
__device__ __forceinline__ void cn_view_row_minsum(const CnView<float, S>& v, int p, int first_iter, float l_max) {
  const int lane = threadIdx.x & 31;
  const int base = v.slice_base[p];
  const int deg = v.slice_base[p + 1] - base;
  const uint32_t par = ((v.zt[p] >> lane) & 1u) << 31;
  const bool store = (v.act >> lane) & 1u;
  const int* cols = v.slot_col + base;
  S* msg = v.msg + int64_t(base) * kMsgStride<S>;
  if (deg == DMAX)
    cn_row_minsum<S, DMAX, false, POL>(deg, cols, v.gsrc, v.ysrc, v.ym, msg, first_iter, par, store, l_max);
  else if (DMAX > 1 && deg == DMAX - 1)
    cn_row_minsum<S, (DMAX > 1 ? DMAX - 1 : 1), false, POL>(deg, cols, v.gsrc, v.ysrc, v.ym, msg, first_iter, par,
                                                            store, l_max);
  else
    cn_row_minsum<S, DMAX, true, POL>(deg, cols, v.gsrc, v.ysrc, v.ym, msg, first_iter, par, store, l_max);
}

template <typename M, typename S, int DMAX, bool FIXED, int POL>
__device__ __forceinline__ void cn_tile_row(const DevCode& c, int tile, int p, uint32_t act, int first_iter,
                                            S* __restrict__ c2v, const M* __restrict__ lsrc,
                                            const uint32_t* __restrict__ yt, const M* __restrict__ ymag,
                                            const uint32_t* __restrict__ zt, M l_max, M d_lmax,
                                            int32_t* __restrict__ lacc, float qscale) {
  const CnView<M, S> v = cn_view<M, S, POL>(c, tile, act, first_iter, c2v, lsrc, yt, ymag, zt, FIXED ? lacc : nullptr);
  cn_view_row<M, S, DMAX, FIXED, POL>(v, p, first_iter, l_max, d_lmax, qscale);
}

// ------------------------------------------------------------- eq. (2)

// Sum of one node's messages, D >= its degree: the slot indices are loaded
// first, then all gathers are in flight together; the sum runs in stacked-row
// order (the order of col_slot). STRIDE: elements from one slot to the next
// (the decoder's message layout by default; buffers of one tile per slot pass
// kLanes).
template <typename M, typename S, int D, int POL, int STRIDE = kMsgStride<S>>
__device__ __forceinline__ M vn_sum(const int* __restrict__ slots, int d, const S* __restrict__ msg, M sum) {
  int slot[D];
#pragma unroll
  for (int k = 0; k < D; ++k) slot[k] = k < d ? __ldg(slots + k) : -1;
  M g[D];
#pragma unroll
  for (int k = 0; k < D; ++k)
    g[k] = slot[k] >= 0 ? M(Store<S>::widen(ld_msg<POL>(msg + int64_t(slot[k]) * STRIDE))) : M(0);
#pragma unroll
  for (int k = 0; k < D; ++k)
    if (slot[k] >= 0) sum += g[k];
  return sum;
}

// One tile's arrays for the variable-node update of its nodes.
template <typename M, typename S>
struct VnView {
  const int32_t* col_ptr;
  const int32_t* col_slot;
  const S* msg;          // the tile's messages, lane
  M* lv;                 // the tile's posteriors, lane
  const M* lp;           // the tile's L_P (general inputs), lane
  const uint32_t* yt;    // the tile's sign words (BSC inputs) or NULL
  M ym;                  // this lane's ln((1 - e)/e) with yt
  uint32_t* xh;          // the tile's decision words (node-major: node i at xh[i * nt])
  int nt;                // tiles of the decode
  uint32_t act;
};

template <typename M, typename S, int POL>
__device__ __forceinline__ VnView<M, S> vn_view(const DevCode& c, int tile, uint32_t act, const S* __restrict__ c2v,
                                                M* __restrict__ lv, const M* __restrict__ lp,
                                                const uint32_t* __restrict__ yt, const M* __restrict__ ymag,
                                                uint32_t* __restrict__ xh, int nt) {
  const int lane = threadIdx.x & 31;
  const int64_t node0 = int64_t(tile) * c.n * kLanes + lane;
  VnView<M, S> v;
  v.col_ptr = c.col_ptr;
  v.col_slot = c.col_slot;
  v.msg = c2v + msg_at<S>(tile, c.s_tot, lane);
  v.lv = lv + node0;
  v.lp = lp + node0;
  v.yt = yt ? yt + int64_t(tile) * c.n : nullptr;
  v.ym = yt ? ld_state<POL>(ymag + tile * kLanes + lane) : M(0);
  v.xh = xh + tile;
  v.nt = nt;
  v.act = act;
  return v;
}

// The update of N nodes of one degree class (degree d <= D) by one warp, all of
// their gathers in flight together: node j is vnode[q0 + j] with slots at
// slots0 + j * d (j < cnt). Each node's sum runs in the order of vn_core.
template <typename M, typename S, int D, int N, int POL>
__device__ __forceinline__ void vn_class_nodes(const VnView<M, S>& v, const int32_t* __restrict__ vnode, int q0,
                                               const int32_t* __restrict__ slots0, int d, int cnt) {
  const int lane = threadIdx.x & 31;
  int col[N];
#pragma unroll
  for (int j = 0; j < N; ++j) col[j] = j < cnt ? __ldg(vnode + q0 + j) : -1;
  M g[N][D];
#pragma unroll
  for (int j = 0; j < N; ++j)
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const bool on = j < cnt && k < d;
      const int slot = on ? __ldg(slots0 + j * d + k) : 0;
      g[j][k] = on ? M(Store<S>::widen(ld_msg<POL>(v.msg + int64_t(slot) * kMsgStride<S>))) : M(0);
    }
#pragma unroll
  for (int j = 0; j < N; ++j) {
    if (j >= cnt) break;
    M sum;
    if (v.yt) sum = ((ld_state<POL>(v.yt + col[j]) >> lane) & 1u) ? -v.ym : v.ym;
    else sum = ld_state<POL>(v.lp + int64_t(col[j]) * kLanes);
#pragma unroll
    for (int k = 0; k < D; ++k)
      if (k < d) sum += g[j][k];
    if ((v.act >> lane) & 1u) v.lv[int64_t(col[j]) * kLanes] = sum;
    const uint32_t hard = __ballot_sync(kFull, sum < M(0));
    if (lane == 0) {
      uint32_t* px = v.xh + int64_t(col[j]) * v.nt;
      *px = v.act == kFull ? hard : (ld_state<POL>(px) & ~v.act) | (hard & v.act);
    }
  }
}

// The variable-node update of node `col` of the view's tile, by one warp: the
// soft decision L_V = L_P + sum of the node's C2V over all matrices (eq. 2) and
// the hard decision, whose 32 lanes are one word of xh. Nodes with more than 16
// edges are summed 16 edges at a time, still in stacked-row order.
// The update of node `col` of the view's tile from its d slots (in stacked-row order).
template <typename M, typename S, int POL>
__device__ __forceinline__ void vn_core(const VnView<M, S>& v, int col, const int32_t* __restrict__ slots, int d) {
  const int lane = threadIdx.x & 31;
  M sum;
  if (v.yt) sum = ((ld_state<POL>(v.yt + col) >> lane) & 1u) ? -v.ym : v.ym;
  else sum = ld_state<POL>(v.lp + int64_t(col) * kLanes);
  if (d <= 4) sum = vn_sum<M, S, 4, POL>(slots, d, v.msg, sum);
  else if (d <= 8) sum = vn_sum<M, S, 8, POL>(slots, d, v.msg, sum);
  else
    for (int b = 0; b < d; b += 16) sum = vn_sum<M, S, 16, POL>(slots + b, d - b, v.msg, sum);
  if ((v.act >> lane) & 1u) v.lv[int64_t(col) * kLanes] = sum;
  const uint32_t hard = __ballot_sync(kFull, sum < M(0));
  if (lane == 0) {  // retired lanes keep their decision
    uint32_t* px = v.xh + int64_t(col) * v.nt;
    *px = v.act == kFull ? hard : (ld_state<POL>(px) & ~v.act) | (hard & v.act);
  }
}

// The variable-node update of node `col` of the view's tile, by one warp: the
// soft decision L_V = L_P + sum of the node's C2V over all matrices (eq. 2) and
// the hard decision, whose 32 lanes are one word of xh. Nodes with more than 16
// edges are summed 16 edges at a time, still in stacked-row order.
template <typename M, typename S, int POL>
__device__ __forceinline__ void vn_view_node(const VnView<M, S>& v, int col) {
  const int a0 = v.col_ptr[col];
  vn_core<M, S, POL>(v, col, v.col_slot + a0, v.col_ptr[col + 1] - a0);
}

template <typename M, typename S, int POL>
__device__ __forceinline__ void vn_node(const DevCode& c, int tile, int col, uint32_t act,
                                        const S* __restrict__ c2v, M* __restrict__ lv, const M* __restrict__ lp,
                                        const uint32_t* __restrict__ yt, const M* __restrict__ ymag,
                                        uint32_t* __restrict__ xh, int nt) {
  vn_view_node<M, S, POL>(vn_view<M, S, POL>(c, tile, act, c2v, lv, lp, yt, ymag, xh, nt), col);
}

// ------------------------------------------------------- stopping rule

// Rows r0 .. r0 + 31 of one tile, one per thread of a warp: the lanes whose hard
// decision breaks the row are ORed into fail[tile][l] (l = the row's matrix).
// The row's columns are all loaded before the decision words (node-major, nt
// tiles) are gathered.
template <int DMAX, int POL>
__device__ __forceinline__ void syn_rows(const DevCode& c, int tile, int r0, uint32_t act,
                                         const uint32_t* __restrict__ xh, int nt, const uint32_t* __restrict__ zt,
                                         uint32_t* __restrict__ fail) {
  const int r = r0 + (threadIdx.x & 31);
  uint32_t bad = 0;
  int l = -1;
  if (r < c.m_tot) {
    const int base = c.slice_base[r];
    const int deg = c.slice_base[r + 1] - base;
    const int* cp = c.slot_col + base;
    int col[DMAX];
#pragma unroll
    for (int k = 0; k < DMAX; ++k) col[k] = k < deg ? __ldg(cp + k) : -1;
    const uint32_t* x = xh + tile;
    uint32_t p = zt[int64_t(tile) * c.m_tot + r];
#pragma unroll
    for (int k = 0; k < DMAX; ++k)
      if (col[k] >= 0) p ^= ld_state<POL>(x + int64_t(col[k]) * nt);
    bad = p & act;
    l = c.row_mat[r];
  }
  const int l0 = __shfl_sync(kFull, l, 0);
  if (__all_sync(kFull, l == l0 || l < 0)) {
    const uint32_t agg = __reduce_or_sync(kFull, bad);
    if ((threadIdx.x & 31) == 0 && agg && l0 >= 0) atomicOr(&fail[tile * c.u + l0], agg);
  } else if (bad) {
    atomicOr(&fail[tile * c.u + l], bad);
  }
}

// Retire the lanes of one tile that satisfied every syndrome (or hit max_iter);
// returns the lanes still decoding.
__device__ __forceinline__ uint32_t update_tile(int tile, int F, int u, int t, int max_iter, int early_exit,
                                                uint32_t* __restrict__ active, uint32_t* __restrict__ fail,
                                                int32_t* __restrict__ iters, uint8_t* __restrict__ success,
                                                uint8_t* __restrict__ synd_ok, const int32_t* __restrict__ perm) {
  uint32_t act = __ldcg(active + tile);
  if (act == 0) return 0;
  uint32_t anyfail = 0;
  for (int l = 0; l < u; ++l) anyfail |= __ldcg(fail + tile * u + l);
  uint32_t done = 0;
  if (t >= max_iter) done = act;
  else if (early_exit) done = act & ~anyfail;
  if (done) {
    // the caller's frames of the tile's slots, loaded before any output is written
    int fr[kLanes];
    const int4* p4 = reinterpret_cast<const int4*>(perm + int64_t(tile) * kLanes);
#pragma unroll
    for (int k = 0; k < kLanes / 4; ++k) {
      const int4 v = __ldg(p4 + k);
      fr[4 * k] = v.x;
      fr[4 * k + 1] = v.y;
      fr[4 * k + 2] = v.z;
      fr[4 * k + 3] = v.w;
    }
#pragma unroll
    for (int lane = 0; lane < kLanes; ++lane) {
      if (!((done >> lane) & 1u) || tile * kLanes + lane >= F) continue;
      const int f = fr[lane];
      iters[f] = t;
      success[f] = uint8_t(!((anyfail >> lane) & 1u));
    }
    if (synd_ok)
      for (int l = 0; l < u; ++l) {
        const uint32_t fw = __ldcg(fail + tile * u + l);
#pragma unroll
        for (int lane = 0; lane < kLanes; ++lane)
          if (((done >> lane) & 1u) && tile * kLanes + lane < F)
            synd_ok[int64_t(fr[lane]) * u + l] = uint8_t(!((fw >> lane) & 1u));
      }
  }
  act &= ~done;
  active[tile] = act;
  for (int l = 0; l < u; ++l) fail[tile * u + l] = 0;
  return act;
}

}  // namespace dev
}  // namespace mbp
