// CUDA kernels and decode driver of libmbp (sm_103a).
//
// One decode iteration (Section 3A, Algorithm 1, flooding over all u matrices)
// is three kernels over the frame tiles that still have unfinished frames:
//   cn_kernel   eq. (6) for every check of every matrix, on V2C = clip(L_V - C2V)
//   vn_kernel   eq. (2): L_V = L_P + sum of the node's C2V over all u matrices,
//               and the hard decision
//   syn_kernel  + update_kernel: the stopping rule H_l x_hat = z^l for every l
// Frames are interleaved kLanes = 8 per tile, so every random access to a
// variable node or an edge moves one contiguous vector of 8 frames.
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
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <mutex>

#include "mbp_internal.h"

// Fixed device scratch of mbp_decode_bsc_static: the decoder state of one call,
// for callers that must not allocate. Every GPU that loads this library holds
// these bytes until the process exits; every call shares them.
static __device__ __align__(256) unsigned char g_static_scratch[MBP_STATIC_SCRATCH_BYTES];

namespace mbp {
namespace {

constexpr uint32_t kFull = 0xffffffffu;

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

// Check-node arithmetic in the halved complement form. With
// delta = (1 - tanh(|v|/2)) / 2 = 1 / (1 + e^{|v|}), the product of eq. (6)
// over a set of edges is 1 - 2 D with D the (+)-combination of their deltas
// under x (+) y = x + y - 2 x y (identity 0), and 2 atanh(1 - 2 D) =
// ln((1 - D) / D).
//
// FP32 messages are kept in log2 units inside the decoder (LLR * log2 e), so
// e^{|v|} is one ex2 and the natural log is one lg2: delta = rcp(1 + ex2(a)),
// magnitude = lg2((1 - D) * rcp(D)). FP64 keeps natural units and the libm
// exp/log. kToInternal / kToLLR convert at the boundary (set-up and outputs).
template <typename M>
struct Arith;

template <>
struct Arith<float> {
  static constexpr double kToInternal = 1.4426950408889634074;  // log2(e)
  static constexpr float kToLLR = 0.69314718055994530942f;      // ln(2)
  static __device__ __forceinline__ float delta(float a) { return rcp_ftz(1.0f + ex2_ftz(a)); }
  static __device__ __forceinline__ float oplus(float p, float d) { return fmaf(d, fmaf(-2.0f, p, 1.0f), p); }
  static __device__ __forceinline__ float mag(float D) { return lg2_ftz((1.0f - D) * rcp_ftz(D)); }
  // min(|v|, L) = L * sat(|v| / L) on the FMA pipe (.sat clamps to [0, 1])
  static __device__ __forceinline__ float clip_abs(float v, float L, float invL) {
    return __saturatef(fabsf(v) * invL) * L;
  }
  // min(mag(D), L); .sat also maps a rounding-level negative magnitude to +0
  static __device__ __forceinline__ float clipped_mag(float D, float L, float invL) {
    return __saturatef(mag(D) * invL) * L;
  }
};

template <>
struct Arith<double> {
  static constexpr double kToInternal = 1.0;
  static constexpr double kToLLR = 1.0;
  static __device__ __forceinline__ double delta(double a) { return 1.0 / (1.0 + exp(a)); }
  static __device__ __forceinline__ double oplus(double p, double d) { return fma(d, fma(-2.0, p, 1.0), p); }
  static __device__ __forceinline__ double mag(double D) { return log((1.0 - D) / D); }
  static __device__ __forceinline__ double clip_abs(double v, double L, double) { return fmin(fabs(v), L); }
  static __device__ __forceinline__ double clipped_mag(double D, double L, double) {
    return fmax(fmin(mag(D), L), 0.0);
  }
};

constexpr uint32_t kSign = 0x80000000u;

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
    return __uint_as_float((__float_as_uint(m) & ~kSignBit) | (word & kSignBit));
  }
  static constexpr uint32_t kSignBit = 0x80000000u;
};

template <>
struct Bits<double> {
  static __device__ __forceinline__ uint32_t sign_word(double x) { return uint32_t(__double2hiint(x)); }
  static __device__ __forceinline__ double with_sign(double m, uint32_t sign) {
    return __hiloint2double(int(uint32_t(__double2hiint(m)) | sign), __double2loint(m));
  }
  static __device__ __forceinline__ double copy_sign(double m, uint32_t word) {
    const uint32_t hi = (uint32_t(__double2hiint(m)) & 0x7fffffffu) | (word & 0x80000000u);
    return __hiloint2double(int(hi), __double2loint(m));
  }
};

// ------------------------------------------------------------- eq. (1)

// One thread per (frame, 32-row word) of matrix l.
__global__ void syndrome_kernel(const DevCode c, int l, const uint32_t* __restrict__ x, int F,
                                uint32_t* __restrict__ z_l) {
  const int wl = (c.m[l] + 31) >> 5;
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= int64_t(F) * wl) return;
  const int f = int(idx / wl), w = int(idx % wl);
  const int wn = (c.n + 31) >> 5;
  const uint32_t* xf = x + int64_t(f) * wn;
  uint32_t bits = 0;
  for (int b = 0; b < 32; ++b) {
    const int j = w * 32 + b;
    if (j >= c.m[l]) break;
    const int r = c.row_first[l] + j;
    uint32_t p = 0;
    for (int e = c.row_ptr[r]; e < c.row_ptr[r + 1]; ++e) {
      const int col = c.col_idx[e];
      p ^= (__ldg(xf + (col >> 5)) >> (col & 31)) & 1u;
    }
    bits |= p << b;
  }
  z_l[int64_t(f) * wl + w] = bits;
}

// ------------------------------------------------------------- eq. (5)

// L_P = (1 - 2y) ln((1 - e)/e); ln((1 - e)/e) once per block in double precision.
template <typename M>
__global__ void bsc_llr_kernel(const uint32_t* __restrict__ y, const double* __restrict__ qber, int n,
                               M* __restrict__ llr) {
  __shared__ double mag;
  const int f = blockIdx.y;
  if (threadIdx.x == 0) {
    const double e = qber[f];
    mag = log((1.0 - e) / e);
  }
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int wn = (n + 31) >> 5;
  const uint32_t bit = (y[int64_t(f) * wn + (i >> 5)] >> (i & 31)) & 1u;
  llr[int64_t(f) * n + i] = M(bit ? -mag : mag);
}

// ln((1 - e)/e) per frame in double precision, times `unit` (the decoder's internal LLR unit).
__global__ void frame_mag_kernel(const double* __restrict__ qber, int F, double unit, double* __restrict__ mag) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f < F) {
    const double e = qber[f];
    mag[f] = log((1.0 - e) / e) * unit;
  }
}

// ------------------------------------------------------------- set-up

// L_P into the interleaved layout and the hard decision of iteration 0.
// Block: 32 columns x 8 lanes.
template <typename M>
__global__ void init_lp_kernel(const DevCode c, int F, const M* __restrict__ llr, const uint32_t* __restrict__ y,
                               const double* __restrict__ mag, M* __restrict__ lp, uint8_t* __restrict__ xh,
                               int32_t* __restrict__ counters, int validate) {
  const int tile = blockIdx.y;
  const int lane = threadIdx.x & 7;
  const int col = blockIdx.x * 32 + (threadIdx.x >> 3);
  const int f = tile * kLanes + lane;
  const bool ok = col < c.n;
  M v = M(0);
  if (ok && f < F) {
    if (llr) {
      v = llr[int64_t(f) * c.n + col];
      if (validate && !isfinite(v)) atomicOr(&counters[1], 1);
      v = M(double(v) * Arith<M>::kToInternal);
    } else {
      const int wn = (c.n + 31) >> 5;
      const uint32_t bit = (y[int64_t(f) * wn + (col >> 5)] >> (col & 31)) & 1u;
      v = M(bit ? -mag[f] : mag[f]);
    }
  }
  if (ok) lp[(int64_t(tile) * c.n + col) * kLanes + lane] = v;
  const uint32_t b = __ballot_sync(kFull, ok && f < F && v < M(0));
  if (ok && lane == 0) xh[int64_t(tile) * c.n + col] = uint8_t(b >> (threadIdx.x & 24));
}

// Alice's syndrome bits, one byte per (tile, stacked row) with bit = lane.
__global__ void init_z_kernel(const DevCode c, int F, int n_tiles, const uint32_t* __restrict__ z,
                              uint8_t* __restrict__ zt) {
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= int64_t(n_tiles) * c.m_tot) return;
  const int tile = int(idx / c.m_tot), r = int(idx % c.m_tot);
  const int l = c.row_mat[r];
  const int j = c.row_local[r];
  int64_t off = 0;
  for (int q = 0; q < l; ++q) off += int64_t(F) * ((c.m[q] + 31) >> 5);
  const int wl = (c.m[l] + 31) >> 5;
  uint32_t byte = 0;
  for (int lane = 0; lane < kLanes; ++lane) {
    const int f = tile * kLanes + lane;
    if (f < F) byte |= ((z[off + int64_t(f) * wl + (j >> 5)] >> (j & 31)) & 1u) << lane;
  }
  zt[idx] = uint8_t(byte);
}

__global__ void init_tiles_kernel(int F, int n_tiles, int u, uint32_t* __restrict__ active,
                                  uint32_t* __restrict__ fail) {
  const int tile = blockIdx.x * blockDim.x + threadIdx.x;
  if (tile >= n_tiles) return;
  const int left = F - tile * kLanes;
  active[tile] = left >= kLanes ? 0xffu : ((1u << left) - 1u);
  for (int l = 0; l < u; ++l) fail[tile * u + l] = 0;
}

// ------------------------------------------------------------- eq. (6)

// One row of a slice for one lane: the check-node update of eq. (6).
// Every load of the row is issued before the first use: the slot columns, then
// the posterior gathers and the old messages, so a warp waits for two memory
// round trips per slice rather than two per edge. CHECKED = false is the path
// for slices whose 4 rows all have exactly D edges (no padding tests at all).
//
// Signs travel in IEEE sign bits: the row's sign parity (with z_j) is the XOR
// of the V2C words' top bits, and each edge's own sign is kept in the sign bit
// of its delta, whose magnitude the (+) operations read through |.|.
//
// FIXED: also add each edge's change of message, q(C2V_new) - q(C2V_old) with
// q(x) = round(x * qscale), to the posterior accumulator lacc of its variable
// node (a 32-bit red.global.add in L2). Integer addition is associative, so
// the accumulated sum sum_e q(C2V_e) is exact and independent of the order of
// the atomics; finalize_kernel turns it into L_V.
// Memory policies. COH = false: kernels of the streaming schedule, which only
// read data written by earlier launches (read-only path for the posterior, and
// evict-first loads/stores for the messages, which are touched once per
// iteration). COH = true: the persistent resident schedule, whose phases read
// data written by other blocks of the same launch, so every such load goes to
// L2 (.cg, no stale L1 line) and messages are stored to stay in L2.
template <bool COH, typename T>
__device__ __forceinline__ T ld_state(const T* p) {
  if constexpr (COH) return __ldcg(p);
  else return __ldg(p);
}
template <bool COH, typename T>
__device__ __forceinline__ T ld_msg(const T* p) {
  if constexpr (COH) return __ldcg(p);
  else return __ldcs(p);
}
template <bool COH, typename T>
__device__ __forceinline__ void st_msg(T* p, T v) {
  if constexpr (COH) __stcg(p, v);
  else __stcs(p, v);
}

template <typename M, int D, bool FIXED, bool CHECKED, bool COH>
__device__ __forceinline__ void cn_row(int deg, const int* __restrict__ cols_p, const M* __restrict__ gsrc,
                                       M* __restrict__ msg, int first_iter, uint32_t par, bool store, M l_max,
                                       M inv_l_max, int32_t* __restrict__ lacc, float qscale) {
  int col[D];
#pragma unroll
  for (int k = 0; k < D; ++k) col[k] = (!CHECKED || k < deg) ? __ldg(cols_p + k * kSliceRows) : -1;
  M v[D];
#pragma unroll
  for (int k = 0; k < D; ++k) v[k] = (!CHECKED || col[k] >= 0) ? ld_state<COH>(gsrc + col[k] * kLanes) : M(0);
  [[maybe_unused]] M old[FIXED ? D : 1];
  if (!first_iter) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const M o = (!CHECKED || col[k] >= 0) ? ld_msg<COH>(msg + k * kSliceRows * kLanes) : M(0);
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
    M d = Arith<M>::delta(Arith<M>::clip_abs(v[k], l_max, inv_l_max));
    if constexpr (CHECKED) d = col[k] >= 0 ? d : M(0);
    v[k] = Bits<M>::with_sign(d, sx & kSign);
    pre[k] = P;
    P = Arith<M>::oplus(P, d);
  }
  if (!store) return;
  M S = M(0);
#pragma unroll
  for (int k = D - 1; k >= 0; --k) {
    if (!CHECKED || col[k] >= 0) {
      const M Dk = Arith<M>::oplus(pre[k], S);
      const M mag = Arith<M>::clipped_mag(Dk, l_max, inv_l_max);
      const M nv = Bits<M>::copy_sign(mag, par ^ Bits<M>::sign_word(v[k]));
      st_msg<COH>(msg + k * kSliceRows * kLanes, nv);
      if constexpr (FIXED) {
        const int32_t dq = __float2int_rn(float(nv) * qscale) - __float2int_rn(float(old[k]) * qscale);
        if (dq != 0) atomicAdd(lacc + col[k] * kLanes, dq);
      }
    }
    S = Arith<M>::oplus(S, fabs(v[k]));
  }
}

// The check-node update of one slice (kSliceRows rows x kLanes frames) of one
// tile, by one warp. Slices of exactly DMAX or DMAX - 1 edges per row take an
// unchecked body.
template <typename M, int DMAX, bool FIXED, bool COH>
__device__ __forceinline__ void cn_slice(const DevCode& c, int tile, int s, uint32_t act, int first_iter,
                                         M* __restrict__ c2v, const M* __restrict__ lsrc,
                                         const uint8_t* __restrict__ zt, M l_max, M inv_l_max,
                                         int32_t* __restrict__ lacc, float qscale) {
  const int lid = threadIdx.x & 31;
  const int q = lid >> 3, lane = lid & 7;
  const int r = s * kSliceRows + q;
  const int base = c.slice_base[s];
  const int deg = (c.slice_base[s + 1] - base) / kSliceRows;
  const bool full = c.slice_full[s];
  const int64_t node0 = int64_t(tile) * c.n * kLanes + lane;
  M* msg = c2v + (int64_t(tile) * c.s_tot + base + q) * kLanes + lane;  // edge k at msg[k * kSliceRows * kLanes]
  const M* gsrc = lsrc + node0;                                         // node i at gsrc[i * kLanes]
  int32_t* lacc_lane = FIXED ? lacc + node0 : nullptr;
  const int* cols_p = c.slot_col + base + q;
  const bool row_ok = r < c.m_tot;
  const uint32_t zbyte = row_ok ? zt[int64_t(tile) * c.m_tot + r] : 0u;
  const uint32_t par = ((zbyte >> lane) & 1u) << 31;
  const bool store = row_ok && ((act >> lane) & 1u);
  if (full && deg == DMAX)
    cn_row<M, DMAX, FIXED, false, COH>(deg, cols_p, gsrc, msg, first_iter, par, store, l_max, inv_l_max, lacc_lane,
                                       qscale);
  else if (DMAX > 1 && full && deg == DMAX - 1)
    cn_row<M, (DMAX > 1 ? DMAX - 1 : 1), FIXED, false, COH>(deg, cols_p, gsrc, msg, first_iter, par, store, l_max,
                                                             inv_l_max, lacc_lane, qscale);
  else
    cn_row<M, DMAX, FIXED, true, COH>(deg, cols_p, gsrc, msg, first_iter, par, store, l_max, inv_l_max, lacc_lane,
                                      qscale);
}

// One warp per slice, 8 slices per block, grid.y = tile.
template <typename M, int DMAX, bool FIXED>
__global__ void __launch_bounds__(256) cn_kernel(const DevCode c, int first_iter, M* __restrict__ c2v,
                                                 const M* __restrict__ lsrc, const uint8_t* __restrict__ zt,
                                                 const uint32_t* __restrict__ active, M l_max,
                                                 int32_t* __restrict__ lacc, float qscale) {
  const int tile = blockIdx.y;
  const uint32_t act = active[tile];
  if (act == 0) return;
  const int s = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (s >= c.n_slices) return;
  cn_slice<M, DMAX, FIXED, false>(c, tile, s, act, first_iter, c2v, lsrc, zt, l_max, M(1) / l_max, lacc, qscale);
}

// ------------------------------------------------------------- eq. (2)

// Sum of one node's messages, D >= its degree: the slot indices are loaded
// first, then all gathers are in flight together; the sum runs in stacked-row
// order (the order of col_slot).
template <typename M, int D, bool COH>
__device__ __forceinline__ M vn_sum(const int* __restrict__ slots, int d, const M* __restrict__ msg, M sum) {
  int slot[D];
#pragma unroll
  for (int k = 0; k < D; ++k) slot[k] = k < d ? __ldg(slots + k) : -1;
  M g[D];
#pragma unroll
  for (int k = 0; k < D; ++k) g[k] = slot[k] >= 0 ? ld_msg<COH>(msg + int64_t(slot[k]) * kLanes) : M(0);
#pragma unroll
  for (int k = 0; k < D; ++k)
    if (slot[k] >= 0) sum += g[k];
  return sum;
}

// The variable-node update of 4 nodes x kLanes frames of one tile, by one warp
// (node = col0 + (lane id >> 3)). The unrolled body is picked from the largest
// degree among the warp's 4 nodes (warp-uniform); nodes with more than 16 edges
// are summed 16 edges at a time, still in stacked-row order.
template <typename M, bool COH>
__device__ __forceinline__ void vn_nodes(const DevCode& c, int tile, int col0, uint32_t act,
                                         const M* __restrict__ c2v, M* __restrict__ lv, const M* __restrict__ lp,
                                         uint8_t* __restrict__ xh) {
  const int lid = threadIdx.x & 31;
  const int lane = lid & 7;
  const int col = col0 + (lid >> 3);
  const bool ok = col < c.n;
  const int64_t at = (int64_t(tile) * c.n + col) * kLanes + lane;
  const M* msg = c2v + int64_t(tile) * c.s_tot * kLanes + lane;
  const int a0 = ok ? c.col_ptr[col] : 0;
  const int d = ok ? c.col_ptr[col + 1] - a0 : 0;
  const int dw = int(__reduce_max_sync(kFull, unsigned(d)));
  M sum = M(0);
  if (ok) {
    sum = lp[at];
    const int* slots = c.col_slot + a0;
    if (dw <= 4) sum = vn_sum<M, 4, COH>(slots, d, msg, sum);
    else if (dw <= 8) sum = vn_sum<M, 8, COH>(slots, d, msg, sum);
    else
      for (int b = 0; b < d; b += 16) sum = vn_sum<M, 16, COH>(slots + b, d - b, msg, sum);
    if ((act >> lane) & 1u) lv[at] = sum;
  }
  const uint32_t b = __ballot_sync(kFull, ok && sum < M(0));
  if (ok && lane == 0) {
    const uint32_t nb = (b >> (lid & 24)) & 0xffu;
    uint8_t* px = xh + int64_t(tile) * c.n + col;
    const uint32_t prev = ld_state<COH>(px);
    *px = uint8_t((prev & ~act) | (nb & act));
  }
}

// Block: 32 variable nodes x 8 lanes, grid.y = tile.
template <typename M>
__global__ void __launch_bounds__(256) vn_kernel(const DevCode c, const M* __restrict__ c2v, M* __restrict__ lv,
                                                 const M* __restrict__ lp, uint8_t* __restrict__ xh,
                                                 const uint32_t* __restrict__ active) {
  const int tile = blockIdx.y;
  const uint32_t act = active[tile];
  if (act == 0) return;
  vn_nodes<M, false>(c, tile, blockIdx.x * 32 + (threadIdx.x >> 5) * 4, act, c2v, lv, lp, xh);
}

// L_V = L_P + lacc / qscale and the hard decision, for the fixed-point single
// pass. Block: 32 variable nodes x 8 lanes.
template <typename M>
__global__ void __launch_bounds__(256) finalize_kernel(const DevCode c, const int32_t* __restrict__ lacc,
                                                       M* __restrict__ lv, const M* __restrict__ lp,
                                                       uint8_t* __restrict__ xh, const uint32_t* __restrict__ active,
                                                       float inv_qscale) {
  const int tile = blockIdx.y;
  const uint32_t act = active[tile];
  if (act == 0) return;
  const int lane = threadIdx.x & 7;
  const int col = blockIdx.x * 32 + (threadIdx.x >> 3);
  const bool ok = col < c.n;
  const int64_t at = (int64_t(tile) * c.n + col) * kLanes + lane;
  M sum = M(0);
  if (ok) {
    sum = lp[at] + M(float(lacc[at]) * inv_qscale);
    if ((act >> lane) & 1u) lv[at] = sum;
  }
  const uint32_t b = __ballot_sync(kFull, ok && sum < M(0));
  if (ok && lane == 0) {
    const uint32_t nb = (b >> (threadIdx.x & 24)) & 0xffu;
    uint8_t* px = xh + int64_t(tile) * c.n + col;
    *px = uint8_t((*px & ~act) | (nb & act));
  }
}

// ------------------------------------------------------- stopping rule

// 32 rows of one tile, by one warp (row = r0 + lane id): lanes whose hard
// decision breaks a row of H_l are ORed into fail[tile][l]. The row's columns
// come from the slot layout and are all loaded before the decision bytes.
template <int DMAX, bool COH>
__device__ __forceinline__ void syn_rows(const DevCode& c, int tile, int r0, uint32_t act,
                                         const uint8_t* __restrict__ xh, const uint8_t* __restrict__ zt,
                                         uint32_t* __restrict__ fail) {
  const int r = r0 + (threadIdx.x & 31);
  uint32_t bad = 0;
  int l = -1;
  if (r < c.m_tot) {
    const int s = r / kSliceRows, q = r % kSliceRows;
    const int base = c.slice_base[s];
    const int deg = (c.slice_base[s + 1] - base) / kSliceRows;
    const int* cp = c.slot_col + base + q;
    int col[DMAX];
#pragma unroll
    for (int k = 0; k < DMAX; ++k) col[k] = k < deg ? __ldg(cp + k * kSliceRows) : -1;
    const uint8_t* x = xh + int64_t(tile) * c.n;
    uint32_t p = zt[int64_t(tile) * c.m_tot + r];
#pragma unroll
    for (int k = 0; k < DMAX; ++k)
      if (col[k] >= 0) p ^= ld_state<COH>(x + col[k]);
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

template <int DMAX>
__global__ void __launch_bounds__(256) syn_kernel(const DevCode c, const uint8_t* __restrict__ xh,
                                                  const uint8_t* __restrict__ zt,
                                                  const uint32_t* __restrict__ active, uint32_t* __restrict__ fail) {
  const int tile = blockIdx.y;
  const uint32_t act = active[tile];
  if (act == 0) return;
  syn_rows<DMAX, false>(c, tile, blockIdx.x * blockDim.x + (threadIdx.x & ~31), act, xh, zt, fail);
}

// Retire the lanes of one tile that satisfied every syndrome (or hit max_iter);
// returns the lanes still decoding.
__device__ __forceinline__ uint32_t update_tile(int tile, int F, int u, int t, int max_iter, int early_exit,
                                                uint32_t* __restrict__ active, uint32_t* __restrict__ fail,
                                                int32_t* __restrict__ iters, uint8_t* __restrict__ success,
                                                uint8_t* __restrict__ synd_ok) {
  uint32_t act = __ldcg(active + tile);
  if (act == 0) return 0;
  uint32_t anyfail = 0;
  for (int l = 0; l < u; ++l) anyfail |= __ldcg(fail + tile * u + l);
  uint32_t done = 0;
  if (t >= max_iter) done = act;
  else if (early_exit) done = act & ~anyfail;
  for (int lane = 0; lane < kLanes; ++lane) {
    if (!((done >> lane) & 1u)) continue;
    const int f = tile * kLanes + lane;
    if (f >= F) continue;
    iters[f] = t;
    success[f] = uint8_t(!((anyfail >> lane) & 1u));
    if (synd_ok)
      for (int l = 0; l < u; ++l) synd_ok[int64_t(f) * u + l] = uint8_t(!((__ldcg(fail + tile * u + l) >> lane) & 1u));
  }
  act &= ~done;
  active[tile] = act;
  for (int l = 0; l < u; ++l) fail[tile * u + l] = 0;
  return act;
}

// One thread per tile.
__global__ void update_kernel(int F, int n_tiles, int u, int t, int max_iter, int early_exit,
                              uint32_t* __restrict__ active, uint32_t* __restrict__ fail,
                              int32_t* __restrict__ iters, uint8_t* __restrict__ success,
                              uint8_t* __restrict__ synd_ok, int32_t* __restrict__ counters) {
  const int tile = blockIdx.x * blockDim.x + threadIdx.x;
  if (tile >= n_tiles) return;
  if (update_tile(tile, F, u, t, max_iter, early_exit, active, fail, iters, success, synd_ok))
    atomicAdd(&counters[0], 1);
}

// ------------------------------------------------------- resident schedule
//
// One cooperative launch decodes the whole batch, a group of G tiles at a
// time: every block takes part in every phase of the group's iterations, the
// phases are separated by a grid-wide barrier, and the group's messages and
// posteriors (a few tens of MB) stay in L2 from one iteration to the next
// instead of streaming through HBM. The barrier wait is bounded: a block that
// waits longer than kBarrierTimeout cycles sets ctl->error and every block
// returns; the host reports MBP_ETIMEOUT.

struct ResidentCtl {
  unsigned bar_count;
  unsigned bar_gen;
  unsigned syn_done;
  int any_active;
  int error;
};

constexpr long long kBarrierTimeout = 4000000000LL;  // about 2 s at 2 GHz

// Barrier parameters: expected arrivals per barrier (the grid size, or more when
// the timeout path is being tested) and the wait limit in SM clock cycles.
struct BarrierCfg {
  unsigned arrivals;
  long long timeout;
};

__device__ __forceinline__ bool grid_sync(ResidentCtl* ctl, unsigned& gen, const BarrierCfg& bc) {
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned target = gen + 1;
    __threadfence();
    if (atomicAdd(&ctl->bar_count, 1u) == bc.arrivals - 1) {
      atomicExch(&ctl->bar_count, 0u);
      __threadfence();
      atomicExch(&ctl->bar_gen, target);
    } else {
      const long long t0 = clock64();
      while (static_cast<int>(*reinterpret_cast<volatile unsigned*>(&ctl->bar_gen) - target) < 0) {
        if (clock64() - t0 > bc.timeout || *reinterpret_cast<volatile int*>(&ctl->error)) {
          atomicExch(&ctl->error, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    gen = target;
    __threadfence();
  }
  __syncthreads();
  return *reinterpret_cast<volatile int*>(&ctl->error) == 0;
}

template <typename M, int DMAX>
__global__ void __launch_bounds__(256) resident_kernel(const DevCode c, int F, int n_tiles, int G, int max_iter,
                                                       int early_exit, M l_max, M* __restrict__ c2v,
                                                       M* __restrict__ lv, const M* __restrict__ lp,
                                                       uint8_t* __restrict__ xh, const uint8_t* __restrict__ zt,
                                                       uint32_t* __restrict__ active, uint32_t* __restrict__ fail,
                                                       int32_t* __restrict__ iters, uint8_t* __restrict__ success,
                                                       uint8_t* __restrict__ synd_ok, ResidentCtl* ctl,
                                                       BarrierCfg bc) {
  unsigned gen = 0;
  const int warps = gridDim.x * (blockDim.x >> 5);
  const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const M inv_l_max = M(1) / l_max;
  const int col_groups = (c.n + 3) / 4;
  const int row_groups = (c.m_tot + 31) / 32;
  __shared__ int last_block;

  // syndrome test of the group's hard decisions, then retirement by the last block to finish
  auto stop_test = [&](int g0, int gt, int t) -> bool {
    for (int it = gw; it < gt * row_groups; it += warps) {
      const int tile = g0 + it / row_groups;
      const uint32_t act = __ldcg(active + tile);
      if (act) syn_rows<DMAX, true>(c, tile, (it % row_groups) * 32, act, xh, zt, fail);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      last_block = atomicAdd(&ctl->syn_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (last_block) {
      __threadfence();
      int any = 0;
      for (int i = threadIdx.x; i < gt; i += blockDim.x)
        any |= update_tile(g0 + i, F, c.u, t, max_iter, early_exit, active, fail, iters, success, synd_ok) != 0;
      any = __syncthreads_or(any);
      if (threadIdx.x == 0) {
        ctl->any_active = any;
        ctl->syn_done = 0;
      }
    }
    return grid_sync(ctl, gen, bc);
  };

  for (int g0 = 0; g0 < n_tiles; g0 += G) {
    const int gt = min(G, n_tiles - g0);
    if (early_exit || max_iter == 0) {
      if (!stop_test(g0, gt, 0)) return;
      if (!*reinterpret_cast<volatile int*>(&ctl->any_active)) continue;
    }
    for (int t = 1; t <= max_iter; ++t) {
      const M* lsrc = t == 1 ? lp : lv;
      for (int it = gw; it < gt * c.n_slices; it += warps) {
        const int tile = g0 + it / c.n_slices;
        const uint32_t act = __ldcg(active + tile);
        if (act) cn_slice<M, DMAX, false, true>(c, tile, it % c.n_slices, act, t == 1, c2v, lsrc, zt, l_max, inv_l_max,
                                                nullptr, 0.f);
      }
      if (!grid_sync(ctl, gen, bc)) return;
      for (int it = gw; it < gt * col_groups; it += warps) {
        const int tile = g0 + it / col_groups;
        const uint32_t act = __ldcg(active + tile);
        if (act) vn_nodes<M, true>(c, tile, (it % col_groups) * 4, act, c2v, lv, lp, xh);
      }
      if (!grid_sync(ctl, gen, bc)) return;
      if (early_exit || t == max_iter) {
        if (!stop_test(g0, gt, t)) return;
        if (!*reinterpret_cast<volatile int*>(&ctl->any_active)) break;
      }
    }
  }
}

// ------------------------------------------------------------- outputs

__global__ void out_bits_kernel(const DevCode c, int F, const uint8_t* __restrict__ xh, uint32_t* __restrict__ out) {
  const int wn = (c.n + 31) >> 5;
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= int64_t(F) * wn) return;
  const int f = int(idx / wn), w = int(idx % wn);
  const int tile = f / kLanes, lane = f % kLanes;
  const uint8_t* x = xh + int64_t(tile) * c.n;
  uint32_t bits = 0;
  for (int b = 0; b < 32; ++b) {
    const int i = w * 32 + b;
    if (i >= c.n) break;
    bits |= uint32_t((x[i] >> lane) & 1u) << b;
  }
  out[idx] = bits;
}

template <typename M>
__global__ void soft_out_kernel(const DevCode c, int F, const M* __restrict__ lv, const M* __restrict__ lp,
                                const int32_t* __restrict__ iters, M* __restrict__ out) {
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= int64_t(F) * c.n) return;
  const int f = int(idx / c.n), i = int(idx % c.n);
  const int64_t at = (int64_t(f / kLanes) * c.n + i) * kLanes + (f % kLanes);
  out[idx] = M((iters[f] == 0 ? lp[at] : lv[at]) * Arith<M>::kToLLR);
}

template <typename M>
__global__ void export_c2v_kernel(const DevCode c, const M* __restrict__ c2v, int frame, M* __restrict__ out) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= c.e_tot) return;
  const int tile = frame / kLanes, lane = frame % kLanes;
  out[e] = M(c2v[(int64_t(tile) * c.s_tot + c.edge_slot[e]) * kLanes + lane] * Arith<M>::kToLLR);
}

// ------------------------------------------------------------- host side

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
inline unsigned blocks_for(int64_t n, int per) { return unsigned((n + per - 1) / per); }

template <typename M, int DMAX, bool FIXED>
void launch_cn(const DevCode& c, const DevState& st, int first_iter, double l_max, float qscale, cudaStream_t s) {
  dim3 grid(blocks_for(c.n_slices, 8), st.n_tiles);
  cn_kernel<M, DMAX, FIXED><<<grid, 256, 0, s>>>(c, first_iter, static_cast<M*>(st.c2v),
                                                 static_cast<const M*>(first_iter ? st.lp : st.lv), st.zt, st.active,
                                                 M(l_max), st.lacc, qscale);
}

template <typename M, bool FIXED>
void launch_cn_any(const DevCode& c, const DevState& st, int first_iter, double l_max, float qscale,
                   cudaStream_t s) {
  const int d = c.max_row_deg;
  if constexpr (sizeof(M) == 4 && !FIXED) {  // the main path: unroll bound at or one above the largest degree
    if (d <= 4) launch_cn<M, 4, FIXED>(c, st, first_iter, l_max, qscale, s);
    else if (d <= 6) launch_cn<M, 6, FIXED>(c, st, first_iter, l_max, qscale, s);
    else if (d <= 8) launch_cn<M, 8, FIXED>(c, st, first_iter, l_max, qscale, s);
    else if (d <= 10) launch_cn<M, 10, FIXED>(c, st, first_iter, l_max, qscale, s);
    else if (d <= 12) launch_cn<M, 12, FIXED>(c, st, first_iter, l_max, qscale, s);
    else if (d <= 14) launch_cn<M, 14, FIXED>(c, st, first_iter, l_max, qscale, s);
    else if (d <= 16) launch_cn<M, 16, FIXED>(c, st, first_iter, l_max, qscale, s);
    else if (d <= 18) launch_cn<M, 18, FIXED>(c, st, first_iter, l_max, qscale, s);
    else if (d <= 20) launch_cn<M, 20, FIXED>(c, st, first_iter, l_max, qscale, s);
    else if (d <= 22) launch_cn<M, 22, FIXED>(c, st, first_iter, l_max, qscale, s);
    else if (d <= 24) launch_cn<M, 24, FIXED>(c, st, first_iter, l_max, qscale, s);
    else if (d <= 32) launch_cn<M, 32, FIXED>(c, st, first_iter, l_max, qscale, s);
    else launch_cn<M, 64, FIXED>(c, st, first_iter, l_max, qscale, s);
  } else {
    if (d <= 8) launch_cn<M, 8, FIXED>(c, st, first_iter, l_max, qscale, s);
    else if (d <= 16) launch_cn<M, 16, FIXED>(c, st, first_iter, l_max, qscale, s);
    else if (d <= 32) launch_cn<M, 32, FIXED>(c, st, first_iter, l_max, qscale, s);
    else launch_cn<M, 64, FIXED>(c, st, first_iter, l_max, qscale, s);
  }
}

template <typename M>
void launch_vn_any(const DevCode& c, const DevState& st, cudaStream_t s) {
  vn_kernel<M><<<dim3(blocks_for(c.n, 32), st.n_tiles), 256, 0, s>>>(
      c, static_cast<const M*>(st.c2v), static_cast<M*>(st.lv), static_cast<const M*>(st.lp), st.xh, st.active);
}

// Tiles per group of the resident schedule: as many as keep the group's
// messages, posteriors and decisions within 3/4 of L2 (0 = does not fit).
template <typename M>
int resident_group(const DevCode& c, int n_tiles) {
  int dev = 0, l2 = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const double per_tile = double(c.s_tot) * kLanes * sizeof(M) + 2.0 * c.n * kLanes * sizeof(M) + c.n + c.m_tot;
  int g = int(0.75 * l2 / per_tile);
  if (const char* ev = std::getenv("MBP_RESIDENT_GROUP_TILES")) g = std::atoi(ev);  // tuning override
  return g < 1 ? 0 : (g < n_tiles ? g : n_tiles);
}

template <typename M, int DMAX>
cudaError_t launch_resident(const DevCode& c, const DevState& st, const DecodeArgs& a, int G, double l_max,
                            cudaStream_t s) {
  auto kern = resident_kernel<M, DMAX>;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorCooperativeLaunchTooLarge;
  int F = st.F, NT = st.n_tiles, max_iter = a.max_iter, early_exit = a.early_exit;
  M lm = M(l_max);
  M* c2v = static_cast<M*>(st.c2v);
  M* lv = static_cast<M*>(st.lv);
  const M* lp = static_cast<const M*>(st.lp);
  uint8_t* xh = st.xh;
  const uint8_t* zt = st.zt;
  uint32_t* active = st.active;
  uint32_t* fail = st.fail;
  int32_t* iters = a.iters;
  uint8_t* success = a.success;
  uint8_t* synd_ok = a.synd_ok;
  ResidentCtl* ctl = static_cast<ResidentCtl*>(st.ctl);
  DevCode cc = c;
  const unsigned grid = unsigned(per_sm * sms);
  BarrierCfg bc{grid, kBarrierTimeout};
  // Test hook for the bounded-wait path: MBP_TEST_BARRIER_EXTRA_ARRIVALS makes every barrier wait for arrivals
  // that never come, and MBP_TEST_BARRIER_TIMEOUT_US shortens the wait limit.
  if (const char* ev = std::getenv("MBP_TEST_BARRIER_EXTRA_ARRIVALS")) bc.arrivals += unsigned(std::atoi(ev));
  if (const char* ev = std::getenv("MBP_TEST_BARRIER_TIMEOUT_US")) bc.timeout = std::atoll(ev) * 2000LL;
  void* args[] = {&cc, &F, &NT, &G, &max_iter, &early_exit, &lm, &c2v, &lv, &lp, &xh, &zt, &active, &fail,
                  &iters, &success, &synd_ok, &ctl, &bc};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(kern), dim3(grid), dim3(256), args, 0, s);
}

template <typename M>
cudaError_t launch_resident_any(const DevCode& c, const DevState& st, const DecodeArgs& a, int G, double l_max,
                                cudaStream_t s) {
  const int d = c.max_row_deg;
  if constexpr (sizeof(M) == 4) {
    if (d <= 8) return launch_resident<M, 8>(c, st, a, G, l_max, s);
    if (d <= 14) return launch_resident<M, 14>(c, st, a, G, l_max, s);
    if (d <= 16) return launch_resident<M, 16>(c, st, a, G, l_max, s);
    if (d <= 24) return launch_resident<M, 24>(c, st, a, G, l_max, s);
    if (d <= 32) return launch_resident<M, 32>(c, st, a, G, l_max, s);
    return launch_resident<M, 64>(c, st, a, G, l_max, s);
  } else {
    if (d <= 8) return launch_resident<M, 8>(c, st, a, G, l_max, s);
    if (d <= 16) return launch_resident<M, 16>(c, st, a, G, l_max, s);
    if (d <= 32) return launch_resident<M, 32>(c, st, a, G, l_max, s);
    return launch_resident<M, 64>(c, st, a, G, l_max, s);
  }
}

// The streaming schedule: per iteration, kernels over every tile that still has
// unfinished frames; the host reads the number of such tiles after each stopping test.
template <typename M>
int stream_iterations(const DevCode& c, DevState& st, const DecodeArgs& a, bool fixed, double l_max, float qscale,
                      float inv_qscale, cudaStream_t s) {
  cudaError_t e;
#define CK(call, what) \
  if ((e = (call)) != cudaSuccess) return cuda_error(e, what)
#define CKL(what) CK(cudaGetLastError(), what)
  const int F = st.F, NT = st.n_tiles;
  const dim3 syn_grid(blocks_for(c.m_tot, 256), NT);
  int32_t host_ctr[1];
  auto stop_check = [&](int t, int* left) -> int {
    prof_begin(MBP_KERNEL_SYNDROME, s);
    if (c.max_row_deg <= 8) syn_kernel<8><<<syn_grid, 256, 0, s>>>(c, st.xh, st.zt, st.active, st.fail);
    else if (c.max_row_deg <= 16) syn_kernel<16><<<syn_grid, 256, 0, s>>>(c, st.xh, st.zt, st.active, st.fail);
    else if (c.max_row_deg <= 32) syn_kernel<32><<<syn_grid, 256, 0, s>>>(c, st.xh, st.zt, st.active, st.fail);
    else syn_kernel<kMaxRowDeg><<<syn_grid, 256, 0, s>>>(c, st.xh, st.zt, st.active, st.fail);
    CKL("syn_kernel");
    prof_end(MBP_KERNEL_SYNDROME, s, 1);
    CK(cudaMemsetAsync(st.counters, 0, sizeof(int32_t), s), "clear counter");
    prof_begin(MBP_KERNEL_RETIRE, s);
    update_kernel<<<blocks_for(NT, 128), 128, 0, s>>>(F, NT, c.u, t, a.max_iter, a.early_exit, st.active, st.fail,
                                                       a.iters, a.success, a.synd_ok, st.counters);
    CKL("update_kernel");
    prof_end(MBP_KERNEL_RETIRE, s, 1);
    CK(cudaMemcpyAsync(host_ctr, st.counters, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "read counter");
    CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    *left = host_ctr[0];
    return MBP_OK;
  };
  int left = NT;
  int rc;
  if (a.early_exit || a.max_iter == 0) {
    if ((rc = stop_check(0, &left))) return rc;
  }
  for (int t = 1; t <= a.max_iter && left > 0; ++t) {
    prof_begin(MBP_KERNEL_CHECK, s);
    if constexpr (sizeof(M) == 4) {
      if (fixed) launch_cn_any<M, true>(c, st, t == 1, l_max, qscale, s);
      else launch_cn_any<M, false>(c, st, t == 1, l_max, qscale, s);
    } else {
      launch_cn_any<M, false>(c, st, t == 1, l_max, qscale, s);
    }
    CKL("cn_kernel");
    prof_end(MBP_KERNEL_CHECK, s, 1);
    prof_begin(MBP_KERNEL_VARIABLE, s);
    if (fixed)
      finalize_kernel<M><<<dim3(blocks_for(c.n, 32), NT), 256, 0, s>>>(
          c, st.lacc, static_cast<M*>(st.lv), static_cast<const M*>(st.lp), st.xh, st.active, inv_qscale);
    else
      launch_vn_any<M>(c, st, s);
    CKL("vn_kernel");
    prof_end(MBP_KERNEL_VARIABLE, s, 1);
    if (a.early_exit || t == a.max_iter) {
      if ((rc = stop_check(t, &left))) return rc;
    }
  }
#undef CKL
#undef CK
  return MBP_OK;
}

template <typename M>
int decode_t(const DevCode& c, DevState& st, const DecodeArgs& a, cudaStream_t s) {
  cudaError_t e;
#define CK(call, what) \
  if ((e = (call)) != cudaSuccess) return cuda_error(e, what)
#define CKL(what) CK(cudaGetLastError(), what)
  const int F = st.F, NT = st.n_tiles;
  const double l_max = a.l_max * Arith<M>::kToInternal;  // clip in the decoder's internal LLR unit
  // accumulation of eq. (2): fixed-point single pass (FP32 messages) or float two-pass
  int qbits = 0;
  {
    const double bound = double(c.max_col_deg > 0 ? c.max_col_deg : 1) * l_max;
    while (qbits < kMaxQBits && bound * std::ldexp(1.0, qbits + 1) < 2147483647.0) ++qbits;
  }
  const bool fixed_ok = sizeof(M) == 4 && st.lacc && qbits >= kMinQBits;
  if (a.accumulate == MBP_ACC_FIXED && !fixed_ok)
    return set_error(MBP_EUNSUPPORTED, "fixed-point accumulation needs FP32 messages and max node degree x l_max"
                                       " <= 2^%d", 31 - kMinQBits);
  const bool fixed = fixed_ok && a.accumulate == MBP_ACC_FIXED;
  const float qscale = float(std::ldexp(1.0, qbits)), inv_qscale = float(std::ldexp(1.0, -qbits));
  CK(cudaMemsetAsync(st.counters, 0, 4 * sizeof(int32_t), s), "clear counters");
  if (fixed) CK(cudaMemsetAsync(st.lacc, 0, size_t(NT) * c.n * kLanes * sizeof(int32_t), s), "clear accumulator");
  prof_begin(MBP_KERNEL_SETUP, s);
  if (a.y_bits) {
    frame_mag_kernel<<<blocks_for(F, 256), 256, 0, s>>>(a.qber, F, Arith<M>::kToInternal, st.llr_mag);
    CKL("frame_mag_kernel");
  }
  init_lp_kernel<M><<<dim3(blocks_for(c.n, 32), NT), 256, 0, s>>>(
      c, F, static_cast<const M*>(a.llr), a.y_bits, st.llr_mag, static_cast<M*>(st.lp), st.xh, st.counters,
      a.validate);
  CKL("init_lp_kernel");
  init_z_kernel<<<blocks_for(int64_t(NT) * c.m_tot, 256), 256, 0, s>>>(c, F, NT, a.z_bits, st.zt);
  CKL("init_z_kernel");
  init_tiles_kernel<<<blocks_for(NT, 256), 256, 0, s>>>(F, NT, c.u, st.active, st.fail);
  CKL("init_tiles_kernel");
  prof_end(MBP_KERNEL_SETUP, s, a.y_bits ? 4 : 3);
  int32_t host_ctr[4];
  if (a.validate) {
    CK(cudaMemcpyAsync(host_ctr, st.counters, sizeof host_ctr, cudaMemcpyDeviceToHost, s), "read validate flag");
    CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    if (host_ctr[1]) return set_error(MBP_EINVAL, "llr holds a non-finite value");
  }
  // schedule: resident (one cooperative launch, groups of tiles kept in L2) or streaming (kernels per iteration)
  const int G = (fixed || a.schedule != MBP_SCHED_RESIDENT) ? 0 : resident_group<M>(c, NT);
  if (a.schedule == MBP_SCHED_RESIDENT && G == 0)
    return set_error(MBP_EUNSUPPORTED, fixed ? "the resident schedule accumulates in floating point only"
                                             : "one tile of this code does not fit the resident schedule's L2 budget");
  if (G > 0 && a.schedule == MBP_SCHED_RESIDENT) {
    CK(cudaMemsetAsync(st.ctl, 0, sizeof(ResidentCtl), s), "clear resident control");
    prof_begin(MBP_KERNEL_PERSISTENT, s);
    CK(launch_resident_any<M>(c, st, a, G, l_max, s), "resident_kernel (cooperative launch)");
    prof_end(MBP_KERNEL_PERSISTENT, s, 1);
    ResidentCtl ctl_h;
    CK(cudaMemcpyAsync(&ctl_h, st.ctl, sizeof ctl_h, cudaMemcpyDeviceToHost, s), "read resident control");
    CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    if (ctl_h.error) return set_error(MBP_ETIMEOUT, "a grid barrier of the resident schedule timed out");
  } else {
    const int rc = stream_iterations<M>(c, st, a, fixed, l_max, qscale, inv_qscale, s);
    if (rc) return rc;
  }
  const int wn = (c.n + 31) >> 5;
  prof_begin(MBP_KERNEL_OUTPUT, s);
  out_bits_kernel<<<blocks_for(int64_t(F) * wn, 256), 256, 0, s>>>(c, F, st.xh, a.x_hat_bits);
  CKL("out_bits_kernel");
  if (a.soft_out) {
    soft_out_kernel<M><<<blocks_for(int64_t(F) * c.n, 256), 256, 0, s>>>(
        c, F, static_cast<const M*>(st.lv), static_cast<const M*>(st.lp), a.iters, static_cast<M*>(a.soft_out));
    CKL("soft_out_kernel");
  }
  prof_end(MBP_KERNEL_OUTPUT, s, a.soft_out ? 2 : 1);
#undef CKL
#undef CK
  return MBP_OK;
}

}  // namespace

cudaError_t launch_syndrome(const DevCode& c, const uint32_t* x_bits, int F, uint32_t* z_bits, cudaStream_t s) {
  int64_t off = 0;
  for (int l = 0; l < c.u; ++l) {
    const int wl = (c.m[l] + 31) >> 5;
    const int64_t work = int64_t(F) * wl;
    if (work > 0) syndrome_kernel<<<blocks_for(work, 128), 128, 0, s>>>(c, l, x_bits, F, z_bits + off);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    off += work;
  }
  return cudaSuccess;
}

cudaError_t launch_bsc_llr(const uint32_t* y_bits, const double* qber, int F, int n, int dtype, void* llr,
                           cudaStream_t s) {
  dim3 grid(blocks_for(n, 256), F);
  if (dtype == MBP_MSG_F64) bsc_llr_kernel<double><<<grid, 256, 0, s>>>(y_bits, qber, n, static_cast<double*>(llr));
  else bsc_llr_kernel<float><<<grid, 256, 0, s>>>(y_bits, qber, n, static_cast<float*>(llr));
  return cudaGetLastError();
}

static size_t msg_size(int msg_dtype) { return msg_dtype == MBP_MSG_F64 ? 8 : 4; }

constexpr int kRegions = 17;

static void layout(const DevCode& c, int F, int msg_dtype, bool host_io, size_t* offs, size_t* total) {
  const size_t NT = (size_t(F) + kLanes - 1) / kLanes;
  const size_t ms = msg_size(msg_dtype);
  const size_t wn = (size_t(c.n) + 31) / 32;
  size_t zw = 0;
  for (int l = 0; l < c.u; ++l) zw += (size_t(c.m[l]) + 31) / 32;
  const size_t sizes[] = {
      NT * size_t(c.s_tot) * kLanes * ms,  // c2v
      NT * size_t(c.n) * kLanes * ms,      // lv
      NT * size_t(c.n) * kLanes * ms,      // lp
      msg_dtype == MBP_MSG_F32 ? NT * size_t(c.n) * kLanes * 4 : 0,  // lacc
      NT * size_t(c.n),                    // xh
      NT * size_t(c.m_tot),                // zt
      NT * 4,                              // active
      NT * size_t(c.u) * 4,                // fail
      size_t(F) * 8,                       // llr_mag
      16,                                  // counters
      64,                                  // resident schedule control block
      host_io ? size_t(F) * wn * 4 : 0,    // io_y
      host_io ? size_t(F) * 8 : 0,         // io_qber
      host_io ? size_t(F) * zw * 4 : 0,    // io_z
      host_io ? size_t(F) * wn * 4 : 0,    // io_xhat
      host_io ? size_t(F) * 4 : 0,         // io_iters
      host_io ? size_t(F) : 0,             // io_success
  };
  size_t t = 0;
  for (int i = 0; i < kRegions; ++i) {
    offs[i] = t;
    t += align256(sizes[i]);
  }
  *total = t;
}

size_t workspace_bytes(const DevCode& c, int F, int msg_dtype, bool host_io) {
  size_t offs[kRegions], total;
  layout(c, F, msg_dtype, host_io, offs, &total);
  return total;
}

void carve_workspace(const DevCode& c, int F, int msg_dtype, bool host_io, void* base, DevState* st) {
  size_t o[kRegions], total;
  layout(c, F, msg_dtype, host_io, o, &total);
  char* b = static_cast<char*>(base);
  st->F = F;
  st->n_tiles = (F + kLanes - 1) / kLanes;
  st->c2v = b + o[0];
  st->lv = b + o[1];
  st->lp = b + o[2];
  st->lacc = msg_dtype == MBP_MSG_F32 ? reinterpret_cast<int32_t*>(b + o[3]) : nullptr;
  st->xh = reinterpret_cast<uint8_t*>(b + o[4]);
  st->zt = reinterpret_cast<uint8_t*>(b + o[5]);
  st->active = reinterpret_cast<uint32_t*>(b + o[6]);
  st->fail = reinterpret_cast<uint32_t*>(b + o[7]);
  st->llr_mag = reinterpret_cast<double*>(b + o[8]);
  st->counters = reinterpret_cast<int32_t*>(b + o[9]);
  st->ctl = b + o[10];
  st->io_y = host_io ? reinterpret_cast<uint32_t*>(b + o[11]) : nullptr;
  st->io_qber = host_io ? reinterpret_cast<double*>(b + o[12]) : nullptr;
  st->io_z = host_io ? reinterpret_cast<uint32_t*>(b + o[13]) : nullptr;
  st->io_xhat = host_io ? reinterpret_cast<uint32_t*>(b + o[14]) : nullptr;
  st->io_iters = host_io ? reinterpret_cast<int32_t*>(b + o[15]) : nullptr;
  st->io_success = host_io ? reinterpret_cast<uint8_t*>(b + o[16]) : nullptr;
}

int decode(const DevCode& c, DevState& st, int msg_dtype, const DecodeArgs& a, cudaStream_t s) {
  if (st.n_tiles > 65535) return set_error(MBP_EUNSUPPORTED, "F = %d exceeds %d frames per call", st.F, 65535 * kLanes);
  return msg_dtype == MBP_MSG_F64 ? decode_t<double>(c, st, a, s) : decode_t<float>(c, st, a, s);
}

// Device address of g_static_scratch on the current device. Host code only holds
// a stand-in for the array's name, so the address is looked up once per device
// (with that device current) and cached.
int static_scratch(void** ptr) {
  static std::mutex mu;
  static void* addr[kMaxDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return set_error(MBP_EUNSUPPORTED, "device %d beyond %d devices", dev, kMaxDevices);
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress of the static scratch");
    addr[dev] = p;
  }
  *ptr = addr[dev];
  return MBP_OK;
}

cudaError_t launch_export_c2v(const DevCode& c, const DevState& st, int msg_dtype, int frame, void* out,
                              cudaStream_t s) {
  if (c.e_tot == 0) return cudaSuccess;
  if (msg_dtype == MBP_MSG_F64)
    export_c2v_kernel<double><<<blocks_for(c.e_tot, 256), 256, 0, s>>>(c, static_cast<const double*>(st.c2v), frame,
                                                                         static_cast<double*>(out));
  else
    export_c2v_kernel<float><<<blocks_for(c.e_tot, 256), 256, 0, s>>>(c, static_cast<const float*>(st.c2v), frame,
                                                                        static_cast<float*>(out));
  return cudaGetLastError();
}

}  // namespace mbp
