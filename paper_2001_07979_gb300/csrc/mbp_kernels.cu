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
// With delta_r = 1 - tanh(|v_r| / 2) = 2 / (1 + e^{|v_r|}) the product becomes
// 1 - D_k with D_k = (+)_{r != k} delta_r under a (+) b = a + b - a b (the
// complement of a product), and 2 atanh(1 - D) = ln((2 - D) / D). Working with
// delta keeps full relative precision for reliable messages (delta ~ 2e^{-|v|})
// where tanh rounds to 1 in FP32. The exclusion r != k uses prefix and suffix
// (+)-combinations, never a division. Per edge this is two MUFU operations in,
// two out (exp + reciprocal, reciprocal + log).
#include <cmath>
#include <cstdio>
#include <mutex>

#include "mbp_internal.h"

// Fixed device scratch of mbp_decode_bsc_static: the decoder state of one call,
// for callers that must not allocate. Every GPU that loads this library holds
// these bytes until the process exits; every call shares them.
static __device__ __align__(256) unsigned char g_static_scratch[MBP_STATIC_SCRATCH_BYTES];

namespace mbp {
namespace {

constexpr uint32_t kFull = 0xffffffffu;

template <typename M>
struct Arith;

template <>
struct Arith<float> {
  // 1 - tanh(a/2) for a >= 0
  static __device__ __forceinline__ float delta(float a) { return __fdividef(2.0f, 1.0f + __expf(a)); }
  // complement product a (+) b = a + b - a b
  static __device__ __forceinline__ float oplus(float p, float d) { return fmaf(d, 1.0f - p, p); }
  // 2 atanh(1 - D) = ln((2 - D) / D) for 0 <= D <= 1 (a value within rounding of 0 may come out as -0 or
  // a tiny negative number; the caller ORs the message sign into the magnitude's sign bit)
  static __device__ __forceinline__ float mag(float D) { return __logf(__fdividef(2.0f - D, D)); }
};

template <>
struct Arith<double> {
  static __device__ __forceinline__ double delta(double a) { return 2.0 / (1.0 + exp(a)); }
  static __device__ __forceinline__ double oplus(double p, double d) { return fma(d, 1.0 - p, p); }
  static __device__ __forceinline__ double mag(double D) { return log((2.0 - D) / D); }
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
};

template <>
struct Bits<double> {
  static __device__ __forceinline__ uint32_t sign_word(double x) { return uint32_t(__double2hiint(x)); }
  static __device__ __forceinline__ double with_sign(double m, uint32_t sign) {
    return __hiloint2double(int(uint32_t(__double2hiint(m)) | sign), __double2loint(m));
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

__global__ void frame_mag_kernel(const double* __restrict__ qber, int F, double* __restrict__ mag) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f < F) {
    const double e = qber[f];
    mag[f] = log((1.0 - e) / e);
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
  const int j = r - c.row_first[l];
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

// One warp per slice (kSliceRows rows x kLanes frames), 8 slices per block.
// Every load of a row is issued before the first use: the slot columns, then
// the posterior gathers and the old messages, so a warp waits for two memory
// round trips per slice rather than two per edge.
//
// Signs travel in IEEE sign bits: the row's sign parity (with z_j) is the XOR
// of the V2C words' top bits, and each edge's own sign is kept in the sign bit
// of its delta, whose magnitude the (+) operations read through |.|.
//
// FIXED: also add each edge's change of message, q(C2V_new) - q(C2V_old) with
// q(x) = round(x * qscale), to the posterior accumulator lacc of its variable
// node (a 32-bit red.global.add in L2). Integer addition is associative, so
// the accumulated sum sum_e q(C2V_e) is exact and independent of the order of
// the atomics; finalize_kernel turns it into L_V. This removes the second read
// of every message that vn_kernel needs.
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
  const int lid = threadIdx.x & 31;
  const int q = lid >> 3, lane = lid & 7;
  const int r = s * kSliceRows + q;
  const int base = c.slice_base[s];
  const int deg = (c.slice_base[s + 1] - base) / kSliceRows;
  const int64_t node0 = int64_t(tile) * c.n * kLanes + lane;
  M* msg = c2v + (int64_t(tile) * c.s_tot + base + q) * kLanes + lane;  // edge k at msg[k * kSliceRows * kLanes]
  const M* gsrc = lsrc + node0;                                         // node i at gsrc[i * kLanes]
  const int* cols_p = c.slot_col + base + q;
  const bool row_ok = r < c.m_tot;
  const uint32_t zbyte = row_ok ? zt[int64_t(tile) * c.m_tot + r] : 0u;

  int col[DMAX];
#pragma unroll
  for (int k = 0; k < DMAX; ++k) col[k] = k < deg ? __ldg(cols_p + k * kSliceRows) : -1;
  M v[DMAX];
#pragma unroll
  for (int k = 0; k < DMAX; ++k) v[k] = col[k] >= 0 ? __ldg(gsrc + col[k] * kLanes) : M(0);
  [[maybe_unused]] M old[FIXED ? DMAX : 1];
  if (!first_iter) {
#pragma unroll
    for (int k = 0; k < DMAX; ++k) {
      const M o = col[k] >= 0 ? __ldcs(msg + k * kSliceRows * kLanes) : M(0);
      if constexpr (FIXED) old[k] = o;
      v[k] -= o;
    }
  } else if constexpr (FIXED) {
#pragma unroll
    for (int k = 0; k < DMAX; ++k) old[k] = M(0);
  }
  uint32_t par = ((zbyte >> lane) & 1u) << 31;
  M pre[DMAX];
  M P = M(0);
#pragma unroll
  for (int k = 0; k < DMAX; ++k) {
    const uint32_t sx = Bits<M>::sign_word(v[k]);
    par ^= sx;
    const M d = col[k] >= 0 ? Arith<M>::delta(fmin(fabs(v[k]), l_max)) : M(0);
    v[k] = Bits<M>::with_sign(d, sx & kSign);
    pre[k] = P;
    P = Arith<M>::oplus(P, d);
  }
  if (!row_ok || !((act >> lane) & 1u)) return;
  M S = M(0);
#pragma unroll
  for (int k = DMAX - 1; k >= 0; --k) {
    if (col[k] >= 0) {
      const M D = Arith<M>::oplus(pre[k], S);
      const M mag = fmin(Arith<M>::mag(D), l_max);
      const M nv = Bits<M>::with_sign(mag, (par ^ Bits<M>::sign_word(v[k])) & kSign);
      __stcs(msg + k * kSliceRows * kLanes, nv);
      if constexpr (FIXED) {
        const int32_t dq = __float2int_rn(float(nv) * qscale) - __float2int_rn(float(old[k]) * qscale);
        if (dq != 0) atomicAdd(lacc + node0 + col[k] * kLanes, dq);
      }
    }
    S = Arith<M>::oplus(S, fabs(v[k]));
  }
}

// ------------------------------------------------------------- eq. (2)

// Block: 32 variable nodes x 8 lanes. Sums in stacked-row order; the slot
// indices of a node are loaded before the message gathers, so the gathers of
// one node are in flight together. DMAX bounds the node degree (all matrices).
template <typename M, int DMAX>
__global__ void __launch_bounds__(256) vn_kernel(const DevCode c, const M* __restrict__ c2v, M* __restrict__ lv,
                                                 const M* __restrict__ lp, uint8_t* __restrict__ xh,
                                                 const uint32_t* __restrict__ active) {
  const int tile = blockIdx.y;
  const uint32_t act = active[tile];
  if (act == 0) return;
  const int lane = threadIdx.x & 7;
  const int col = blockIdx.x * 32 + (threadIdx.x >> 3);
  const bool ok = col < c.n;
  const int64_t at = (int64_t(tile) * c.n + col) * kLanes + lane;
  const M* msg = c2v + int64_t(tile) * c.s_tot * kLanes + lane;
  M sum = M(0);
  if (ok) {
    const int a0 = c.col_ptr[col];
    const int d = c.col_ptr[col + 1] - a0;
    int slot[DMAX];
#pragma unroll
    for (int k = 0; k < DMAX; ++k) slot[k] = k < d ? __ldg(c.col_slot + a0 + k) : -1;
    M g[DMAX];
#pragma unroll
    for (int k = 0; k < DMAX; ++k) g[k] = slot[k] >= 0 ? __ldcs(msg + int64_t(slot[k]) * kLanes) : M(0);
    sum = lp[at];
#pragma unroll
    for (int k = 0; k < DMAX; ++k)
      if (slot[k] >= 0) sum += g[k];
    if ((act >> lane) & 1u) lv[at] = sum;
  }
  const uint32_t b = __ballot_sync(kFull, ok && sum < M(0));
  if (ok && lane == 0) {
    const uint32_t nb = (b >> (threadIdx.x & 24)) & 0xffu;
    uint8_t* px = xh + int64_t(tile) * c.n + col;
    *px = uint8_t((*px & ~act) | (nb & act));
  }
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

// One thread per (tile, stacked row): lanes whose hard decision breaks the row.
// The row's columns come from the slot layout and are all loaded before the
// decision bytes are gathered.
template <int DMAX>
__global__ void __launch_bounds__(256) syn_kernel(const DevCode c, const uint8_t* __restrict__ xh,
                                                  const uint8_t* __restrict__ zt,
                                                  const uint32_t* __restrict__ active, uint32_t* __restrict__ fail) {
  const int tile = blockIdx.y;
  const uint32_t act = active[tile];
  if (act == 0) return;
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
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
      if (col[k] >= 0) p ^= x[col[k]];
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

// One thread per tile: retire lanes that satisfied every syndrome (or hit max_iter).
__global__ void update_kernel(int F, int n_tiles, int u, int t, int max_iter, int early_exit,
                              uint32_t* __restrict__ active, uint32_t* __restrict__ fail,
                              int32_t* __restrict__ iters, uint8_t* __restrict__ success,
                              uint8_t* __restrict__ synd_ok, int32_t* __restrict__ counters) {
  const int tile = blockIdx.x * blockDim.x + threadIdx.x;
  if (tile >= n_tiles) return;
  uint32_t act = active[tile];
  if (act == 0) return;
  uint32_t anyfail = 0;
  for (int l = 0; l < u; ++l) anyfail |= fail[tile * u + l];
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
      for (int l = 0; l < u; ++l) synd_ok[int64_t(f) * u + l] = uint8_t(!((fail[tile * u + l] >> lane) & 1u));
  }
  act &= ~done;
  active[tile] = act;
  for (int l = 0; l < u; ++l) fail[tile * u + l] = 0;
  if (act) atomicAdd(&counters[0], 1);
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
  out[idx] = iters[f] == 0 ? lp[at] : lv[at];
}

template <typename M>
__global__ void export_c2v_kernel(const DevCode c, const M* __restrict__ c2v, int frame, M* __restrict__ out) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= c.e_tot) return;
  const int tile = frame / kLanes, lane = frame % kLanes;
  out[e] = c2v[(int64_t(tile) * c.s_tot + c.edge_slot[e]) * kLanes + lane];
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
  if (c.max_row_deg <= 8) launch_cn<M, 8, FIXED>(c, st, first_iter, l_max, qscale, s);
  else if (c.max_row_deg <= 16) launch_cn<M, 16, FIXED>(c, st, first_iter, l_max, qscale, s);
  else if (c.max_row_deg <= 32) launch_cn<M, 32, FIXED>(c, st, first_iter, l_max, qscale, s);
  else launch_cn<M, 64, FIXED>(c, st, first_iter, l_max, qscale, s);
}

template <typename M, int DMAX>
void launch_vn(const DevCode& c, const DevState& st, cudaStream_t s) {
  vn_kernel<M, DMAX><<<dim3(blocks_for(c.n, 32), st.n_tiles), 256, 0, s>>>(
      c, static_cast<const M*>(st.c2v), static_cast<M*>(st.lv), static_cast<const M*>(st.lp), st.xh, st.active);
}

template <typename M>
void launch_vn_any(const DevCode& c, const DevState& st, cudaStream_t s) {
  if (c.max_col_deg <= 8) launch_vn<M, 8>(c, st, s);
  else if (c.max_col_deg <= 16) launch_vn<M, 16>(c, st, s);
  else if (c.max_col_deg <= 32) launch_vn<M, 32>(c, st, s);
  else launch_vn<M, kMaxColDeg>(c, st, s);
}

template <typename M>
int decode_t(const DevCode& c, DevState& st, const DecodeArgs& a, cudaStream_t s) {
  cudaError_t e;
#define CK(call, what) \
  if ((e = (call)) != cudaSuccess) return cuda_error(e, what)
#define CKL(what) CK(cudaGetLastError(), what)
  const int F = st.F, NT = st.n_tiles;
  // accumulation of eq. (2): fixed-point single pass (FP32 messages) or float two-pass
  int qbits = 0;
  {
    const double bound = double(c.max_col_deg > 0 ? c.max_col_deg : 1) * a.l_max;
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
    frame_mag_kernel<<<blocks_for(F, 256), 256, 0, s>>>(a.qber, F, st.llr_mag);
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
  const dim3 syn_grid(blocks_for(c.m_tot, 256), NT);
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
      if (fixed) launch_cn_any<M, true>(c, st, t == 1, a.l_max, qscale, s);
      else launch_cn_any<M, false>(c, st, t == 1, a.l_max, qscale, s);
    } else {
      launch_cn_any<M, false>(c, st, t == 1, a.l_max, qscale, s);
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

constexpr int kRegions = 16;

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
  st->io_y = host_io ? reinterpret_cast<uint32_t*>(b + o[10]) : nullptr;
  st->io_qber = host_io ? reinterpret_cast<double*>(b + o[11]) : nullptr;
  st->io_z = host_io ? reinterpret_cast<uint32_t*>(b + o[12]) : nullptr;
  st->io_xhat = host_io ? reinterpret_cast<uint32_t*>(b + o[13]) : nullptr;
  st->io_iters = host_io ? reinterpret_cast<int32_t*>(b + o[14]) : nullptr;
  st->io_success = host_io ? reinterpret_cast<uint8_t*>(b + o[15]) : nullptr;
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
