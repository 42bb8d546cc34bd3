// Streaming kernels of tile pairs (FP32, FP16 and BF16 messages; FP32
// arithmetic). Tiles 2q and 2q + 1 store the messages of an edge together
// (msg_at): 2-byte messages in one 128-byte line, one 32-bit word per lane;
// 4-byte messages in two adjacent 128-byte lines. One warp takes the pair, each
// lane the same frame position of both tiles, so every message access of the
// warp covers the pair's whole unit (128 or 256 contiguous bytes) and the row's
// columns and slots are loaded once for 64 frames. Per frame the arithmetic is
// that of cn_row / cn_row_signs / vn_class_nodes, in the same order, so a
// frame's messages and posteriors do not depend on the kernel that produced
// them.
//
// A tile whose frames have all retired (or the missing partner of an odd tile
// count) is neither read nor written; in a pair with one live tile, a lane
// writes only its live frames' messages.
#pragma once

#include <type_traits>

#include "mbp_device.cuh"

namespace mbp {
namespace dev {

// Per storage type: T, the element type a lane addresses (one per slot and lane
// for 2-byte pairs); kSlot, the T elements from one slot of a pair to the next;
// W, what a lane loads for both tiles' message of an edge.
template <typename S>
struct Pair;

template <>
struct Pair<__half> {
  using T = __half2;
  using W = uint32_t;  // low half: tile 2q
  static constexpr int kSlot = kLanes;
  static __device__ __forceinline__ T narrow(float a, float b) { return __floats2half2_rn(a, b); }
};

template <>
struct Pair<__nv_bfloat16> {
  using T = __nv_bfloat162;
  using W = uint32_t;
  static constexpr int kSlot = kLanes;
  static __device__ __forceinline__ T narrow(float a, float b) { return __floats2bfloat162_rn(a, b); }
};

template <>
struct Pair<float> {
  using T = float;  // tile 2q at the lane's element, tile 2q + 1 one line (kLanes elements) later
  using W = float2;
  static constexpr int kSlot = 2 * kLanes;
};

// Both tiles' message of an edge.
template <typename S>
__device__ __forceinline__ typename Pair<S>::W ld_pair(const typename Pair<S>::T* p) {
  if constexpr (std::is_same<S, float>::value) return make_float2(__ldcs(p), __ldcs(p + kLanes));
  else return __ldcs(reinterpret_cast<const unsigned int*>(p));
}

// s0 += message of tile 2q, s1 += message of tile 2q + 1, and v0 -= ..., v1 -= ...
// as FP32 operations with one rounding each. For 2-byte messages sm_100's
// mixed-precision add / fma take the 16-bit operand as is (its widening to FP32
// is exact), in one instruction.
template <typename S>
__device__ __forceinline__ void add_pair(float& s0, float& s1, typename Pair<S>::W w) {
  if constexpr (std::is_same<S, float>::value) {
    s0 += w.x;
    s1 += w.y;
  } else if constexpr (std::is_same<S, __half>::value) {
    asm("{.reg .b16 l, h; mov.b32 {l, h}, %2; add.rn.f32.f16 %0, l, %0; add.rn.f32.f16 %1, h, %1;}"
        : "+f"(s0), "+f"(s1) : "r"(w));
  } else {
    asm("{.reg .b16 l, h; mov.b32 {l, h}, %2; add.rn.f32.bf16 %0, l, %0; add.rn.f32.bf16 %1, h, %1;}"
        : "+f"(s0), "+f"(s1) : "r"(w));
  }
}

template <typename S>
__device__ __forceinline__ void sub_pair(float& v0, float& v1, typename Pair<S>::W w) {
  if constexpr (std::is_same<S, float>::value) {
    v0 -= w.x;
    v1 -= w.y;
  } else if constexpr (std::is_same<S, __half>::value) {
    const unsigned short m1 = 0xBC00u;  // -1 in FP16
    asm("{.reg .b16 l, h; mov.b32 {l, h}, %2; fma.rn.f32.f16 %0, l, %3, %0; fma.rn.f32.f16 %1, h, %3, %1;}"
        : "+f"(v0), "+f"(v1) : "r"(w), "h"(m1));
  } else {
    const unsigned short m1 = 0xBF80u;  // -1 in BF16
    asm("{.reg .b16 l, h; mov.b32 {l, h}, %2; fma.rn.f32.bf16 %0, l, %3, %0; fma.rn.f32.bf16 %1, h, %3, %1;}"
        : "+f"(v0), "+f"(v1) : "r"(w), "h"(m1));
  }
}

// Store a lane's two messages; a retired frame keeps its stored message.
template <typename S>
__device__ __forceinline__ void st_pair(typename Pair<S>::T* p, float a, float b, bool s0, bool s1) {
  if constexpr (std::is_same<S, float>::value) {
    if (s0) __stcs(p, a);
    if (s1) __stcs(p + kLanes, b);
  } else if (s0 && s1) {
    __stcs(p, Pair<S>::narrow(a, b));
  } else {
    S* h = reinterpret_cast<S*>(p);
    if (s0) __stcs(h, Store<S>::narrow(a));
    if (s1) __stcs(h + 1, Store<S>::narrow(b));
  }
}

// Everything a warp needs about the two tiles of pair q for the lane's frames.
struct PairTiles {
  int t0, t1;        // tile indices (t1 may be past the last tile)
  uint32_t a0, a1;   // lanes still decoding (0 for a missing tile)
  bool s0, s1;       // this lane's frame is still decoding, per tile
};

__device__ __forceinline__ PairTiles pair_tiles(int q, int n_tiles, const uint32_t* __restrict__ active) {
  const int lane = threadIdx.x & 31;
  PairTiles p;
  p.t0 = 2 * q;
  p.t1 = 2 * q + 1;
  p.a0 = active[p.t0];
  p.a1 = p.t1 < n_tiles ? active[p.t1] : 0u;
  p.s0 = (p.a0 >> lane) & 1u;
  p.s1 = (p.a1 >> lane) & 1u;
  return p;
}

// Rows of more than 16 edges keep only the prefix folds before even edges (the
// one before an odd edge k is formed again from the one before k - 1 and delta
// k - 1: the same operation on the same values), so that the two tiles' rows
// fit three blocks per SM.
template <int D>
constexpr bool kHalfPrefix = D > 16;
template <int D>
constexpr int kPrefixLen = kHalfPrefix<D> ? (D + 1) / 2 : D;

// The (+) fold of edges 0 .. k - 1; v[k - 1] holds delta k - 1 (its sign bit
// carries the V2C's sign).
template <int D>
__device__ __forceinline__ float pair_prefix(const float (&pre)[kPrefixLen<D>], const float (&v)[D], int k) {
  if constexpr (kHalfPrefix<D>) {
    if (k & 1) return Arith<float>::oplus(pre[k >> 1], fabsf(v[k - 1]));
    return pre[k >> 1];
  } else {
    return pre[k];
  }
}

// The prefix pass of eq. (6) for one frame: the row's sign parity into par,
// each V2C replaced by its delta carrying the V2C's sign bit, pre the (+)
// folds of edges 0 .. k - 1 (padding edges fold as 0).
template <int D, bool CHECKED>
__device__ __forceinline__ void cn_pair_fold(int deg, float (&v)[D], float (&pre)[kPrefixLen<D>], uint32_t& par,
                                             float l_max, float d_lmax) {
  using A = Arith<float>;
  using B = Bits<float>;
  float P = 0.f;
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const uint32_t x = B::sign_word(v[k]);
    par ^= x;
    float d = A::clipped_delta(v[k], l_max, d_lmax);
    if constexpr (CHECKED) d = k < deg ? d : 0.f;
    v[k] = B::with_sign(d, x & kSign);
    if (!kHalfPrefix<D> || (k & 1) == 0) pre[kHalfPrefix<D> ? k >> 1 : k] = P;
    P = A::oplus(P, d);
  }
}

// Eq. (6) for one row of both tiles: V2C = clip(L_V - C2V) (L_V alone in the
// first iteration of general inputs), prefix / suffix (+) folds per frame,
// output magnitude and sign as in cn_row. g0 / g1 are the tiles' posteriors at
// this lane; h0 / h1 say whether a tile has live frames (warp-uniform).
// rp != NULL (iteration 2 after a row-form iteration 1): the old messages are
// rebuilt from the tiles' row magnitudes rp->m (this lane) and sign words rp->s
// and Bob's sign words rp->y (row_msg), as the stored ones would read.
struct PairRows {
  float m0, m1;
  uint32_t s0, s1;
  const uint32_t* y0;
  const uint32_t* y1;
};

template <typename S, int D, bool CHECKED>
__device__ __forceinline__ void cn_pair_row(int deg, const int* __restrict__ cols, const float* __restrict__ g0,
                                            const float* __restrict__ g1, bool h0, bool h1,
                                            typename Pair<S>::T* __restrict__ msg, int first_iter, uint32_t par0,
                                            uint32_t par1, bool s0, bool s1, float l_max, float d_lmax,
                                            const PairRows* rp) {
  using A = Arith<float>;
  using B = Bits<float>;
  int col[D];
#pragma unroll
  for (int k = 0; k < D; ++k) col[k] = (!CHECKED || k < deg) ? __ldg(cols + k) : 0;
  float v0[D], v1[D];
#pragma unroll
  for (int k = 0; k < D; ++k) {
    const bool on = !CHECKED || k < deg;
    v0[k] = on && h0 ? __ldg(g0 + col[k] * kLanes) : 0.f;
    v1[k] = on && h1 ? __ldg(g1 + col[k] * kLanes) : 0.f;
  }
  if (rp) {
    // lane k fetches edge k's sign words (two gathers for the row); one bit transpose per tile gives lane f
    // every edge's bit of frame f (bit k: edge k). The old message of edge k is the row's magnitude with the
    // sign bit lane of rs ^ y_k (row_msg); v - old is formed as v + (-old), which rounds the same, with -old's
    // sign bit taken from bit k of ~(R) (R = the transposed word xor the row's own sign bit of this frame).
    const int lane = threadIdx.x & 31;
    const int mycol = lane < deg ? __ldg(cols + lane) : 0;
    const uint32_t my0 = lane < deg && h0 ? __ldg(rp->y0 + mycol) : 0u;
    const uint32_t my1 = lane < deg && h1 ? __ldg(rp->y1 + mycol) : 0u;
    const uint32_t n0 = ~(warp_transpose32(my0) ^ (0u - ((rp->s0 >> lane) & 1u)));
    const uint32_t n1 = ~(warp_transpose32(my1) ^ (0u - ((rp->s1 >> lane) & 1u)));
    const uint32_t m0 = __float_as_uint(rp->m0) & ~kSign, m1 = __float_as_uint(rp->m1) & ~kSign;
#pragma unroll
    for (int k = 0; k < D; ++k)
      if (!CHECKED || k < deg) {
        static_assert(D <= 32, "one transposed bit per edge");
        if (h0) v0[k] += __uint_as_float(m0 | ((n0 << (31 - k)) & kSign));
        if (h1) v1[k] += __uint_as_float(m1 | ((n1 << (31 - k)) & kSign));
      }
  } else if (!first_iter) {
#pragma unroll
    for (int k = 0; k < D; ++k)
      if (!CHECKED || k < deg) sub_pair<S>(v0[k], v1[k], ld_pair<S>(msg + k * Pair<S>::kSlot));
  }
  if (!s0 && !s1) return;
  // tile 0, then tile 1, sharing the prefix array; tile 0's outputs replace its deltas in v0
  float pre[kPrefixLen<D>];
  cn_pair_fold<D, CHECKED>(deg, v0, pre, par0, l_max, d_lmax);
  float q = 0.f;
#pragma unroll
  for (int k = D - 1; k >= 0; --k) {
    const float d = v0[k];
    if (!CHECKED || k < deg)
      v0[k] = B::copy_sign(A::clipped_mag(A::oplus(pair_prefix<D>(pre, v0, k), q), l_max), par0 ^ B::sign_word(d));
    q = A::oplus(q, fabsf(d));
  }
  cn_pair_fold<D, CHECKED>(deg, v1, pre, par1, l_max, d_lmax);
  q = 0.f;
#pragma unroll
  for (int k = D - 1; k >= 0; --k) {
    if (!CHECKED || k < deg) {
      const float m1 = A::clipped_mag(A::oplus(pair_prefix<D>(pre, v1, k), q), l_max);
      st_pair<S>(msg + k * Pair<S>::kSlot, v0[k], B::copy_sign(m1, par1 ^ B::sign_word(v1[k])), s0, s1);
    }
    q = A::oplus(q, fabsf(v1[k]));
  }
}

// The first iteration of BSC inputs for one row of both tiles (cn_row_signs per
// frame): Bob's bits of the row as one mask per tile, one output magnitude per
// row and frame.
template <typename S, int D, bool CHECKED>
__device__ __forceinline__ void cn_pair_row_signs(int deg, const int* __restrict__ cols,
                                                  const uint32_t* __restrict__ y0, const uint32_t* __restrict__ y1,
                                                  bool h0, bool h1, float ym0, float ym1,
                                                  typename Pair<S>::T* __restrict__ msg, uint32_t par0,
                                                  uint32_t par1, bool s0, bool s1, float l_max, float d_lmax) {
  static_assert(D <= 32, "one bit per edge");
  const int lane = threadIdx.x & 31;
  uint32_t b0 = 0, b1 = 0;
#pragma unroll
  for (int k = 0; k < D; ++k)
    if (!CHECKED || k < deg) {
      const int col = __ldg(cols + k);
      if (h0) b0 |= ((__ldg(y0 + col) >> lane) & 1u) << k;
      if (h1) b1 |= ((__ldg(y1 + col) >> lane) & 1u) << k;
    }
  if (!s0 && !s1) return;
  par0 ^= uint32_t(__popc(b0) & 1) << 31;
  par1 ^= uint32_t(__popc(b1) & 1) << 31;
  const float m0 = cn_first_mag<float, D, CHECKED>(deg, ym0, l_max, d_lmax);
  const float m1 = cn_first_mag<float, D, CHECKED>(deg, ym1, l_max, d_lmax);
#pragma unroll
  for (int k = 0; k < D; ++k)
    if (!CHECKED || k < deg)
      st_pair<S>(msg + k * Pair<S>::kSlot, Bits<float>::copy_sign(m0, par0 ^ (((b0 >> k) & 1u) << 31)),
                 Bits<float>::copy_sign(m1, par1 ^ (((b1 >> k) & 1u) << 31)), s0, s1);
}

// Resident blocks of 256 threads per SM for the pair check kernel: two frames
// per lane double the row's registers.
constexpr int cn_pair_min_blocks(int dmax) { return dmax <= 14 ? 4 : 3; }

// One warp per (tile pair, check row): 8 rows per block, pair = blockIdx.y,
// rows p0 .. p1 - 1. RIN: iteration 2 after a row-form iteration 1 (fmag, rsgn;
// the kernel clears the row-form flag counters[2]).
template <typename S, int DMAX, bool RIN>
__global__ void __launch_bounds__(256, cn_pair_min_blocks(DMAX))
    cn_pair_kernel(const DevCode c, int p0, int p1, int first_iter, S* __restrict__ c2v,
                   const float* __restrict__ lsrc, const uint32_t* __restrict__ zt,
                   const uint32_t* __restrict__ active, int n_tiles, float l_max, const float* __restrict__ fmag,
                   const uint32_t* __restrict__ rsgn, const uint32_t* __restrict__ yt,
                   int32_t* __restrict__ counters) {
  if (RIN && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) counters[2] = 0;
  const PairTiles t = pair_tiles(blockIdx.y, n_tiles, active);
  if ((t.a0 | t.a1) == 0) return;
  const int p = p0 + blockIdx.x * 8 + (threadIdx.x >> 5);
  if (p >= p1) return;
  const int lane = threadIdx.x & 31;
  const int base = c.slice_base[p];
  const int deg = c.slice_base[p + 1] - base;
  const bool h0 = t.a0 != 0, h1 = t.a1 != 0;
  const uint32_t par0 = h0 ? ((zt[int64_t(t.t0) * c.m_tot + p] >> lane) & 1u) << 31 : 0u;
  const uint32_t par1 = h1 ? ((zt[int64_t(t.t1) * c.m_tot + p] >> lane) & 1u) << 31 : 0u;
  using T = typename Pair<S>::T;
  T* msg = reinterpret_cast<T*>(c2v) + (int64_t(blockIdx.y) * c.s_tot + base) * Pair<S>::kSlot + lane;
  const float* g0 = lsrc + int64_t(t.t0) * c.n * kLanes + lane;
  const float* g1 = h1 ? lsrc + int64_t(t.t1) * c.n * kLanes + lane : g0;
  const int* cols = c.slot_col + base;
  const float inv = Arith<float>::delta(l_max);  // d_lmax
  PairRows rows;
  if constexpr (RIN) {
    const int64_t r0 = int64_t(p) * n_tiles + t.t0, r1 = int64_t(p) * n_tiles + t.t1;
    rows.m0 = h0 ? __ldg(fmag + (int64_t(t.t0) * kMaxRowDeg + deg - 1) * kLanes + lane) : 0.f;
    rows.m1 = h1 ? __ldg(fmag + (int64_t(t.t1) * kMaxRowDeg + deg - 1) * kLanes + lane) : 0.f;
    rows.s0 = h0 ? __ldg(rsgn + r0) : 0u;
    rows.s1 = h1 ? __ldg(rsgn + r1) : 0u;
    rows.y0 = yt + int64_t(t.t0) * c.n;
    rows.y1 = h1 ? yt + int64_t(t.t1) * c.n : rows.y0;
  }
  const PairRows* rp = RIN ? &rows : nullptr;
  if (deg == DMAX)
    cn_pair_row<S, DMAX, false>(deg, cols, g0, g1, h0, h1, msg, first_iter, par0, par1, t.s0, t.s1, l_max, inv, rp);
  else if (DMAX > 1 && deg == DMAX - 1)
    cn_pair_row<S, (DMAX > 1 ? DMAX - 1 : 1), false>(deg, cols, g0, g1, h0, h1, msg, first_iter, par0, par1, t.s0,
                                                     t.s1, l_max, inv, rp);
  else
    cn_pair_row<S, DMAX, true>(deg, cols, g0, g1, h0, h1, msg, first_iter, par0, par1, t.s0, t.s1, l_max, inv, rp);
}

// Iteration 1 of BSC inputs for a tile pair.
template <typename S, int DMAX>
__global__ void __launch_bounds__(256) cn_first_pair_kernel(const DevCode c, int p0, int p1, S* __restrict__ c2v,
                                                            const uint32_t* __restrict__ yt,
                                                            const float* __restrict__ ymag,
                                                            const uint32_t* __restrict__ zt,
                                                            const uint32_t* __restrict__ active, int n_tiles,
                                                            float l_max) {
  const PairTiles t = pair_tiles(blockIdx.y, n_tiles, active);
  if ((t.a0 | t.a1) == 0) return;
  const int p = p0 + blockIdx.x * 8 + (threadIdx.x >> 5);
  if (p >= p1) return;
  const int lane = threadIdx.x & 31;
  const int base = c.slice_base[p];
  const int deg = c.slice_base[p + 1] - base;
  const bool h0 = t.a0 != 0, h1 = t.a1 != 0;
  const uint32_t par0 = h0 ? ((zt[int64_t(t.t0) * c.m_tot + p] >> lane) & 1u) << 31 : 0u;
  const uint32_t par1 = h1 ? ((zt[int64_t(t.t1) * c.m_tot + p] >> lane) & 1u) << 31 : 0u;
  const float ym0 = h0 ? __ldg(ymag + t.t0 * kLanes + lane) : 0.f;
  const float ym1 = h1 ? __ldg(ymag + t.t1 * kLanes + lane) : 0.f;
  using T = typename Pair<S>::T;
  T* msg = reinterpret_cast<T*>(c2v) + (int64_t(blockIdx.y) * c.s_tot + base) * Pair<S>::kSlot + lane;
  const uint32_t* y0 = yt + int64_t(t.t0) * c.n;
  const uint32_t* y1 = h1 ? yt + int64_t(t.t1) * c.n : y0;
  const int* cols = c.slot_col + base;
  const float inv = Arith<float>::delta(l_max);  // d_lmax
  if (deg == DMAX)
    cn_pair_row_signs<S, DMAX, false>(deg, cols, y0, y1, h0, h1, ym0, ym1, msg, par0, par1, t.s0, t.s1, l_max, inv);
  else
    cn_pair_row_signs<S, DMAX, true>(deg, cols, y0, y1, h0, h1, ym0, ym1, msg, par0, par1, t.s0, t.s1, l_max, inv);
}

// Eq. (2) and the hard decision for N nodes of one degree class (degree d <= D)
// of both tiles: every gather covers both tiles' C2V of the edge (one 32-bit
// word per lane, or two adjacent lines for FP32), the sums run in stacked-row
// order as in vn_class_nodes.
template <typename S, int D, int N>
__global__ void __launch_bounds__(256) vn_class_pair_kernel(const DevCode c, int cls, const S* __restrict__ c2v,
                                                            float* __restrict__ lv, const float* __restrict__ lp,
                                                            const uint32_t* __restrict__ yt,
                                                            const float* __restrict__ ymag, uint32_t* __restrict__ xh,
                                                            const uint32_t* __restrict__ active, int n_tiles) {
  static_assert(D <= 32, "classes of up to 32 edges");
  const PairTiles t = pair_tiles(blockIdx.y, n_tiles, active);
  if ((t.a0 | t.a1) == 0) return;
  const int first = c.vclass_first[cls], count = c.vclass_first[cls + 1] - first;
  const int qq = (blockIdx.x * 8 + (threadIdx.x >> 5)) * N;
  if (qq >= count) return;
  const int lane = threadIdx.x & 31;
  const int d = c.vclass_deg[cls];
  const int cnt = min(N, count - qq);
  const bool h0 = t.a0 != 0, h1 = t.a1 != 0;
  using T = typename Pair<S>::T;
  const T* msg = reinterpret_cast<const T*>(c2v) + int64_t(blockIdx.y) * c.s_tot * Pair<S>::kSlot + lane;
  const int32_t* slots0 = c.vslot + c.vclass_toff[cls] + int64_t(qq) * d;
  int col[N];
#pragma unroll
  for (int j = 0; j < N; ++j) col[j] = j < cnt ? __ldg(c.vnode + first + qq + j) : 0;
  const int64_t n0 = int64_t(t.t0) * c.n, n1 = int64_t(t.t1) * c.n;
  typename Pair<S>::W g[N][D];
#pragma unroll
  for (int j = 0; j < N; ++j)
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const bool on = j < cnt && k < d;
      const int slot = on ? __ldg(slots0 + j * d + k) : 0;
      g[j][k] = on ? ld_pair<S>(msg + int64_t(slot) * Pair<S>::kSlot) : typename Pair<S>::W{};
    }
  const float ym0 = yt && h0 ? __ldg(ymag + t.t0 * kLanes + lane) : 0.f;
  const float ym1 = yt && h1 ? __ldg(ymag + t.t1 * kLanes + lane) : 0.f;
#pragma unroll
  for (int j = 0; j < N; ++j) {
    if (j >= cnt) break;
    const int v = col[j];
    float sum0 = 0.f, sum1 = 0.f;
    if (yt) {
      if (h0) sum0 = ((__ldg(yt + n0 + v) >> lane) & 1u) ? -ym0 : ym0;
      if (h1) sum1 = ((__ldg(yt + n1 + v) >> lane) & 1u) ? -ym1 : ym1;
    } else {
      if (h0) sum0 = __ldg(lp + (n0 + v) * kLanes + lane);
      if (h1) sum1 = __ldg(lp + (n1 + v) * kLanes + lane);
    }
#pragma unroll
    for (int k = 0; k < D; ++k)
      if (k < d) add_pair<S>(sum0, sum1, g[j][k]);
    if (h0) {
      if (t.s0) lv[(n0 + v) * kLanes + lane] = sum0;
      const uint32_t hard = __ballot_sync(kFull, sum0 < 0.f);
      if (lane == 0) {
        uint32_t* px = xh + int64_t(v) * n_tiles + t.t0;
        *px = t.a0 == kFull ? hard : (__ldg(px) & ~t.a0) | (hard & t.a0);
      }
    }
    if (h1) {
      if (t.s1) lv[(n1 + v) * kLanes + lane] = sum1;
      const uint32_t hard = __ballot_sync(kFull, sum1 < 0.f);
      if (lane == 1) {
        uint32_t* px = xh + int64_t(v) * n_tiles + t.t1;
        *px = t.a1 == kFull ? hard : (__ldg(px) & ~t.a1) | (hard & t.a1);
      }
    }
  }
}

// vn_rows_kernel for a tile pair (the row-form magnitudes of 2-byte messages are
// stored rounded to the message type): each lane sums its frame in both tiles.
template <int D>
__global__ void __launch_bounds__(256) vn_rows_pair_kernel(const DevCode c, int cls, float* __restrict__ lv,
                                                           const uint32_t* __restrict__ yt,
                                                           const float* __restrict__ ymag, uint32_t* __restrict__ xh,
                                                           const uint32_t* __restrict__ active, int n_tiles,
                                                           const float* __restrict__ fmag,
                                                           const uint32_t* __restrict__ rsgn) {
  __shared__ float fm[2][kMaxRowDeg * kLanes];
  const PairTiles t = pair_tiles(blockIdx.y, n_tiles, active);
  if ((t.a0 | t.a1) == 0) return;
  const bool h0 = t.a0 != 0, h1 = t.a1 != 0;
  for (int i = threadIdx.x; i < c.max_row_deg * kLanes; i += blockDim.x) {
    fm[0][i] = h0 ? fmag[int64_t(t.t0) * kMaxRowDeg * kLanes + i] : 0.f;
    fm[1][i] = h1 ? fmag[int64_t(t.t1) * kMaxRowDeg * kLanes + i] : 0.f;
  }
  __syncthreads();
  const int d = c.vclass_deg[cls], N = kLanes / d;
  const int first = c.vclass_first[cls], count = c.vclass_first[cls + 1] - first;
  const int q0 = (blockIdx.x * 8 + (threadIdx.x >> 5)) * N;
  if (q0 >= count) return;
  const int lane = threadIdx.x & 31;
  const int cnt = min(N, count - q0);
  const bool on = lane < cnt * d;
  const int e = on ? __ldg(c.vrow + c.vclass_toff[cls] + int64_t(q0) * d + lane) : 0;  // row << 6 | degree - 1
  const uint32_t rs0 = on && h0 ? __ldg(rsgn + int64_t(e >> 6) * n_tiles + t.t0) : 0u;
  const uint32_t rs1 = on && h1 ? __ldg(rsgn + int64_t(e >> 6) * n_tiles + t.t1) : 0u;
  const int mycol = lane < cnt ? __ldg(c.vnode + first + q0 + lane) : 0;
  const int64_t n0 = int64_t(t.t0) * c.n, n1 = int64_t(t.t1) * c.n;
  const uint32_t my0 = lane < cnt && h0 ? __ldg(yt + n0 + mycol) : 0u;
  const uint32_t my1 = lane < cnt && h1 ? __ldg(yt + n1 + mycol) : 0u;
  const float ym0 = h0 ? __ldg(ymag + t.t0 * kLanes + lane) : 0.f;
  const float ym1 = h1 ? __ldg(ymag + t.t1 * kLanes + lane) : 0.f;
  for (int j = 0; j < cnt; ++j) {
    const int v = __shfl_sync(kFull, mycol, j);
    const uint32_t y0 = __shfl_sync(kFull, my0, j), y1 = __shfl_sync(kFull, my1, j);
    float sum0 = ((y0 >> lane) & 1u) ? -ym0 : ym0;
    float sum1 = ((y1 >> lane) & 1u) ? -ym1 : ym1;
#pragma unroll
    for (int k = 0; k < D; ++k)
      if (k < d) {
        const int src = j * d + k;
        const uint32_t r0 = __shfl_sync(kFull, rs0, src), r1 = __shfl_sync(kFull, rs1, src);
        const int dg = __shfl_sync(kFull, e, src) & 63;
        sum0 += row_msg(fm[0][dg * kLanes + lane], r0, y0, lane);
        sum1 += row_msg(fm[1][dg * kLanes + lane], r1, y1, lane);
      }
    if (h0) {
      if (t.s0) lv[(n0 + v) * kLanes + lane] = sum0;
      const uint32_t hard = __ballot_sync(kFull, sum0 < 0.f);
      if (lane == 0) {
        uint32_t* px = xh + int64_t(v) * n_tiles + t.t0;
        *px = t.a0 == kFull ? hard : (__ldg(px) & ~t.a0) | (hard & t.a0);
      }
    }
    if (h1) {
      if (t.s1) lv[(n1 + v) * kLanes + lane] = sum1;
      const uint32_t hard = __ballot_sync(kFull, sum1 < 0.f);
      if (lane == 1) {
        uint32_t* px = xh + int64_t(v) * n_tiles + t.t1;
        *px = t.a1 == kFull ? hard : (__ldg(px) & ~t.a1) | (hard & t.a1);
      }
    }
  }
}

// vn_rows4_kernel (check degrees within 4 values) for a tile pair: one bit
// transpose per tile, the degree offsets from two ballots, each tile's four
// magnitudes in registers. EXACT: every node of the class has D edges (no
// per-edge test, the node loop unrolled).
template <int D, int NB, bool EXACT = false>
__global__ void __launch_bounds__(256) vn_rows4_pair_kernel(const DevCode c, int cls, float* __restrict__ lv,
                                                            const uint32_t* __restrict__ yt,
                                                            const float* __restrict__ ymag, uint32_t* __restrict__ xh,
                                                            const uint32_t* __restrict__ active, int n_tiles,
                                                            const float* __restrict__ fmag,
                                                            const uint32_t* __restrict__ rsgn) {
  static_assert(NB == 1 || NB == 2, "check degrees within 2 or 4 values");
  const PairTiles t = pair_tiles(blockIdx.y, n_tiles, active);
  if ((t.a0 | t.a1) == 0) return;
  const bool h0 = t.a0 != 0, h1 = t.a1 != 0;
  const int d = EXACT ? D : c.vclass_deg[cls], N = kLanes / d;
  const int first = c.vclass_first[cls], count = c.vclass_first[cls + 1] - first;
  const int q0 = (blockIdx.x * 8 + (threadIdx.x >> 5)) * N;
  if (q0 >= count) return;
  const int lane = threadIdx.x & 31;
  const int cnt = min(N, count - q0);
  const bool on = lane < cnt * d;
  const int e = on ? __ldg(c.vrow + c.vclass_toff[cls] + int64_t(q0) * d + lane) : 0;  // row << 6 | degree - 1
  const uint32_t T0 = warp_transpose32(on && h0 ? __ldg(rsgn + int64_t(e >> 6) * n_tiles + t.t0) : 0u);
  const uint32_t T1 = warp_transpose32(on && h1 ? __ldg(rsgn + int64_t(e >> 6) * n_tiles + t.t1) : 0u);
  const int rel = on ? (e & 63) + 1 - c.min_row_deg : 0;  // 0 .. 2^NB - 1
  const uint32_t b0 = __ballot_sync(kFull, rel & 1), b1 = NB > 1 ? __ballot_sync(kFull, (rel >> 1) & 1) : 0u;
  const int mycol = lane < cnt ? __ldg(c.vnode + first + q0 + lane) : 0;
  const int64_t n0 = int64_t(t.t0) * c.n, n1 = int64_t(t.t1) * c.n;
  const uint32_t my0 = lane < cnt && h0 ? __ldg(yt + n0 + mycol) : 0u;
  const uint32_t my1 = lane < cnt && h1 ? __ldg(yt + n1 + mycol) : 0u;
  const int g0 = c.min_row_deg - 1;
  float ma[1 << NB], mb[1 << NB];
#pragma unroll
  for (int i = 0; i < (1 << NB); ++i) {
    const int g = min(g0 + i, kMaxRowDeg - 1);
    ma[i] = h0 ? __ldg(fmag + (int64_t(t.t0) * kMaxRowDeg + g) * kLanes + lane) : 0.f;
    mb[i] = h1 ? __ldg(fmag + (int64_t(t.t1) * kMaxRowDeg + g) * kLanes + lane) : 0.f;
  }
  const float ym0 = h0 ? __ldg(ymag + t.t0 * kLanes + lane) : 0.f;
  const float ym1 = h1 ? __ldg(ymag + t.t1 * kLanes + lane) : 0.f;
  const uint32_t a0b = __float_as_uint(ma[0]), da = __float_as_uint(ma[1 % (1 << NB)]) - a0b;
  const uint32_t b0b = __float_as_uint(mb[0]), db = __float_as_uint(mb[1 % (1 << NB)]) - b0b;
  // the two magnitudes' bit patterns differ in xa / xb (NB = 1): an edge's pattern is a0b ^ (mask & xa)
  const uint32_t xa = __float_as_uint(ma[1 % (1 << NB)]) ^ a0b, xb = __float_as_uint(mb[1 % (1 << NB)]) ^ b0b;
#pragma unroll(EXACT ? kLanes / D : 1)
  for (int j = 0; j < (EXACT ? kLanes / D : cnt); ++j) {
    if (EXACT && j >= cnt) break;
    const int v = __shfl_sync(kFull, mycol, j);
    const uint32_t yl0 = (__shfl_sync(kFull, my0, j) >> lane) & 1u, yl1 = (__shfl_sync(kFull, my1, j) >> lane) & 1u;
    float sum0 = yl0 ? -ym0 : ym0, sum1 = yl1 ? -ym1 : ym1;
    const int base = j * d;
    const uint32_t sg0 = (T0 ^ (0u - yl0)) >> base, sg1 = (T1 ^ (0u - yl1)) >> base;
    const uint32_t r0 = b0 >> base, r1 = b1 >> base;
#pragma unroll
    for (int k = 0; k < D; ++k)
      if (EXACT || k < d) {
        if constexpr (NB == 1) {
          // edge k's degree bit and sign bits moved to bit 31 by constant shifts: the magnitude's pattern
          // (a0b or a0b ^ xa, the same value as a0b + rb * da) with the sign bit set where the sign is negative
          const uint32_t mk = uint32_t(int32_t(r0 << (31 - k)) >> 31);
          sum0 += __uint_as_float((a0b ^ (mk & xa)) | ((sg0 << (31 - k)) & kSign));
          sum1 += __uint_as_float((b0b ^ (mk & xb)) | ((sg1 << (31 - k)) & kSign));
        } else {
          const bool c0 = r0 & (1u << k), c1 = r1 & (1u << k);
          const float x0 = c1 ? (c0 ? ma[3] : ma[2]) : (c0 ? ma[1] : ma[0]);
          const float x1 = c1 ? (c0 ? mb[3] : mb[2]) : (c0 ? mb[1] : mb[0]);
          sum0 += Bits<float>::copy_sign(x0, sg0 << (31 - k));
          sum1 += Bits<float>::copy_sign(x1, sg1 << (31 - k));
        }
      }
    if (h0) {
      if (t.s0) lv[(n0 + v) * kLanes + lane] = sum0;
      const uint32_t hard = __ballot_sync(kFull, sum0 < 0.f);
      if (lane == 0) {
        uint32_t* px = xh + int64_t(v) * n_tiles + t.t0;
        *px = t.a0 == kFull ? hard : (__ldg(px) & ~t.a0) | (hard & t.a0);
      }
    }
    if (h1) {
      if (t.s1) lv[(n1 + v) * kLanes + lane] = sum1;
      const uint32_t hard = __ballot_sync(kFull, sum1 < 0.f);
      if (lane == 1) {
        uint32_t* px = xh + int64_t(v) * n_tiles + t.t1;
        *px = t.a1 == kFull ? hard : (__ldg(px) & ~t.a1) | (hard & t.a1);
      }
    }
  }
}

}  // namespace dev
}  // namespace mbp
