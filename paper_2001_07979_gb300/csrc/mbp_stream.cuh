// The streaming schedule of libmbp: per iteration (Section 3A, Algorithm 1,
// flooding over all u matrices), kernels over every tile that still has
// unfinished frames:
//   cn_kernel      eq. (6) for every check of every matrix, on V2C = clip(L_V - C2V)
//   vn_kernel      eq. (2): L_V = L_P + sum of the node's C2V over all u matrices,
//                  and the hard decision
//   syn_kernel     the stopping rule H_l x_hat = z^l, per frame and matrix
//   update_kernel  retire the frames that satisfied it (or ran out of iterations)
// and the host reads the number of tiles still decoding after each stopping test.
//
// M is the arithmetic type (float or double), S the stored message type (M
// itself, or __half / __nv_bfloat16 with M = float). Each (M, S) pair is
// instantiated in a file of its own (mbp_stream_<type>.cu) so they build in
// parallel.
#pragma once

#include <cmath>
#include <cstdio>

#include "mbp_device.cuh"
#include "mbp_pair.cuh"

namespace mbp {
namespace {  // every file that includes this keeps its own copies
namespace stream {

using namespace dev;

inline unsigned blocks_for(int64_t n, int per) { return unsigned((n + per - 1) / per); }

// Check rows per warp of the kernels that take rows with lane = tile (stopping
// test, first-iteration row signs).
constexpr int kSynRows = 8;

// FP32 arithmetic on 2- or 4-byte messages stored in tile pairs (msg_at): the
// check and variable-node passes of the sum-product rule take a tile pair per
// warp (mbp_pair.cuh).
template <typename M, typename S>
constexpr bool kPairKernels = sizeof(M) == 4 && sizeof(S) <= 4;

// Resident blocks of 256 threads the check kernel is compiled for: 5 per SM (48
// registers, no spills) for float rows of up to 14 edges, more latency hiding
// than the 4 that 64 registers allow; longer rows (and FP64) keep the
// compiler's choice.
template <typename M>
constexpr int cn_min_blocks(int dmax) {
  return sizeof(M) == 4 && dmax <= 14 ? 5 : 1;
}

// One warp per (tile, check row): 8 rows per block, rows p0 .. p1 - 1 (every
// row for flooding, one matrix's rows for the serial order). Tiles that share
// message slots (msg_at) run side by side: the blocks of tiles 2q and 2q + 1
// alternate along x (cn_grid), so both lines of an edge's slot are read and
// written at about the same time; otherwise tile = blockIdx.y.
// RIN: iteration 2 after a row-form iteration 1 (the old messages are rebuilt
// from fmag / rsgn and Bob's sign words yt); the kernel then clears the row-form
// flag counters[2], as the messages are per edge again.
template <typename S>
inline dim3 cn_grid(int rows, int n_tiles) {
  if (kMsgTiles<S> == 2) return dim3(2 * blocks_for(rows, 8), unsigned((n_tiles + 1) / 2));
  return dim3(blocks_for(rows, 8), unsigned(n_tiles));
}

template <typename M, typename S, int DMAX, bool FIXED, bool RIN = false>
__global__ void __launch_bounds__(256, cn_min_blocks<M>(DMAX)) cn_kernel(const DevCode c, int p0, int p1, int first_iter,
                                                 S* __restrict__ c2v, const M* __restrict__ lsrc,
                                                 const uint32_t* __restrict__ yt, const M* __restrict__ ymag,
                                                 const uint32_t* __restrict__ zt,
                                                 const uint32_t* __restrict__ active, int n_tiles, M l_max,
                                                 int32_t* __restrict__ lacc, float qscale,
                                                 const M* __restrict__ fmag, const uint32_t* __restrict__ rsgn,
                                                 int32_t* __restrict__ counters) {
  if (RIN && blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) counters[2] = 0;
  constexpr bool kPaired = kMsgTiles<S> == 2;
  const int tile = kPaired ? 2 * int(blockIdx.y) + int(blockIdx.x & 1u) : int(blockIdx.y);
  if (tile >= n_tiles) return;
  const uint32_t act = active[tile];
  if (act == 0) return;
  const int p = p0 + int(kPaired ? blockIdx.x >> 1 : blockIdx.x) * 8 + (threadIdx.x >> 5);
  if (p >= p1) return;
  CnView<M, S> v = cn_view<M, S, kPolStream>(c, tile, act, first_iter, c2v, lsrc, yt, ymag, zt,
                                             FIXED ? lacc : nullptr);
  if constexpr (RIN) {
    v.rm = fmag + int64_t(tile) * kMaxRowDeg * kLanes + (threadIdx.x & 31);
    v.rs = rsgn + tile;
    v.rs_nt = n_tiles;
    v.yprev = yt + int64_t(tile) * c.n;
  }
  cn_view_row<M, S, DMAX, FIXED, kPolStream, RIN>(v, p, first_iter, l_max, Arith<M>::delta(l_max), qscale);
}

// Iteration 1 of BSC inputs in a kernel of its own (sign words in, messages
// out; far fewer registers than cn_kernel, so more warps keep writes in flight).
template <typename M, typename S, int DMAX>
__global__ void __launch_bounds__(256) cn_first_kernel(const DevCode c, int p0, int p1, S* __restrict__ c2v,
                                                       const uint32_t* __restrict__ yt, const M* __restrict__ ymag,
                                                       const uint32_t* __restrict__ zt,
                                                       const uint32_t* __restrict__ active, M l_max) {
  const int tile = blockIdx.y;
  const uint32_t act = active[tile];
  if (act == 0) return;
  const int p = p0 + blockIdx.x * 8 + (threadIdx.x >> 5);
  if (p >= p1) return;
  const int lane = threadIdx.x & 31;
  const int base = c.slice_base[p];
  const int deg = c.slice_base[p + 1] - base;
  const int* cols = c.slot_col + base;
  const uint32_t par = ((zt[int64_t(tile) * c.m_tot + p] >> lane) & 1u) << 31;
  const bool store = (act >> lane) & 1u;
  const M ym = __ldg(ymag + tile * kLanes + lane);
  S* msg = c2v + msg_at<S>(tile, c.s_tot, lane) + int64_t(base) * kMsgStride<S>;
  const uint32_t* ysrc = yt + int64_t(tile) * c.n;
  const M inv = Arith<M>::delta(l_max);  // d_lmax
  if (deg == DMAX) cn_row_signs<M, S, DMAX, false, kPolStream>(deg, cols, ysrc, ym, msg, par, store, l_max, inv);
  else cn_row_signs<M, S, DMAX, true, kPolStream>(deg, cols, ysrc, ym, msg, par, store, l_max, inv);
}

// Iteration 1 of BSC inputs in row form (DevState::fmag), part 1: the sign word of
// each row, z_j xor the row's parity of Bob's bits, for the 32 frames of a tile at
// once. Before iteration 1's variable-node pass the decision words are Bob's bits
// (node-major: one coalesced line per edge for 32 tiles) wherever the frame's
// channel magnitude is positive; the bits of other frames come from yt. A warp
// takes kSynRows rows, lane = tile, and writes the words row-major; the kernel
// sets the row-form flag counters[2]. The row's parity before the correction to
// Bob's bits is that of the hard decision of iteration 0, so with fail != NULL
// the kernel is also the stopping test before iteration 1: as in syn_kernel, the
// failing lanes are ORed per block and then into fail[tile][l].
template <int DMAX>
__global__ void __launch_bounds__(256) first_rows_kernel(const DevCode c, int n_tiles, const uint32_t* __restrict__ xh,
                                                         const uint32_t* __restrict__ ztt,
                                                         const uint32_t* __restrict__ yt,
                                                         const uint32_t* __restrict__ ppos,
                                                         const uint32_t* __restrict__ active,
                                                         uint32_t* __restrict__ rsgn, int32_t* __restrict__ counters,
                                                         uint32_t* __restrict__ fail) {
  __shared__ uint32_t s_fail[kMaxU][kLanes];
  if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) counters[2] = 1;
  const int lane = threadIdx.x & 31;
  const int tile = blockIdx.y * kLanes + lane;
  const bool tv = tile < n_tiles;
  const uint32_t act = tv ? active[tile] : 0u;
  if (__syncthreads_or(act != 0) == 0) return;  // every tile of the block has finished
  if (fail) {
    for (int i = threadIdx.x; i < c.u * kLanes; i += blockDim.x) s_fail[i / kLanes][i % kLanes] = 0u;
    __syncthreads();
  }
  const int r0 = (blockIdx.x * 8 + (threadIdx.x >> 5)) * kSynRows;
  if (r0 < c.m_tot) {
    const uint32_t pp = tv ? ppos[tile] : kFull;
    const uint32_t* y = yt + int64_t(tv ? tile : 0) * c.n;
    uint32_t acc = 0;
    int lcur = c.row_mat[r0];
#pragma unroll
    for (int i = 0; i < kSynRows; ++i) {
      const int r = r0 + i;
      if (r < c.m_tot) {
        const int base = c.slice_base[r];
        const int deg = c.slice_base[r + 1] - base;
        uint32_t x = tv ? __ldg(ztt + int64_t(r) * n_tiles + tile) : 0u;
        uint32_t yb = 0u;
#pragma unroll
        for (int k = 0; k < DMAX; ++k)
          if (k < deg) {
            const int col = __ldg(c.slot_col + base + k);
            if (tv) {
              x ^= __ldg(xh + int64_t(col) * n_tiles + tile);
              if (pp != kFull) yb ^= __ldg(y + col) & ~pp;
            }
          }
        if (fail) {  // the stopping test before iteration 1: the row's failing lanes of the hard decision x_0
          const int l = c.row_mat[r];
          if (l != lcur) {  // warp-uniform
            if (acc) atomicOr(&s_fail[lcur][lane], acc);
            acc = 0;
            lcur = l;
          }
          acc |= x & act;
        }
        if (tv) rsgn[int64_t(r) * n_tiles + tile] = x ^ yb;
      }
    }
    if (fail && acc) atomicOr(&s_fail[lcur][lane], acc);
  }
  if (!fail) return;
  __syncthreads();
  for (int i = threadIdx.x; i < c.u * kLanes; i += blockDim.x) {
    const uint32_t v = s_fail[i / kLanes][i % kLanes];
    const int t = blockIdx.y * kLanes + i % kLanes;
    if (v && t < n_tiles) {
      uint32_t* f = fail + int64_t(t) * c.u + i / kLanes;
      if ((__ldcg(f) & v) != v) atomicOr(f, v);
    }
  }
}

// Part 2: the output magnitude of a row of degree d (the same for every row of
// that degree: all of a frame's inputs have the magnitude ln((1 - e)/e)), per
// frame, rounded to the message type: fmag[tile][d - 1][lane].
template <typename M, typename S>
__global__ void first_mag_kernel(int n_tiles, int max_deg, const M* __restrict__ ymag, M l_max,
                                 M* __restrict__ fmag) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;  // (tile, degree - 1, lane)
  if (i >= n_tiles * max_deg * kLanes) return;
  const int lane = i % kLanes, d = (i / kLanes) % max_deg, tile = i / (kLanes * max_deg);
  fmag[(int64_t(tile) * kMaxRowDeg + d) * kLanes + lane] =
      row_mag<M, S>(cn_first_mag_any<M>(d + 1, ymag[tile * kLanes + lane], l_max, Arith<M>::delta(l_max)));
}

// The min-sum check rule (variant), FP32 arithmetic; same layout as cn_kernel.
template <typename S, int DMAX>
__global__ void __launch_bounds__(256) cn_minsum_kernel(const DevCode c, int p0, int p1, int first_iter,
                                                        S* __restrict__ c2v, const float* __restrict__ lsrc,
                                                        const uint32_t* __restrict__ yt,
                                                        const float* __restrict__ ymag,
                                                        const uint32_t* __restrict__ zt,
                                                        const uint32_t* __restrict__ active, float l_max) {
  const int tile = blockIdx.y;
  const uint32_t act = active[tile];
  if (act == 0) return;
  const int p = p0 + blockIdx.x * 8 + (threadIdx.x >> 5);
  if (p >= p1) return;
  const CnView<float, S> v = cn_view<float, S, kPolStream>(c, tile, act, first_iter, c2v, lsrc, yt, ymag, zt, nullptr);
  cn_view_row_minsum<S, DMAX, kPolStream>(v, p, first_iter, l_max);
}

// One warp per (tile, variable node): 8 nodes per block.
template <typename M, typename S>
__global__ void __launch_bounds__(256) vn_kernel(const DevCode c, const S* __restrict__ c2v, M* __restrict__ lv,
                                                 const M* __restrict__ lp, const uint32_t* __restrict__ yt,
                                                 const M* __restrict__ ymag, uint32_t* __restrict__ xh,
                                                 const uint32_t* __restrict__ active) {
  const int tile = blockIdx.y;
  const uint32_t act = active[tile];
  if (act == 0) return;
  const int col = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (col >= c.n) return;
  vn_node<M, S, kPolStream>(c, tile, col, act, c2v, lv, lp, yt, ymag, xh, gridDim.y);
}

// The same update for the nodes of one degree class (DevCode::vclass_*): a
// node and its slots are loaded together (one dependent round trip fewer), and
// a warp takes N nodes of degree <= D so that 12 to 16 gathers are in flight
// (one tile per warp: FP64 messages and classes of more than 16 edges; the
// other storage types take vn_class_pair_kernel).
template <typename M, typename S, int D, int N>
__global__ void __launch_bounds__(256) vn_class_kernel(const DevCode c, int cls, const S* __restrict__ c2v,
                                                       M* __restrict__ lv, const M* __restrict__ lp,
                                                       const uint32_t* __restrict__ yt, const M* __restrict__ ymag,
                                                       uint32_t* __restrict__ xh,
                                                       const uint32_t* __restrict__ active) {
  const int tile = blockIdx.y;
  const uint32_t act = active[tile];
  if (act == 0) return;
  const int first = c.vclass_first[cls], count = c.vclass_first[cls + 1] - first;
  const int qq = (blockIdx.x * 8 + (threadIdx.x >> 5)) * N;
  if (qq >= count) return;
  const int d = c.vclass_deg[cls];
  const VnView<M, S> v = vn_view<M, S, kPolStream>(c, tile, act, c2v, lv, lp, yt, ymag, xh, gridDim.y);
  const int32_t* slots = c.vslot + c.vclass_toff[cls] + int64_t(qq) * d;
  if constexpr (D > 16) {  // long nodes: one per warp, 16 edges at a time
    vn_core<M, S, kPolStream>(v, __ldg(c.vnode + first + qq), slots, d);
  } else {
    vn_class_nodes<M, S, D, N, kPolStream>(v, c.vnode, first + qq, slots, d, min(N, count - qq));
  }
}

// Eq. (2) in iteration 1 when its messages are in row form (fmag / rsgn, BSC
// inputs): a warp takes the N = 32 / d nodes of one class (degree d <= D <= 16)
// whose N d edges fit its lanes. Lane l fetches edge l % d of node l / d -- its
// row entry (DevCode::vrow, one coalesced load) and that row's sign word (one
// gather) -- and each node then sums its edges in stacked-row order, taking every
// edge's word from its lane (shuffles) and the magnitude of the row's degree from
// the tile's table in shared memory.
template <typename M, int D>
__global__ void __launch_bounds__(256) vn_rows_kernel(const DevCode c, int cls, M* __restrict__ lv,
                                                      const uint32_t* __restrict__ yt, const M* __restrict__ ymag,
                                                      uint32_t* __restrict__ xh, const uint32_t* __restrict__ active,
                                                      const M* __restrict__ fmag, const uint32_t* __restrict__ rsgn) {
  __shared__ M fm[kMaxRowDeg * kLanes];
  const int tile = blockIdx.y;
  const uint32_t act = active[tile];
  if (act == 0) return;
  for (int i = threadIdx.x; i < c.max_row_deg * kLanes; i += blockDim.x)
    fm[i] = fmag[int64_t(tile) * kMaxRowDeg * kLanes + i];
  __syncthreads();
  const int d = c.vclass_deg[cls], N = kLanes / d;
  const int first = c.vclass_first[cls], count = c.vclass_first[cls + 1] - first;
  const int q0 = (blockIdx.x * 8 + (threadIdx.x >> 5)) * N;
  if (q0 >= count) return;
  const int lane = threadIdx.x & 31;
  const int cnt = min(N, count - q0);
  const bool on = lane < cnt * d;
  const int e = on ? __ldg(c.vrow + c.vclass_toff[cls] + int64_t(q0) * d + lane) : 0;  // row << 6 | degree - 1
  const uint32_t rs = on ? __ldg(rsgn + int64_t(e >> 6) * gridDim.y + tile) : 0u;
  const int mycol = lane < cnt ? __ldg(c.vnode + first + q0 + lane) : 0;
  const uint32_t myy = lane < cnt ? __ldg(yt + int64_t(tile) * c.n + mycol) : 0u;
  const M ym = __ldg(ymag + tile * kLanes + lane);
  const int64_t node0 = int64_t(tile) * c.n;
  for (int j = 0; j < cnt; ++j) {
    const int col = __shfl_sync(kFull, mycol, j);
    const uint32_t yv = __shfl_sync(kFull, myy, j);
    M sum = ((yv >> lane) & 1u) ? -ym : ym;
#pragma unroll
    for (int k = 0; k < D; ++k)
      if (k < d) {
        const uint32_t r = __shfl_sync(kFull, rs, j * d + k);
        const int dg = __shfl_sync(kFull, e, j * d + k) & 63;
        sum += row_msg(fm[dg * kLanes + lane], r, yv, lane);
      }
    if ((act >> lane) & 1u) lv[(node0 + col) * kLanes + lane] = sum;
    const uint32_t hard = __ballot_sync(kFull, sum < M(0));
    if (lane == 0) {
      uint32_t* px = xh + int64_t(col) * gridDim.y + tile;
      *px = act == kFull ? hard : (__ldg(px) & ~act) | (hard & act);
    }
  }
}

// vn_rows_kernel for codes whose check degrees span at most 4 values (PEG codes:
// a degree or two around the mean), without per-edge exchanges: one warp-wide
// bit transpose of the edges' sign words gives each lane (frame) every edge's
// sign bit, two ballots give every edge's degree offset from the smallest check
// degree, and the four magnitudes of those degrees sit in registers; each edge
// is then a few ALU instructions. Same values, same order as vn_rows_kernel.
template <typename M, int D, int NB>
__global__ void __launch_bounds__(256) vn_rows4_kernel(const DevCode c, int cls, M* __restrict__ lv,
                                                       const uint32_t* __restrict__ yt, const M* __restrict__ ymag,
                                                       uint32_t* __restrict__ xh, const uint32_t* __restrict__ active,
                                                       const M* __restrict__ fmag, const uint32_t* __restrict__ rsgn) {
  static_assert(NB == 1 || NB == 2, "check degrees within 2 or 4 values");
  const int tile = blockIdx.y;
  const uint32_t act = active[tile];
  if (act == 0) return;
  const int d = c.vclass_deg[cls], N = kLanes / d;
  const int first = c.vclass_first[cls], count = c.vclass_first[cls + 1] - first;
  const int q0 = (blockIdx.x * 8 + (threadIdx.x >> 5)) * N;
  if (q0 >= count) return;
  const int lane = threadIdx.x & 31;
  const int cnt = min(N, count - q0);
  const bool on = lane < cnt * d;
  const int e = on ? __ldg(c.vrow + c.vclass_toff[cls] + int64_t(q0) * d + lane) : 0;  // row << 6 | degree - 1
  const uint32_t T = warp_transpose32(on ? __ldg(rsgn + int64_t(e >> 6) * gridDim.y + tile) : 0u);
  const int rel = on ? (e & 63) + 1 - c.min_row_deg : 0;  // 0 .. 2^NB - 1
  const uint32_t b0 = __ballot_sync(kFull, rel & 1), b1 = NB > 1 ? __ballot_sync(kFull, (rel >> 1) & 1) : 0u;
  const int mycol = lane < cnt ? __ldg(c.vnode + first + q0 + lane) : 0;
  const int64_t node0 = int64_t(tile) * c.n;
  const uint32_t myy = lane < cnt ? __ldg(yt + node0 + mycol) : 0u;
  const M* fm = fmag + int64_t(tile) * kMaxRowDeg * kLanes + lane;
  const int g0 = c.min_row_deg - 1;
  M mg[1 << NB];
#pragma unroll
  for (int i = 0; i < (1 << NB); ++i) mg[i] = __ldg(fm + min(g0 + i, kMaxRowDeg - 1) * kLanes);
  const M ym = __ldg(ymag + tile * kLanes + lane);
  [[maybe_unused]] uint32_t m0b = 0, dmb = 0;
  if constexpr (NB == 1 && sizeof(M) == 4) {
    m0b = __float_as_uint(float(mg[0]));
    dmb = __float_as_uint(float(mg[1])) - m0b;
  }
  for (int j = 0; j < cnt; ++j) {
    const int col = __shfl_sync(kFull, mycol, j);
    const uint32_t yl = (__shfl_sync(kFull, myy, j) >> lane) & 1u;
    M sum = yl ? -ym : ym;
    // node j's edges at bits 0 .. d - 1: sign (Bob's bit folded in) and degree offset
    const int base = j * d;
    const uint32_t sg = (T ^ (0u - yl)) >> base, r0 = b0 >> base, r1 = b1 >> base;
#pragma unroll
    for (int k = 0; k < D; ++k)
      if (k < d) {
        if constexpr (NB == 1 && sizeof(M) == 4) {
          // the signed magnitude's bit pattern by integer multiply-adds (the FMA pipe): the degree bit picks
          // m1 over m0, the sign bit sets bit 31 (both magnitudes are non-negative)
          const uint32_t rb = (r0 >> k) & 1u, sb = (sg >> k) & 1u;
          sum += __uint_as_float(m0b + rb * dmb + sb * 0x80000000u);
        } else {
          M m;
          if constexpr (NB == 1) m = (r0 & (1u << k)) ? mg[1] : mg[0];
          else m = (r1 & (1u << k)) ? ((r0 & (1u << k)) ? mg[3] : mg[2]) : ((r0 & (1u << k)) ? mg[1] : mg[0]);
          sum += Bits<M>::copy_sign(m, sg << (31 - k));
        }
      }
    if ((act >> lane) & 1u) lv[(node0 + col) * kLanes + lane] = sum;
    const uint32_t hard = __ballot_sync(kFull, sum < M(0));
    if (lane == 0) {
      uint32_t* px = xh + int64_t(col) * gridDim.y + tile;
      *px = act == kFull ? hard : (__ldg(px) & ~act) | (hard & act);
    }
  }
}

// Whether iteration 1 of a flooding sum-product decode keeps its messages in row
// form (DevState::fmag): BSC inputs (one channel magnitude per frame) and every
// variable-node class of at most 32 edges.
inline bool rows_ok(const DevCode& c, const DevState& st) {
  return st.yt && st.fmag && c.vrow && c.n_vclass > 0 && c.vclass_deg[c.n_vclass - 1] <= 32 &&
         c.max_row_deg <= 32;
}

// Eq. (2) for every node of every unfinished tile: one launch per degree class, or one over all nodes.
// rows: iteration 1 in row form (rows_ok).
template <typename M, typename S>
void launch_vn(const DevCode& c, const DevState& st, bool rows, cudaStream_t s0, const StreamFork* fork = nullptr) {
  if (c.n_vclass > 0) {
    // with a fork (graph capture), classes 1, 2, ... run on the auxiliary streams, beside class 0
    const bool forked = fork && c.n_vclass > 1;
    const int n_aux = forked ? (c.n_vclass - 1 < 2 ? c.n_vclass - 1 : 2) : 0;
    if (forked) {
      cudaEventRecord(fork->fork, s0);
      for (int j = 0; j < n_aux; ++j) cudaStreamWaitEvent(fork->aux[j], fork->fork, 0);
    }
    for (int k = 0; k < c.n_vclass; ++k) {
      const cudaStream_t s = forked && k > 0 ? fork->aux[(k - 1) % 2] : s0;
      const int count = c.vclass_first[k + 1] - c.vclass_first[k], d = c.vclass_deg[k];
      if (rows) {  // classes of up to 32 edges (rows_ok), 32 / d nodes per warp
        const int per_warp = kLanes / d;
        const unsigned blocks = blocks_for(count, 8 * per_warp);
        if constexpr (kPairKernels<M, S>) {
          const unsigned pairs = unsigned((st.n_tiles + 1) / 2);
#define MBP_VR2(K, ...)                                                                                        \
  K<__VA_ARGS__><<<dim3(blocks, pairs), 256, 0, s>>>(c, k, static_cast<float*>(st.lv), st.yt,                    \
                                           static_cast<const float*>(st.chan_mag), st.xh, st.active, st.n_tiles, \
                                           static_cast<const float*>(st.fmag), st.rsgn)
          if (c.max_row_deg - c.min_row_deg <= 1) {
            if (d == 4) MBP_VR2(vn_rows4_pair_kernel, 4, 1, true);
            else if (d == 6) MBP_VR2(vn_rows4_pair_kernel, 6, 1, true);
            else if (d == 8) MBP_VR2(vn_rows4_pair_kernel, 8, 1, true);
            else if (d == 16) MBP_VR2(vn_rows4_pair_kernel, 16, 1, true);
            else if (d == 24) MBP_VR2(vn_rows4_pair_kernel, 24, 1, true);
            else if (d <= 4) MBP_VR2(vn_rows4_pair_kernel, 4, 1);
            else if (d <= 8) MBP_VR2(vn_rows4_pair_kernel, 8, 1);
            else if (d <= 16) MBP_VR2(vn_rows4_pair_kernel, 16, 1);
            else MBP_VR2(vn_rows4_pair_kernel, 32, 1);
          } else if (c.max_row_deg - c.min_row_deg <= 3) {
            if (d <= 4) MBP_VR2(vn_rows4_pair_kernel, 4, 2);
            else if (d <= 8) MBP_VR2(vn_rows4_pair_kernel, 8, 2);
            else if (d <= 16) MBP_VR2(vn_rows4_pair_kernel, 16, 2);
            else MBP_VR2(vn_rows4_pair_kernel, 32, 2);
          } else {
            if (d <= 4) MBP_VR2(vn_rows_pair_kernel, 4);
            else if (d <= 8) MBP_VR2(vn_rows_pair_kernel, 8);
            else if (d <= 16) MBP_VR2(vn_rows_pair_kernel, 16);
            else MBP_VR2(vn_rows_pair_kernel, 32);
          }
#undef MBP_VR2
        } else {
#define MBP_VR(K, ...)                                                                                         \
  K<M, __VA_ARGS__><<<dim3(blocks, st.n_tiles), 256, 0, s>>>(c, k, static_cast<M*>(st.lv), st.yt,                \
                                                   static_cast<const M*>(st.chan_mag), st.xh, st.active,           \
                                                   static_cast<const M*>(st.fmag), st.rsgn)
          if (c.max_row_deg - c.min_row_deg <= 1) {
            if (d <= 4) MBP_VR(vn_rows4_kernel, 4, 1);
            else if (d <= 8) MBP_VR(vn_rows4_kernel, 8, 1);
            else if (d <= 16) MBP_VR(vn_rows4_kernel, 16, 1);
            else MBP_VR(vn_rows4_kernel, 32, 1);
          } else if (c.max_row_deg - c.min_row_deg <= 3) {
            if (d <= 4) MBP_VR(vn_rows4_kernel, 4, 2);
            else if (d <= 8) MBP_VR(vn_rows4_kernel, 8, 2);
            else if (d <= 16) MBP_VR(vn_rows4_kernel, 16, 2);
            else MBP_VR(vn_rows4_kernel, 32, 2);
          } else {
            if (d <= 4) MBP_VR(vn_rows_kernel, 4);
            else if (d <= 8) MBP_VR(vn_rows_kernel, 8);
            else if (d <= 16) MBP_VR(vn_rows_kernel, 16);
            else MBP_VR(vn_rows_kernel, 32);
          }
#undef MBP_VR
        }
        continue;
      }
      if constexpr (kPairKernels<M, S>) {  // tile pairs for classes of up to 16 edges
        const unsigned pairs = unsigned((st.n_tiles + 1) / 2);
#define MBP_VN2(D, N)                                                                                         \
  vn_class_pair_kernel<S, D, N><<<dim3(blocks_for(count, 8 * N), pairs), 256, 0, s>>>(                        \
      c, k, static_cast<const S*>(st.c2v), static_cast<float*>(st.lv), static_cast<const float*>(st.lp), st.yt, \
      static_cast<const float*>(st.chan_mag), st.xh, st.active, st.n_tiles)
        // N nodes per warp: small enough for 5 blocks per SM (47-48 registers); the short classes are bound by
        // each warp's chain of index loads and gathers, so resident warps count for more than gathers per warp
        // (degree 4: N = 3 over N = 4 and 6; degree 6: an exact D = 6 with N = 2 over D = 8 and over N = 3)
        if (d <= 4) { MBP_VN2(4, 3); continue; }
        if (d <= 6) { MBP_VN2(6, 2); continue; }
        if (d <= 8) { MBP_VN2(8, 2); continue; }
        if (d <= 16) { MBP_VN2(16, 1); continue; }
        if (d <= 24) { MBP_VN2(24, 1); continue; }
        if (d <= 32) { MBP_VN2(32, 1); continue; }
#undef MBP_VN2
      }
#define MBP_VN(D, N)                                                                                        \
  vn_class_kernel<M, S, D, N><<<dim3(blocks_for(count, 8 * N), st.n_tiles), 256, 0, s>>>(                  \
      c, k, static_cast<const S*>(st.c2v), static_cast<M*>(st.lv), static_cast<const M*>(st.lp), st.yt,     \
      static_cast<const M*>(st.chan_mag), st.xh, st.active)
      if (d <= 4) MBP_VN(4, 4);
      else if (d <= 8) MBP_VN(8, 2);
      else if (d <= 16) MBP_VN(16, 1);
      else MBP_VN(64, 1);
#undef MBP_VN
    }
    if (forked)
      for (int j = 0; j < n_aux; ++j) {
        cudaEventRecord(fork->join[j], fork->aux[j]);
        cudaStreamWaitEvent(s0, fork->join[j], 0);
      }
  } else {
    const cudaStream_t s = s0;
    vn_kernel<M, S><<<dim3(blocks_for(c.n, 8), st.n_tiles), 256, 0, s>>>(
        c, static_cast<const S*>(st.c2v), static_cast<M*>(st.lv), static_cast<const M*>(st.lp), st.yt,
        static_cast<const M*>(st.chan_mag), st.xh, st.active);
  }
}

// L_V = L_P + lacc / qscale and the hard decision, for the fixed-point single
// pass. One warp per (tile, variable node).
template <typename M>
__global__ void __launch_bounds__(256) finalize_kernel(const DevCode c, const int32_t* __restrict__ lacc,
                                                       M* __restrict__ lv, const M* __restrict__ lp,
                                                       const uint32_t* __restrict__ yt, const M* __restrict__ ymag,
                                                       uint32_t* __restrict__ xh, const uint32_t* __restrict__ active,
                                                       float inv_qscale) {
  const int tile = blockIdx.y;
  const uint32_t act = active[tile];
  if (act == 0) return;
  const int col = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (col >= c.n) return;
  const int lane = threadIdx.x & 31;
  const int64_t tn = int64_t(tile) * c.n + col;
  const int64_t at = tn * kLanes + lane;
  const M sum = channel_llr<M, kPolStream>(lp, yt, ymag, tn, tile, lane) + M(float(lacc[at]) * inv_qscale);
  if ((act >> lane) & 1u) lv[at] = sum;
  const uint32_t hard = __ballot_sync(kFull, sum < M(0));
  if (lane == 0) {
    uint32_t* px = xh + int64_t(col) * gridDim.y + tile;
    *px = (*px & ~act) | (hard & act);
  }
}

// The stopping test (the node-major decision words, DevState::xh): a warp takes kSynRows
// consecutive check rows (in position order, so one matrix except where the
// matrices meet) for 32 tiles, lane = tile (tiles 32 y .. 32 y + 31, y =
// blockIdx.y): every edge's words for those tiles are one coalesced line. The
// failing lanes of each tile are ORed over the warp's rows, then over the
// block's warps in shared memory, and each block ORs its result into
// fail[tile][l] only where it sets bits that are not set yet (in the iterations
// where most frames still fail, the first blocks set them and the others skip
// the global atomic, which would otherwise queue thousands of times on the same
// few words).
template <int DMAX>
__global__ void __launch_bounds__(256) syn_kernel(const DevCode c, int n_tiles, const uint32_t* __restrict__ xh,
                                                  const uint32_t* __restrict__ ztt,
                                                  const uint32_t* __restrict__ active, uint32_t* __restrict__ fail) {
  __shared__ uint32_t s_fail[kMaxU][kLanes];
  const int lane = threadIdx.x & 31;
  const int tile = blockIdx.y * kLanes + lane;
  const bool tv = tile < n_tiles;
  const uint32_t act = tv ? active[tile] : 0u;
  if (__syncthreads_or(act != 0) == 0) return;  // every tile of the block has finished
  for (int i = threadIdx.x; i < c.u * kLanes; i += blockDim.x) s_fail[i / kLanes][i % kLanes] = 0u;
  __syncthreads();
  const int r0 = (blockIdx.x * 8 + (threadIdx.x >> 5)) * kSynRows;
  if (r0 < c.m_tot) {
    uint32_t acc = 0;
    int lcur = c.row_mat[r0];
#pragma unroll
    for (int i = 0; i < kSynRows; ++i) {
      const int r = r0 + i;
      if (r >= c.m_tot) break;
      const int l = c.row_mat[r];
      if (l != lcur) {  // warp-uniform
        if (acc) atomicOr(&s_fail[lcur][lane], acc);
        acc = 0;
        lcur = l;
      }
      const int base = c.slice_base[r];
      const int deg = c.slice_base[r + 1] - base;
      int col[DMAX];
#pragma unroll
      for (int k = 0; k < DMAX; ++k) col[k] = k < deg ? __ldg(c.slot_col + base + k) : -1;
      uint32_t w = tv ? __ldg(ztt + int64_t(r) * n_tiles + tile) : 0u;
#pragma unroll
      for (int k = 0; k < DMAX; ++k)
        if (col[k] >= 0 && tv) w ^= __ldg(xh + int64_t(col[k]) * n_tiles + tile);
      acc |= w & act;
    }
    if (acc) atomicOr(&s_fail[lcur][lane], acc);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < c.u * kLanes; i += blockDim.x) {
    const uint32_t v = s_fail[i / kLanes][i % kLanes];
    const int t = blockIdx.y * kLanes + i % kLanes;
    if (v && t < n_tiles) {
      uint32_t* f = fail + int64_t(t) * c.u + i / kLanes;
      if ((__ldcg(f) & v) != v) atomicOr(f, v);
    }
  }
}

template <int DMAX>
void launch_syn(const DevCode& c, const DevState& st, cudaStream_t s) {
  const dim3 grid(blocks_for(c.m_tot, 8 * kSynRows), unsigned((st.n_tiles + kLanes - 1) / kLanes));
  syn_kernel<DMAX><<<grid, 256, 0, s>>>(c, st.n_tiles, st.xh, st.ztt, st.active, st.fail);
}

inline void launch_syn_any(const DevCode& c, const DevState& st, cudaStream_t s) {
  if (c.max_row_deg <= 8) launch_syn<8>(c, st, s);
  else if (c.max_row_deg <= 16) launch_syn<16>(c, st, s);
  else if (c.max_row_deg <= 32) launch_syn<32>(c, st, s);
  else launch_syn<kMaxRowDeg>(c, st, s);
}

// One thread per tile.
__global__ void update_kernel(int F, int n_tiles, int u, int t, int max_iter, int early_exit,
                              uint32_t* __restrict__ active, uint32_t* __restrict__ fail,
                              int32_t* __restrict__ iters, uint8_t* __restrict__ success,
                              uint8_t* __restrict__ synd_ok, const int32_t* __restrict__ perm,
                              int32_t* __restrict__ counters) {
  const int tile = blockIdx.x * blockDim.x + threadIdx.x;
  if (tile >= n_tiles) return;
  if (update_tile(tile, F, u, t, max_iter, early_exit, active, fail, iters, success, synd_ok, perm))
    atomicAdd(&counters[0], 1);
}

// The rows' sign words of iteration 1 in row form; with fail, also the stopping test before iteration 1.
template <int DMAX>
void launch_first_rows(const DevCode& c, const DevState& st, const uint32_t* yt, uint32_t* fail, cudaStream_t s) {
  first_rows_kernel<DMAX><<<dim3(blocks_for(c.m_tot, 8 * kSynRows), unsigned((st.n_tiles + kLanes - 1) / kLanes)),
                            256, 0, s>>>(c, st.n_tiles, st.xh, st.ztt, yt, st.ppos, st.active, st.rsgn, st.counters,
                                         fail);
}

// The same unroll bounds as the check kernels of FP32 arithmetic (rows of at most 32 edges: rows_ok).
inline void launch_first_rows_any(const DevCode& c, const DevState& st, uint32_t* fail, cudaStream_t s) {
  const int d = c.max_row_deg;
#define MBP_FR(D) launch_first_rows<D>(c, st, st.yt, fail, s)
  if (d <= 4) MBP_FR(4);
  else if (d <= 6) MBP_FR(6);
  else if (d <= 8) MBP_FR(8);
  else if (d <= 10) MBP_FR(10);
  else if (d <= 12) MBP_FR(12);
  else if (d <= 14) MBP_FR(14);
  else if (d <= 16) MBP_FR(16);
  else if (d <= 18) MBP_FR(18);
  else if (d <= 20) MBP_FR(20);
  else if (d <= 22) MBP_FR(22);
  else if (d <= 24) MBP_FR(24);
  else MBP_FR(32);
#undef MBP_FR
}

// Rows p0 .. p1 - 1 of every tile that is still decoding, from the posterior (or L_P) lsrc, or from the sign
// words yt in the first iteration of BSC inputs.
// rows: 1 = iteration 1 writes its messages in row form, 3 = the same with the
// rows' sign words already formed (by the stopping test before iteration 1),
// 2 = iteration 2 reads the previous messages in row form, 0 = per edge.
struct CnLaunch {
  int p0, p1, first_iter;
  const void* lsrc;
  const uint32_t* yt;
  int rows;
};

template <typename M, typename S, int DMAX, bool FIXED>
void launch_cn(const DevCode& c, const DevState& st, const CnLaunch& q, double l_max, float qscale, int rule,
               cudaStream_t s) {
  const dim3 grid(blocks_for(q.p1 - q.p0, 8), st.n_tiles);
  if constexpr (!FIXED && DMAX <= 32) {
    if (q.rows == 1 || q.rows == 3) {  // iteration 1 in row form: the rows' sign words and the magnitude table
      if (q.rows == 1) launch_first_rows<DMAX>(c, st, q.yt, nullptr, s);
      const int cells = st.n_tiles * c.max_row_deg * kLanes;
      first_mag_kernel<M, S><<<blocks_for(cells, 256), 256, 0, s>>>(st.n_tiles, c.max_row_deg,
                                                                   static_cast<const M*>(st.chan_mag), M(l_max),
                                                                   static_cast<M*>(st.fmag));
      return;
    }
  }
  const M* rm_in = q.rows == 2 ? static_cast<const M*>(st.fmag) : nullptr;
  // Tile pairs (mbp_pair.cuh): every sum-product pass of rows up to 24 edges. On the paired FP32 layout the
  // pair kernel measured faster than the one-tile cn_kernel for rows of 14 edges (iteration 2, issue-bound,
  // shares the row's loads between two tiles; later iterations, memory-bound, keep a row's two lines per
  // slot in one warp) and of 21 edges (whole decodes at rate 0.8: 7 to 11% more throughput).
  if constexpr (kPairKernels<M, S> && !FIXED && DMAX <= 24) {
    if (rule == MBP_RULE_SUM_PRODUCT) {
      const dim3 pgrid(grid.x, unsigned((st.n_tiles + 1) / 2));
      if (q.first_iter && q.yt)
        cn_first_pair_kernel<S, DMAX><<<pgrid, 256, 0, s>>>(c, q.p0, q.p1, static_cast<S*>(st.c2v), q.yt,
                                                            static_cast<const float*>(st.chan_mag), st.zt, st.active,
                                                            st.n_tiles, float(l_max));
      else if (rm_in)
        cn_pair_kernel<S, DMAX, true><<<pgrid, 256, 0, s>>>(c, q.p0, q.p1, q.first_iter, static_cast<S*>(st.c2v),
                                                            static_cast<const float*>(q.lsrc), st.zt, st.active,
                                                            st.n_tiles, float(l_max), rm_in, st.rsgn, st.yt,
                                                            st.counters);
      else
        cn_pair_kernel<S, DMAX, false><<<pgrid, 256, 0, s>>>(c, q.p0, q.p1, q.first_iter, static_cast<S*>(st.c2v),
                                                             static_cast<const float*>(q.lsrc), st.zt, st.active,
                                                             st.n_tiles, float(l_max), nullptr, nullptr, nullptr,
                                                             st.counters);
      return;
    }
  }
  if constexpr (!FIXED && DMAX <= 32) {
    if (q.first_iter && q.yt && rule == MBP_RULE_SUM_PRODUCT) {
      cn_first_kernel<M, S, DMAX><<<grid, 256, 0, s>>>(c, q.p0, q.p1, static_cast<S*>(st.c2v), q.yt,
                                                       static_cast<const M*>(st.chan_mag), st.zt, st.active,
                                                       M(l_max));
      return;
    }
  }
  if constexpr (sizeof(M) == 4 && !FIXED) {
    if (rule == MBP_RULE_MIN_SUM) {
      cn_minsum_kernel<S, DMAX><<<grid, 256, 0, s>>>(c, q.p0, q.p1, q.first_iter, static_cast<S*>(st.c2v),
                                                     static_cast<const float*>(q.lsrc), q.yt,
                                                     static_cast<const float*>(st.chan_mag), st.zt, st.active,
                                                     float(l_max));
      return;
    }
  }
  if constexpr (!FIXED && DMAX <= 32) {
    if (rm_in) {
      cn_kernel<M, S, DMAX, false, true><<<cn_grid<S>(q.p1 - q.p0, st.n_tiles), 256, 0, s>>>(
          c, q.p0, q.p1, q.first_iter, static_cast<S*>(st.c2v), static_cast<const M*>(q.lsrc), st.yt,
          static_cast<const M*>(st.chan_mag), st.zt, st.active, st.n_tiles, M(l_max), st.lacc, qscale, rm_in,
          st.rsgn, st.counters);
      return;
    }
  }
  cn_kernel<M, S, DMAX, FIXED><<<cn_grid<S>(q.p1 - q.p0, st.n_tiles), 256, 0, s>>>(
      c, q.p0, q.p1, q.first_iter, static_cast<S*>(st.c2v), static_cast<const M*>(q.lsrc), q.yt,
      static_cast<const M*>(st.chan_mag), st.zt, st.active, st.n_tiles, M(l_max), st.lacc, qscale, nullptr, nullptr,
      st.counters);
}

// Unroll bound at or one above the largest check degree (the last two degrees run without per-edge tests).
template <typename M, typename S, bool FIXED>
void launch_cn_any(const DevCode& c, const DevState& st, const CnLaunch& q, double l_max, float qscale, int rule,
                   cudaStream_t s) {
  const int d = c.max_row_deg;
#define MBP_CN(D) launch_cn<M, S, D, FIXED>(c, st, q, l_max, qscale, rule, s)
  if constexpr (sizeof(M) == 4 && !FIXED) {
    if (d <= 4) MBP_CN(4);
    else if (d <= 6) MBP_CN(6);
    else if (d <= 8) MBP_CN(8);
    else if (d <= 10) MBP_CN(10);
    else if (d <= 12) MBP_CN(12);
    else if (d <= 14) MBP_CN(14);
    else if (d <= 16) MBP_CN(16);
    else if (d <= 18) MBP_CN(18);
    else if (d <= 20) MBP_CN(20);
    else if (d <= 22) MBP_CN(22);
    else if (d <= 24) MBP_CN(24);
    else if (d <= 32) MBP_CN(32);
    else MBP_CN(64);
  } else {
    if (d <= 8) MBP_CN(8);
    else if (d <= 16) MBP_CN(16);
    else if (d <= 32) MBP_CN(32);
    else MBP_CN(64);
  }
#undef MBP_CN
}

// One flooding sum-product iteration of one group without any host synchronisation (the grid kernels of the
// grouped decode): eq. (6) over every row, eq. (2) and the hard decision, and the stopping test; the caller
// retires the finished frames.
// iter: 1, 2, or 0 for any later iteration (iterations 1 and 2 differ in where their messages come from);
// kStopTestOnly: the stopping test before iteration 1.
template <typename M, typename S>
cudaError_t group_step(const DevCode& c, const DevState& st, int iter, double l_max, cudaStream_t s,
                       const StreamFork* fork = nullptr) {
  const bool rows = rows_ok(c, st);
  if (iter == kStopTestOnly) {  // with the row form, the sign words of iteration 1 and the test together
    if (rows) launch_first_rows_any(c, st, st.fail, s);
    else launch_syn_any(c, st, s);
    return cudaGetLastError();
  }
  // iteration 1 in row form follows the stopping test, which formed the rows' sign words (rows = 3)
  const CnLaunch q{0, c.m_tot, iter == 1, iter == 1 ? st.lp : st.lv, st.yt, rows ? (iter == 1 ? 3 : iter == 2 ? 2 : 0) : 0};
  const int fam = q.rows ? MBP_KERNEL_CHECK_ROWS : MBP_KERNEL_CHECK;
  prof_begin(fam, s);
  launch_cn_any<M, S, false>(c, st, q, l_max, 0.f, MBP_RULE_SUM_PRODUCT, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  prof_end(fam, s, q.rows == 1 ? 2 : 1);
  prof_begin(MBP_KERNEL_VARIABLE, s);
  launch_vn<M, S>(c, st, rows && iter == 1, s, fork);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  prof_end(MBP_KERNEL_VARIABLE, s, c.n_vclass > 0 ? c.n_vclass : 1);
  prof_begin(MBP_KERNEL_SYNDROME, s);
  launch_syn_any(c, st, s);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  prof_end(MBP_KERNEL_SYNDROME, s, 1);
  return cudaSuccess;
}

template <typename M, typename S>
int run(const DevCode& c, DevState& st, const DecodeArgs& a, bool fixed, double l_max, float qscale,
                      float inv_qscale, cudaStream_t s) {
  cudaError_t e;
#define CK(call, what) \
  if ((e = (call)) != cudaSuccess) return cuda_error(e, what)
#define CKL(what) CK(cudaGetLastError(), what)
  const int F = st.F, NT = st.n_tiles;
  const dim3 node_grid(blocks_for(c.n, 8), NT);
  int32_t host_ctr[1];
  // tested: the syndrome test already ran (folded into the first row-form kernel before iteration 1)
  auto stop_check = [&](int t, int* left, bool tested = false) -> int {
    if (!tested) {
      prof_begin(MBP_KERNEL_SYNDROME, s);
      launch_syn_any(c, st, s);
      CKL("syn_kernel");
      prof_end(MBP_KERNEL_SYNDROME, s, 1);
    }
    CK(cudaMemsetAsync(st.counters, 0, sizeof(int32_t), s), "clear counter");
    prof_begin(MBP_KERNEL_RETIRE, s);
    update_kernel<<<blocks_for(NT, 128), 128, 0, s>>>(F, NT, c.u, t, a.max_iter, a.early_exit, st.active, st.fail,
                                                       a.iters, a.success, a.synd_ok, st.perm, st.counters);
    CKL("update_kernel");
    prof_end(MBP_KERNEL_RETIRE, s, 1);
    CK(cudaMemcpyAsync(host_ctr, st.counters, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "read counter");
    CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    *left = host_ctr[0];
    return MBP_OK;
  };
  int left = NT;
  int rc;
  const bool serial0 = a.update == MBP_UPDATE_MATRIX_SERIAL && c.u > 1;
  // iteration 1 in row form: its rows' sign words come with the stopping test before it (rows0)
  const bool rows0 = !fixed && !serial0 && a.rule == MBP_RULE_SUM_PRODUCT && rows_ok(c, st) && a.max_iter > 0;
  if (rows0) {
    prof_begin(MBP_KERNEL_CHECK_ROWS, s);
    launch_first_rows_any(c, st, a.early_exit ? st.fail : nullptr, s);
    CKL("first_rows_kernel");
    prof_end(MBP_KERNEL_CHECK_ROWS, s, 1);
    if (a.early_exit && (rc = stop_check(0, &left, true))) return rc;
  } else if (a.early_exit || a.max_iter == 0) {
    if ((rc = stop_check(0, &left))) return rc;
  }
  auto variable = [&](bool rows) -> int {
    prof_begin(MBP_KERNEL_VARIABLE, s);
    if (fixed)
      finalize_kernel<M><<<node_grid, 256, 0, s>>>(c, st.lacc, static_cast<M*>(st.lv), static_cast<const M*>(st.lp),
                                                   st.yt, static_cast<const M*>(st.chan_mag), st.xh, st.active,
                                                   inv_qscale);
    else
      launch_vn<M, S>(c, st, rows, s);
    CKL("vn_kernel");
    prof_end(MBP_KERNEL_VARIABLE, s, fixed || c.n_vclass == 0 ? 1 : c.n_vclass);
    return MBP_OK;
  };
  auto check = [&](const CnLaunch& q) -> int {
    const int fam = q.rows ? MBP_KERNEL_CHECK_ROWS : MBP_KERNEL_CHECK;
    prof_begin(fam, s);
    if constexpr (sizeof(M) == 4 && sizeof(S) == 4) {
      if (fixed) launch_cn_any<M, S, true>(c, st, q, l_max, qscale, a.rule, s);
      else launch_cn_any<M, S, false>(c, st, q, l_max, qscale, a.rule, s);
    } else {
      launch_cn_any<M, S, false>(c, st, q, l_max, qscale, a.rule, s);
    }
    CKL("cn_kernel");
    prof_end(fam, s, q.rows == 1 ? 2 : 1);
    return MBP_OK;
  };
  const bool serial = a.update == MBP_UPDATE_MATRIX_SERIAL && c.u > 1;
  const bool rows = !fixed && !serial && a.rule == MBP_RULE_SUM_PRODUCT && rows_ok(c, st);
  if (serial && a.max_iter > 0 && left > 0)  // matrices not yet visited in iteration 1 contribute 0 to eq. (2)
    CK(cudaMemsetAsync(st.c2v, 0, msg_tiles(NT, sizeof(S)) * c.s_tot * kLanes * sizeof(S), s), "clear messages");
  for (int t = 1; t <= a.max_iter && left > 0; ++t) {
    if (serial) {
      // Algorithm 1's nesting: each matrix's checks, then eq. (2) with its new messages, before the next matrix
      for (int l = 0; l < c.u; ++l) {
        const bool from_lp = t == 1 && l == 0;
        const CnLaunch q{c.row_pos[l], c.row_pos[l + 1], t == 1, from_lp ? st.lp : st.lv, from_lp ? st.yt : nullptr,
                         0};
        if ((rc = check(q))) return rc;
        if ((rc = variable(false))) return rc;
      }
    } else {
      const CnLaunch q{0, c.m_tot, t == 1, t == 1 ? st.lp : st.lv, st.yt, rows ? (t == 1 ? 3 : t == 2 ? 2 : 0) : 0};
      if ((rc = check(q))) return rc;
      if ((rc = variable(rows && t == 1))) return rc;
    }
    if (a.early_exit || t == a.max_iter) {
      if ((rc = stop_check(t, &left))) return rc;
    }
  }
#undef CKL
#undef CK
  return MBP_OK;
}

}  // namespace stream
}  // namespace
}  // namespace mbp
