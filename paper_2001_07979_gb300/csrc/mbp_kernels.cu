// Set-up and output kernels, eq. (1) and eq. (5), the decode driver and the
// workspace layout of libmbp (sm_103a). The iterations themselves run in
// mbp_stream.cu (one kernel per step and iteration) or mbp_resident.cu (one
// cooperative launch); both use the building blocks of mbp_device.cuh.
//
// Frames are interleaved kLanes = 32 per tile: every per-edge or per-node
// array holds the tile's 32 frames of one edge or node contiguously, and hard
// decisions and syndrome bits are 32-bit words with one bit per frame.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <mutex>

#include "mbp_device.cuh"
#include "mbp_multi.h"

// Fixed device scratch of mbp_decode_bsc_static: the decoder state of one call,
// for callers that must not allocate. Every GPU that loads this library holds
// these bytes until the process exits; every call shares them.
static __device__ __align__(256) unsigned char g_static_scratch[MBP_STATIC_SCRATCH_BYTES];

namespace mbp {
namespace {

using namespace dev;

inline unsigned blocks_for(int64_t n, int per) { return unsigned((n + per - 1) / per); }

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

// ln((1 - e)/e) per frame in double precision, times `unit` (the decoder's
// internal LLR unit), rounded once to M; one value per (tile, lane), 0 for the
// lanes past the last frame.
template <typename M>
__global__ void chan_mag_kernel(const double* __restrict__ qber, int F, int n_lanes, double unit,
                                M* __restrict__ mag, const int32_t* __restrict__ perm) {
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n_lanes) return;
  M v = M(0);
  if (f < F) {
    const double e = qber[perm[f]];
    v = M(log((1.0 - e) / e) * unit);
  }
  mag[f] = v;
}

// ------------------------------------------------------------- set-up

// Batches up to this many frames are ordered by QBER (the rank of every frame is
// counted over all frames: F^2 comparisons, under a millisecond at this size);
// larger ones keep the caller's order.
constexpr int kOrderMax = 1 << 16;

// The frame held by each slot (perm) and the slot of each frame (slot_of). With
// per-frame QBERs, slots follow ascending QBER, ties in frame order (a stable
// order over the doubles' bit patterns mapped to a total order, so that every
// input gives a permutation); otherwise, and for F > kOrderMax, slot = frame.
// Slots past F hold themselves. One warp per slot index f: the lanes compare
// frame f's key with every 32nd frame's and the ballots' population counts add
// up to f's rank.
__global__ void __launch_bounds__(256) frame_order_kernel(const double* __restrict__ qber, int F, int n_slots,
                                                          int32_t* __restrict__ perm, int32_t* __restrict__ slot_of) {
  const int f = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (f >= n_slots) return;
  if (f >= F || qber == nullptr || F > kOrderMax) {
    if (lane == 0) {
      perm[f] = f;
      if (f < F) slot_of[f] = f;
    }
    return;
  }
  auto key = [](double q) {
    const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(q));
    return (b >> 63) ? ~b : (b | (1ull << 63));
  };
  const unsigned long long kf = key(__ldg(qber + f));
  int rank = 0;
#pragma unroll 8
  for (int g0 = 0; g0 < F; g0 += kLanes) {  // unrolled: several key loads in flight
    const int g = g0 + lane;
    const unsigned long long kg = g < F ? key(__ldg(qber + g)) : ~0ull;
    rank += __popc(__ballot_sync(kFull, g < F && (kg < kf || (kg == kf && g < f))));
  }
  if (lane == 0) {
    perm[rank] = f;
    slot_of[f] = rank;
  }
}

// BSC inputs: Bob's bits into one word per (tile, node) with bit = lane (the
// sign words of L_P = (1 - 2y) mag, eq. 5), and the hard decision of iteration
// 0, [L_P < 0] = y where mag > 0. One warp per (tile, 32-node word): lane l
// reads frame l's word, and a warp bit transpose gives lane b node 32 w + b's
// word.
template <typename M>
__global__ void init_bits_kernel(const DevCode c, int F, const uint32_t* __restrict__ y, const M* __restrict__ mag,
                                 uint32_t* __restrict__ yt, uint32_t* __restrict__ xh, uint32_t* __restrict__ ppos,
                                 const int32_t* __restrict__ perm) {
  const int wn = (c.n + 31) >> 5;
  const int tile = blockIdx.y;
  const int w = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (w >= wn) return;
  const int lane = threadIdx.x & 31;
  const int f = tile * kLanes + lane;
  const uint32_t yw = f < F ? y[int64_t(perm[f]) * wn + w] : 0u;
  const uint32_t pos = __ballot_sync(kFull, mag[tile * kLanes + lane] > M(0));
  if (w == 0 && lane == 0) ppos[tile] = pos;
  const uint32_t word = warp_transpose32(yw);  // lane b: node 32 w + b, bit = frame
  const int i = w * 32 + lane;
  if (i < c.n) {
    yt[int64_t(tile) * c.n + i] = word;
    xh[int64_t(i) * gridDim.y + tile] = word & pos;
  }
}

// General inputs: L_P into the interleaved layout (internal unit) and the hard
// decision of iteration 0. One warp per (tile, variable node), lane = frame.
template <typename M>
__global__ void init_lp_kernel(const DevCode c, int F, const M* __restrict__ llr, M* __restrict__ lp,
                               uint32_t* __restrict__ xh, int32_t* __restrict__ counters, int validate) {
  const int tile = blockIdx.y;
  const int col = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (col >= c.n) return;
  const int lane = threadIdx.x & 31;
  const int f = tile * kLanes + lane;
  M v = M(0);
  if (f < F) {
    v = llr[int64_t(f) * c.n + col];
    if (validate && !isfinite(v)) atomicOr(&counters[1], 1);
    v = M(double(v) * Arith<M>::kToInternal);
  }
  lp[(int64_t(tile) * c.n + col) * kLanes + lane] = v;
  const uint32_t hard = __ballot_sync(kFull, f < F && v < M(0));
  if (lane == 0) xh[int64_t(col) * gridDim.y + tile] = hard;
}

// Alice's syndrome bits into one word per (tile, check row in degree order) with
// bit = lane, tile-major (zt) and row-major (ztt). One warp per (tile, 32-row
// word of one matrix): lane f reads frame f's word, and a warp bit transpose
// gives lane b the word of row 32 g + b of H_l.
__global__ void init_z_kernel(const DevCode c, int F, int n_tiles, const uint32_t* __restrict__ z,
                              uint32_t* __restrict__ zt, uint32_t* __restrict__ ztt, const int32_t* __restrict__ perm) {
  const int tile = blockIdx.y;
  int g = blockIdx.x * 8 + (threadIdx.x >> 5);  // word over all matrices, then within H_l
  int l = 0;
  int64_t off = 0;
  while (l < c.u && g >= ((c.m[l] + 31) >> 5)) {
    const int wl = (c.m[l] + 31) >> 5;
    g -= wl;
    off += int64_t(F) * wl;
    ++l;
  }
  if (l >= c.u) return;
  const int wl = (c.m[l] + 31) >> 5;
  const int lane = threadIdx.x & 31;
  const int f = tile * kLanes + lane;
  const uint32_t word = warp_transpose32(f < F ? z[off + int64_t(perm[f]) * wl + g] : 0u);
  const int j = g * 32 + lane;
  if (j < c.m[l]) {
    const int p = c.row_at[c.row_first[l] + j];
    zt[int64_t(tile) * c.m_tot + p] = word;
    ztt[int64_t(p) * n_tiles + tile] = word;
  }
}

__global__ void init_tiles_kernel(int F, int n_tiles, int u, uint32_t* __restrict__ active,
                                  uint32_t* __restrict__ fail) {
  const int tile = blockIdx.x * blockDim.x + threadIdx.x;
  if (tile >= n_tiles) return;
  const int left = F - tile * kLanes;
  active[tile] = left >= kLanes ? kFull : ((1u << left) - 1u);
  for (int l = 0; l < u; ++l) fail[tile * u + l] = 0;
}

// ------------------------------------------------------------- outputs

// One warp per (tile, 32-node word): lane i reads node 32 w + i's decision word
// (one bit per frame); a warp bit transpose gives lane f frame f's output word.
__global__ void out_bits_kernel(const DevCode c, int F, const uint32_t* __restrict__ xh, uint32_t* __restrict__ out,
                                const int32_t* __restrict__ perm) {
  const int wn = (c.n + 31) >> 5;
  const int tile = blockIdx.y;
  const int w = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (w >= wn) return;
  const int lane = threadIdx.x & 31;
  const int i = w * 32 + lane;
  const uint32_t word = i < c.n ? xh[int64_t(i) * gridDim.y + tile] : 0u;
  const uint32_t bits = warp_transpose32(word);  // lane f: frame f's bits of nodes 32 w .. 32 w + 31
  const int f = tile * kLanes + lane;
  if (f < F) out[int64_t(perm[f]) * wn + w] = bits;
}

template <typename M>
__global__ void soft_out_kernel(const DevCode c, int F, const M* __restrict__ lv, const M* __restrict__ lp,
                                const uint32_t* __restrict__ yt, const M* __restrict__ ymag,
                                const int32_t* __restrict__ iters, M* __restrict__ out,
                                const int32_t* __restrict__ slot_of) {
  const int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (idx >= int64_t(F) * c.n) return;
  const int f = int(idx / c.n), i = int(idx % c.n);  // the caller's frame f, at slot slot_of[f]
  const int sl = slot_of[f];
  const int tile = sl / kLanes, lane = sl % kLanes;
  const int64_t tn = int64_t(tile) * c.n + i;
  const M v = iters[f] == 0 ? channel_llr<M, kPolStream>(lp, yt, ymag, tn, tile, lane) : lv[tn * kLanes + lane];
  out[idx] = M(v * Arith<M>::kToLLR);
}

// One frame's C2V per stacked CSR edge; when the decode stopped after a
// row-form iteration 1 (flag counters[2]), rebuilt from the rows (row_msg).
template <typename M, typename S>
__global__ void export_c2v_kernel(const DevCode c, const S* __restrict__ c2v, int frame, M* __restrict__ out,
                                  int n_tiles, const M* __restrict__ fmag, const uint32_t* __restrict__ rsgn,
                                  const uint32_t* __restrict__ yt, const int32_t* __restrict__ counters,
                                  const int32_t* __restrict__ slot_of) {
  const int64_t e = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= c.e_tot) return;
  const int sl = slot_of[frame];
  const int tile = sl / kLanes, lane = sl % kLanes;
  const int slot = c.edge_slot[e];
  M v;
  if (counters[2]) {
    int lo = 0, hi = c.m_tot;  // the row position p with slice_base[p] <= slot < slice_base[p + 1]
    while (hi - lo > 1) {
      const int mid = (lo + hi) >> 1;
      if (c.slice_base[mid] <= slot) lo = mid;
      else hi = mid;
    }
    const int deg = c.slice_base[lo + 1] - c.slice_base[lo];
    v = row_msg(fmag[(int64_t(tile) * kMaxRowDeg + deg - 1) * kLanes + lane], rsgn[int64_t(lo) * n_tiles + tile],
                yt[int64_t(tile) * c.n + c.col_idx[e]], lane);
  } else {
    v = M(Store<S>::widen(c2v[msg_at<S>(tile, c.s_tot, lane) + int64_t(slot) * kMsgStride<S>]));
  }
  out[e] = v * Arith<M>::kToLLR;
}

// ------------------------------------------------------------- driver

// Channel LLRs, syndrome words and tile state into the workspace (and the
// non-finite check of validate mode).
template <typename M>
int setup_t(const DevCode& c, DevState& st, const DecodeArgs& a, cudaStream_t s) {
  cudaError_t e;
#define CK(call, what) \
  if ((e = (call)) != cudaSuccess) return cuda_error(e, what)
#define CKL(what) CK(cudaGetLastError(), what)
  const int F = st.F, NT = st.n_tiles;
  CK(cudaMemsetAsync(st.counters, 0, 4 * sizeof(int32_t), s), "clear counters");
  prof_begin(MBP_KERNEL_SETUP, s);
  frame_order_kernel<<<blocks_for(NT * kLanes, 8), 256, 0, s>>>(a.y_bits ? a.qber : nullptr, F, NT * kLanes,
                                                                st.perm, st.slot_of);
  CKL("frame_order_kernel");
  if (a.y_bits) {  // BSC inputs: sign words and per-frame magnitudes, no LLR array
    chan_mag_kernel<M><<<blocks_for(NT * kLanes, 256), 256, 0, s>>>(a.qber, F, NT * kLanes, Arith<M>::kToInternal,
                                                                   static_cast<M*>(st.chan_mag), st.perm);
    CKL("chan_mag_kernel");
    init_bits_kernel<M><<<dim3(blocks_for((c.n + 31) >> 5, 8), NT), 256, 0, s>>>(
        c, F, a.y_bits, static_cast<const M*>(st.chan_mag), st.yt, st.xh, st.ppos, st.perm);
    CKL("init_bits_kernel");
  } else {
    st.yt = nullptr;
    init_lp_kernel<M><<<dim3(blocks_for(c.n, 8), NT), 256, 0, s>>>(c, F, static_cast<const M*>(a.llr),
                                                                   static_cast<M*>(st.lp), st.xh, st.counters,
                                                                   a.validate);
    CKL("init_lp_kernel");
  }
  int zwords = 0;
  for (int l = 0; l < c.u; ++l) zwords += (c.m[l] + 31) >> 5;
  if (zwords > 0)
    init_z_kernel<<<dim3(blocks_for(zwords, 8), NT), 256, 0, s>>>(c, F, NT, a.z_bits, st.zt, st.ztt, st.perm);
  CKL("init_z_kernel");
  init_tiles_kernel<<<blocks_for(NT, 256), 256, 0, s>>>(F, NT, c.u, st.active, st.fail);
  CKL("init_tiles_kernel");
  prof_end(MBP_KERNEL_SETUP, s, a.y_bits ? 5 : 4);
  if (a.validate) {
    int32_t host_ctr[4];
    CK(cudaMemcpyAsync(host_ctr, st.counters, sizeof host_ctr, cudaMemcpyDeviceToHost, s), "read validate flag");
    CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    if (host_ctr[1]) return set_error(MBP_EINVAL, "llr holds a non-finite value");
  }
  return MBP_OK;
}

// Output bits (and soft values) of the frames of one decode.
template <typename M>
int output_t(const DevCode& c, DevState& st, const DecodeArgs& a, cudaStream_t s) {
  cudaError_t e;
  const int F = st.F, NT = st.n_tiles;
  const int wn = (c.n + 31) >> 5;
  prof_begin(MBP_KERNEL_OUTPUT, s);
  out_bits_kernel<<<dim3(blocks_for(wn, 8), NT), 256, 0, s>>>(c, F, st.xh, a.x_hat_bits, st.perm);
  CKL("out_bits_kernel");
  if (a.soft_out) {
    soft_out_kernel<M><<<blocks_for(int64_t(F) * c.n, 256), 256, 0, s>>>(
        c, F, static_cast<const M*>(st.lv), static_cast<const M*>(st.lp), st.yt, static_cast<const M*>(st.chan_mag),
        a.iters, static_cast<M*>(a.soft_out), st.slot_of);
    CKL("soft_out_kernel");
  }
  prof_end(MBP_KERNEL_OUTPUT, s, a.soft_out ? 2 : 1);
  return MBP_OK;
}

template <typename M, typename S>
int decode_t(const DevCode& c, DevState& st, const DecodeArgs& a, cudaStream_t s) {
  cudaError_t e;
  const int NT = st.n_tiles;
  const double l_max = a.l_max * Arith<M>::kToInternal;  // clip in the decoder's internal LLR unit
  // accumulation of eq. (2): fixed-point single pass (FP32 messages) or float two-pass
  int qbits = 0;
  {
    const double bound = double(c.max_col_deg > 0 ? c.max_col_deg : 1) * l_max;
    while (qbits < kMaxQBits && bound * std::ldexp(1.0, qbits + 1) < 2147483647.0) ++qbits;
  }
  const bool fixed_ok = sizeof(M) == 4 && sizeof(S) == 4 && st.lacc && qbits >= kMinQBits;
  if (a.accumulate == MBP_ACC_FIXED && !fixed_ok)
    return set_error(MBP_EUNSUPPORTED, "fixed-point accumulation needs FP32 message storage and max node degree x"
                                       " l_max <= 2^%d", 31 - kMinQBits);
  const bool fixed = fixed_ok && a.accumulate == MBP_ACC_FIXED;
  const float qscale = float(std::ldexp(1.0, qbits)), inv_qscale = float(std::ldexp(1.0, -qbits));
  if (fixed) CK(cudaMemsetAsync(st.lacc, 0, size_t(NT) * c.n * kLanes * sizeof(int32_t), s), "clear accumulator");
  int rc = setup_t<M>(c, st, a, s);
  if (rc) return rc;
  // schedule: resident (one cooperative launch, groups of tiles kept in L2) or streaming (kernels per iteration)
  constexpr bool same_store = sizeof(M) == sizeof(S);
  const int G = (fixed || !same_store || a.schedule != MBP_SCHED_RESIDENT) ? 0 : resident_group<M>(c, NT);
  if (a.schedule == MBP_SCHED_RESIDENT && G == 0)
    return set_error(MBP_EUNSUPPORTED, fixed ? "the resident schedule accumulates in floating point only"
                                       : !same_store ? "the resident schedule stores FP32 or FP64 messages only"
                                             : "one tile of this code does not fit the resident schedule's L2 budget");
  if (G > 0) {
    CK(cudaMemsetAsync(st.ctl, 0, resident_ctl_bytes(), s), "clear resident control");
    prof_begin(MBP_KERNEL_PERSISTENT, s);
    CK(launch_resident_any<M>(c, st, a, G, l_max, s), "resident_kernel (cooperative launch)");
    prof_end(MBP_KERNEL_PERSISTENT, s, 1);
    alignas(8) unsigned char ctl_h[64];
    CK(cudaMemcpyAsync(ctl_h, st.ctl, resident_ctl_bytes(), cudaMemcpyDeviceToHost, s), "read resident control");
    CK(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    if (resident_error(ctl_h)) return set_error(MBP_ETIMEOUT, "a grid barrier of the resident schedule timed out");
  } else {
    rc = stream_iterations<M, S>(c, st, a, fixed, l_max, qscale, inv_qscale, s);
    if (rc) return rc;
  }
  return output_t<M>(c, st, a, s);
#undef CKL
#undef CK
}

constexpr int kRegions = 23;

// bytes of one stored message and of one posterior / channel value
size_t msg_size(int msg_dtype) {
  return msg_dtype == MBP_MSG_F64 ? 8 : (msg_dtype == MBP_MSG_F32 ? 4 : 2);
}
size_t node_size(int msg_dtype) { return msg_dtype == MBP_MSG_F64 ? 8 : 4; }

inline size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

void layout(const DevCode& c, int F, int msg_dtype, bool host_io, size_t* offs, size_t* total) {
  const size_t NT = (size_t(F) + kLanes - 1) / kLanes;
  const size_t ms = msg_size(msg_dtype);
  const size_t wn = (size_t(c.n) + 31) / 32;
  size_t zw = 0;
  for (int l = 0; l < c.u; ++l) zw += (size_t(c.m[l]) + 31) / 32;
  const size_t sizes[kRegions] = {
      msg_tiles(NT, ms) * size_t(c.s_tot) * kLanes * ms,              // c2v
      NT * size_t(c.n) * kLanes * node_size(msg_dtype),               // lv
      NT * size_t(c.n) * kLanes * node_size(msg_dtype),               // lp
      msg_dtype == MBP_MSG_F32 ? NT * size_t(c.n) * kLanes * 4 : 0,  // lacc
      NT * size_t(c.n) * 4,                                           // xh
      NT * size_t(c.m_tot) * 4,                                       // zt
      NT * 4,                                                         // active
      NT * size_t(c.u) * 4,                                           // fail
      NT * kLanes * node_size(msg_dtype),                             // chan_mag
      16,                                                             // counters
      64,                                                             // resident schedule control block
      host_io ? size_t(F) * wn * 4 : 0,                               // io_y
      host_io ? size_t(F) * 8 : 0,                                    // io_qber
      host_io ? size_t(F) * zw * 4 : 0,                               // io_z
      host_io ? size_t(F) * wn * 4 : 0,                               // io_xhat
      host_io ? size_t(F) * 4 : 0,                                    // io_iters
      host_io ? size_t(F) : 0,                                        // io_success
      NT * size_t(c.n) * 4,                                           // yt
      NT * size_t(kMaxRowDeg) * kLanes * node_size(msg_dtype),        // fmag
      NT * size_t(c.m_tot) * 4,                                       // rsgn
      NT * size_t(c.m_tot) * 4,                                       // ztt
      NT * 4,                                                         // ppos
      2 * NT * kLanes * 4,                                            // perm, slot_of
  };
  size_t t = 0;
  for (int i = 0; i < kRegions; ++i) {
    offs[i] = t;
    t += align256(sizes[i]);
  }
  *total = t;
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
  st->xh = reinterpret_cast<uint32_t*>(b + o[4]);
  st->zt = reinterpret_cast<uint32_t*>(b + o[5]);
  st->active = reinterpret_cast<uint32_t*>(b + o[6]);
  st->fail = reinterpret_cast<uint32_t*>(b + o[7]);
  st->chan_mag = b + o[8];
  st->yt = reinterpret_cast<uint32_t*>(b + o[17]);
  st->fmag = b + o[18];
  st->rsgn = reinterpret_cast<uint32_t*>(b + o[19]);
  st->ztt = reinterpret_cast<uint32_t*>(b + o[20]);
  st->ppos = reinterpret_cast<uint32_t*>(b + o[21]);
  st->perm = reinterpret_cast<int32_t*>(b + o[22]);
  st->slot_of = st->perm + int64_t(st->n_tiles) * kLanes;
  st->counters = reinterpret_cast<int32_t*>(b + o[9]);
  st->ctl = b + o[10];
  st->io_y = host_io ? reinterpret_cast<uint32_t*>(b + o[11]) : nullptr;
  st->io_qber = host_io ? reinterpret_cast<double*>(b + o[12]) : nullptr;
  st->io_z = host_io ? reinterpret_cast<uint32_t*>(b + o[13]) : nullptr;
  st->io_xhat = host_io ? reinterpret_cast<uint32_t*>(b + o[14]) : nullptr;
  st->io_iters = host_io ? reinterpret_cast<int32_t*>(b + o[15]) : nullptr;
  st->io_success = host_io ? reinterpret_cast<uint8_t*>(b + o[16]) : nullptr;
}

int group_setup(const DevCode& c, DevState& st, int msg_dtype, const DecodeArgs& a, cudaStream_t s) {
  return msg_dtype == MBP_MSG_F64 ? setup_t<double>(c, st, a, s) : setup_t<float>(c, st, a, s);
}

int group_output(const DevCode& c, DevState& st, int msg_dtype, const DecodeArgs& a, cudaStream_t s) {
  return msg_dtype == MBP_MSG_F64 ? output_t<double>(c, st, a, s) : output_t<float>(c, st, a, s);
}

void group_layout(const DevCode& c, int F, int msg_dtype, size_t* bytes) { *bytes = workspace_bytes(c, F, msg_dtype, false); }

int decode(const DevCode& c, DevState& st, int msg_dtype, const DecodeArgs& a, cudaStream_t s) {
  if (st.n_tiles > 65535) return set_error(MBP_EUNSUPPORTED, "F = %d exceeds %d frames per call", st.F, 65535 * kLanes);
  switch (msg_dtype) {
    case MBP_MSG_F64: return decode_t<double, double>(c, st, a, s);
    case MBP_MSG_F16: return decode_t<float, __half>(c, st, a, s);
    case MBP_MSG_BF16: return decode_t<float, __nv_bfloat16>(c, st, a, s);
    default: return decode_t<float, float>(c, st, a, s);
  }
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
  const unsigned grid = blocks_for(c.e_tot, 256);
#define MBP_EXPORT(M, S)                                                                                     \
  export_c2v_kernel<M, S><<<grid, 256, 0, s>>>(c, static_cast<const S*>(st.c2v), frame, static_cast<M*>(out), \
                                               st.n_tiles, static_cast<const M*>(st.fmag), st.rsgn, st.yt, st.counters, \
                                               st.slot_of)
  if (msg_dtype == MBP_MSG_F64) MBP_EXPORT(double, double);
  else if (msg_dtype == MBP_MSG_F16) MBP_EXPORT(float, __half);
  else if (msg_dtype == MBP_MSG_BF16) MBP_EXPORT(float, __nv_bfloat16);
  else MBP_EXPORT(float, float);
#undef MBP_EXPORT
  return cudaGetLastError();
}

}  // namespace mbp
