// Kernels of the grouped decode (see mbp_multi.h): persistent check-node,
// variable-node and syndrome kernels over the device-built lists of unfinished
// tiles, and the single-block kernel that retires frames and rebuilds the lists.
//
// S is the stored message type (float, __half or __nv_bfloat16); arithmetic is
// float. Each S is instantiated in a file of its own (mbp_multi_<type>.cu).
#pragma once

#include <algorithm>

#include "mbp_device.cuh"
#include "mbp_multi.h"

namespace mbp {
namespace {  // every file that includes this keeps its own copies
namespace multi {

using namespace dev;

// The entry e of a list with pre[e] <= r < pre[e + 1] (pre[0] = 0 <= r < pre[n]):
// the largest e with pre[e] <= r, so entries without rows are skipped.
__device__ __forceinline__ int locate(const int64_t* __restrict__ pre, int n, int64_t r) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(pre + mid) <= r) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// From entry e (pre[e] <= r) forward to the entry that holds position r.
__device__ __forceinline__ int advance(const int64_t* __restrict__ pre, int e, int64_t r) {
  while (__ldg(pre + e + 1) <= r) ++e;
  return e;
}

// Check rows of every unfinished tile of one degree class, one warp per row;
// warp w of the grid takes positions w, w + W, w + 2W, ... of the class's rows
// (tiles one after another, rows in degree order inside a tile).
// Blocks of at most 256 threads; rows of up to 16 edges are held to 64 registers (4 blocks of 256 per SM, as
// the streaming kernel), longer rows keep more registers.
constexpr int cn_max_threads(int) { return 256; }
constexpr int cn_min_blocks(int dmax) { return dmax <= 16 ? 4 : 1; }

template <typename S, int DMAX>
__global__ void __launch_bounds__(cn_max_threads(DMAX), cn_min_blocks(DMAX)) cn_multi_kernel(const MultiGroup* __restrict__ gr,
                                                       const MultiCtl* __restrict__ ctl,
                                                       const int32_t* __restrict__ tile_group,
                                                       const int32_t* __restrict__ list,
                                                       const int64_t* __restrict__ pre, int cls) {
  const int n_ent = ctl->n_ent[cls];
  if (n_ent == 0) return;
  const int64_t total = __ldg(pre + n_ent);
  const int wpb = blockDim.x >> 5;
  const int64_t stride = int64_t(gridDim.x) * wpb;
  int64_t r = int64_t(blockIdx.x) * wpb + (threadIdx.x >> 5);
  if (r >= total) return;
  const int first_iter = ctl->t == 1;
  const float l_max = ctl->l_max, d_lmax = Arith<float>::delta(l_max);
  int e = locate(pre, n_ent, r), cur = -1;
  int64_t row0 = 0;
  CnView<float, S> v;
  for (; r < total; r += stride) {
    e = advance(pre, e, r);
    if (e != cur) {  // a new tile: its view stays in registers while the warp works on its rows
      cur = e;
      row0 = __ldg(pre + e);
      const int gt = __ldg(list + e);
      const MultiGroup& G = gr[__ldg(tile_group + gt)];
      const int tile = gt - G.tile_base;
      v = cn_view<float, S, kPolStream>(G.c, tile, G.st.active[tile], first_iter, static_cast<S*>(G.st.c2v),
                                        static_cast<const float*>(first_iter ? G.st.lp : G.st.lv), G.st.yt,
                                        static_cast<const float*>(G.st.chan_mag), G.st.zt, nullptr);
    }
    cn_view_row<float, S, DMAX, false, kPolStream>(v, int(r - row0), first_iter, l_max, d_lmax, 0.f);
  }
}

// Variable nodes (eq. 2 and the hard decision) of every unfinished tile.
template <typename S>
__global__ void __launch_bounds__(256, 6) vn_multi_kernel(const MultiGroup* __restrict__ gr,
                                                       const MultiCtl* __restrict__ ctl,
                                                       const int32_t* __restrict__ tile_group,
                                                       const int32_t* __restrict__ list,
                                                       const int64_t* __restrict__ pre) {
  const int n_ent = ctl->n_all;
  if (n_ent == 0) return;
  const int64_t total = __ldg(pre + n_ent);
  const int wpb = blockDim.x >> 5;
  const int64_t stride = int64_t(gridDim.x) * wpb;
  int64_t r = int64_t(blockIdx.x) * wpb + (threadIdx.x >> 5);
  if (r >= total) return;
  int e = locate(pre, n_ent, r), cur = -1;
  int64_t node0 = 0;
  VnView<float, S> v;
  for (; r < total; r += stride) {
    e = advance(pre, e, r);
    if (e != cur) {
      cur = e;
      node0 = __ldg(pre + e);
      const int gt = __ldg(list + e);
      const MultiGroup& G = gr[__ldg(tile_group + gt)];
      const int tile = gt - G.tile_base;
      v = vn_view<float, S, kPolStream>(G.c, tile, G.st.active[tile], static_cast<const S*>(G.st.c2v),
                                        static_cast<float*>(G.st.lv), static_cast<const float*>(G.st.lp), G.st.yt,
                                        static_cast<const float*>(G.st.chan_mag), G.st.xh, G.st.n_tiles);
    }
    vn_view_node<float, S, kPolStream>(v, int(r - node0));
  }
}

// The stopping test of one degree class, 32 rows per warp (positions count
// groups of 32 rows of a tile). Runs only when its result is used.
template <int DMAX>
__global__ void __launch_bounds__(512) syn_multi_kernel(const MultiGroup* __restrict__ gr,
                                                        const MultiCtl* __restrict__ ctl,
                                                        const int32_t* __restrict__ tile_group,
                                                        const int32_t* __restrict__ list,
                                                        const int64_t* __restrict__ pre, int cls) {
  if (!ctl->early_exit && ctl->t != ctl->max_iter) return;
  const int n_ent = ctl->n_ent[cls];
  if (n_ent == 0) return;
  const int64_t total = __ldg(pre + n_ent);
  const int wpb = blockDim.x >> 5;
  const int64_t stride = int64_t(gridDim.x) * wpb;
  int64_t r = int64_t(blockIdx.x) * wpb + (threadIdx.x >> 5);
  if (r >= total) return;
  int e = locate(pre, n_ent, r);
  for (; r < total; r += stride) {
    e = advance(pre, e, r);
    const int gt = __ldg(list + e);
    const MultiGroup& G = gr[__ldg(tile_group + gt)];
    const int tile = gt - G.tile_base;
    const uint32_t act = G.st.active[tile];
    syn_rows<DMAX, kPolStream>(G.c, tile, int(r - __ldg(pre + e)) * 32, act, G.st.xh, G.st.n_tiles, G.st.zt,
                               G.st.fail);
  }
}

// Exclusive block-wide prefix sum of v (blockDim.x = 1024); *total gets the sum.
__device__ __forceinline__ int64_t block_exclusive_scan(int64_t v, int64_t* sh, int64_t* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(kFull, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) sh[warp] = x;
  __syncthreads();
  if (warp == 0) {
    int64_t w = lane < int(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int64_t y = __shfl_up_sync(kFull, w, o);
      if (lane >= o) w += y;
    }
    sh[lane] = w;  // inclusive sums of the warp totals
  }
  __syncthreads();
  const int64_t before = (warp > 0 ? sh[warp - 1] : 0) + x - v;
  *total = sh[(blockDim.x >> 5) - 1];
  __syncthreads();
  return before;
}

// Pack a list position count (bits 47..62) and a row / node count (bits 0..46)
// so one scan gives both: a batch has fewer than 2^16 tiles, and fewer than
// 2^16 tiles of fewer than 2^31 rows each hold fewer than 2^47 rows.
constexpr int kCountShift = 47;
constexpr int64_t kValueMask = (int64_t(1) << kCountShift) - 1;
constexpr int64_t kOne = int64_t(1) << kCountShift;

// One block of 1024 threads. retire = 1: close iteration ctl->t (retire the
// lanes that satisfied every syndrome, or all lanes at max_iter), advance t and
// set the loop condition (also the WHILE node's, inside a graph). retire = 0:
// only build the lists of the tiles still active. retire = 2: retire and set
// the conditions without rebuilding the lists (the grid kernels need none). Lists follow global tile
// order: list k (k < n_cls) holds the unfinished tiles of class k with prefix
// sums of their rows (pre[k]) and syndrome warps (pre[n_cls + k]); list n_cls
// holds every unfinished tile with prefix sums of its nodes (pre[2 n_cls]).
__global__ void __launch_bounds__(1024) lists_kernel(MultiGroup* __restrict__ gr, MultiCtl* __restrict__ ctl,
                                                     const int32_t* __restrict__ tile_group, int T, int n_cls,
                                                     int32_t* __restrict__ lists, int64_t* __restrict__ pre,
                                                     int retire, int in_graph, unsigned long long cond_handle,
                                                     const __grid_constant__ GroupConds gc) {
  __shared__ int64_t sh[32];
  __shared__ int g_active[kMaxGroups];  // groups with an unfinished tile (for the per-group conditions)
  for (int g = threadIdx.x; g < gc.n; g += blockDim.x) g_active[g] = 0;
  __shared__ int64_t carry[kMaxClasses + 1];  // class k: count << 47 | rows; [n_cls]: count << 47 | nodes
  __shared__ int64_t carry_syn[kMaxClasses];
  const int t = ctl->t, max_iter = ctl->max_iter, early = ctl->early_exit;
  if (threadIdx.x <= kMaxClasses) carry[threadIdx.x] = 0;
  if (threadIdx.x < kMaxClasses) carry_syn[threadIdx.x] = 0;
  __syncthreads();
  const size_t Tp = size_t(T) + 1;
  for (int base = 0; base < T; base += blockDim.x) {
    const int gt = base + threadIdx.x;
    uint32_t act = 0;
    int cls = -1, rows = 0, synw = 0, nodes = 0;
    if (gt < T) {
      MultiGroup& G = gr[tile_group[gt]];
      const int tile = gt - G.tile_base;
      act = retire ? update_tile(tile, G.st.F, G.c.u, t, max_iter, early, G.st.active, G.st.fail, G.iters,
                                 G.success, G.synd_ok, G.st.perm)
                   : G.st.active[tile];
      if (act) {
        if (gc.n) g_active[tile_group[gt]] = 1;
        cls = G.cls;
        rows = G.c.m_tot;
        synw = (G.c.m_tot + 31) >> 5;
        nodes = G.c.n;
      }
    }
    if (retire == 2) {  // no lists: only whether anything is left
      if (__syncthreads_or(act != 0) && threadIdx.x == 0) carry[n_cls] |= kOne;
      continue;
    }
    for (int k = 0; k <= n_cls; ++k) {
      const bool all = k == n_cls;
      const bool mine = all ? act != 0 : cls == k;
      int64_t tot_a = 0, tot_b = 0;
      const int64_t a = block_exclusive_scan(mine ? kOne | (all ? nodes : rows) : 0, sh, &tot_a);
      const int64_t b = all ? 0 : block_exclusive_scan(mine ? synw : 0, sh, &tot_b);
      if (mine) {
        const int64_t ca = carry[k];
        const int idx = int((ca >> kCountShift) + (a >> kCountShift));
        lists[size_t(k) * T + idx] = gt;
        pre[size_t(all ? 2 * n_cls : k) * Tp + idx] = (ca & kValueMask) + (a & kValueMask);
        if (!all) pre[size_t(n_cls + k) * Tp + idx] = carry_syn[k] + b;
      }
      __syncthreads();
      if (threadIdx.x == 0) {
        carry[k] += tot_a;
        if (!all) carry_syn[k] += tot_b;
      }
      __syncthreads();
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int k = 0; k <= n_cls && retire != 2; ++k) {
      const bool all = k == n_cls;
      const int cnt = int(carry[k] >> kCountShift);
      pre[size_t(all ? 2 * n_cls : k) * Tp + cnt] = carry[k] & kValueMask;
      if (all) {
        ctl->n_all = cnt;
      } else {
        pre[size_t(n_cls + k) * Tp + cnt] = carry_syn[k];
        ctl->n_ent[k] = cnt;
      }
    }
    if (retire) {
      const int t_next = t + 1;
      const int cond = (carry[n_cls] >> kCountShift) > 0 && t_next <= max_iter;
      ctl->t = t_next;
      ctl->cond = cond;
      if (in_graph) cudaGraphSetConditional(cond_handle, unsigned(cond));
    }
  }
  if (gc.n) {
    __syncthreads();
    for (int g = threadIdx.x; g < gc.n; g += blockDim.x)
      if (gc.h[g] != ~0ull) cudaGraphSetConditional(gc.h[g], unsigned(g_active[g]));  // ~0: group without frames
  }
}

// Persistent launch: (resident blocks per SM / waves) x SMs blocks.
template <typename... P, typename... A>
cudaError_t persist(void (*kern)(P...), int threads, int waves, int sms, cudaStream_t s, A... args) {
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kern);
  if (e != cudaSuccess) return e;
  if (threads > fa.maxThreadsPerBlock) threads = fa.maxThreadsPerBlock & ~31;  // the kernel's launch bound
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, 0);
  if (e != cudaSuccess) return e;
  int blocks = per_sm * sms / (waves > 1 ? waves : 1);
  if (blocks < 1) blocks = 1;
  kern<<<blocks, threads, 0, s>>>(args...);
  return cudaGetLastError();
}

}  // namespace multi
}  // namespace

template <typename S>
cudaError_t MultiLaunch<S>::build_lists(const MultiTables& tb, const MultiShape& sh, int retire, int in_graph,
                                        unsigned long long cond_handle, const GroupConds& gc, cudaStream_t s) {
  multi::lists_kernel<<<1, 1024, 0, s>>>(tb.groups, tb.ctl, tb.tile_group, sh.T, sh.n_cls, tb.lists, tb.pre, retire,
                                         in_graph, cond_handle, gc);
  return cudaGetLastError();
}

template <typename S>
cudaError_t MultiLaunch<S>::check(const MultiTables& tb, const MultiShape& sh, int cls, const MultiTuning& tu,
                                  int sms, cudaStream_t s) {
  const int32_t* list = tb.lists + size_t(cls) * sh.T;
  const int64_t* pre = tb.pre + size_t(cls) * (sh.T + 1);
  const int threads = 32 * tu.cn_warps;
#define MBP_CN(D)                                                                                            \
  case D:                                                                                                    \
    return multi::persist(multi::cn_multi_kernel<S, D>, std::min(threads, multi::cn_max_threads(D)),         \
                          tu.cn_waves, sms, s, tb.groups,                                                     \
                          static_cast<const MultiCtl*>(tb.ctl), static_cast<const int32_t*>(tb.tile_group),   \
                          list, pre, cls)
  switch (sh.cls_dmax[cls]) {
    MBP_CN(4);
    MBP_CN(6);
    MBP_CN(8);
    MBP_CN(10);
    MBP_CN(12);
    MBP_CN(14);
    MBP_CN(16);
    MBP_CN(18);
    MBP_CN(20);
    MBP_CN(22);
    MBP_CN(24);
    MBP_CN(32);
    MBP_CN(64);
    default: return cudaErrorInvalidValue;
  }
#undef MBP_CN
}

template <typename S>
cudaError_t MultiLaunch<S>::variable(const MultiTables& tb, const MultiShape& sh, const MultiTuning& tu, int sms,
                                     cudaStream_t s) {
  const int32_t* list = tb.lists + size_t(sh.n_cls) * sh.T;
  const int64_t* pre = tb.pre + size_t(2 * sh.n_cls) * (sh.T + 1);
  return multi::persist(multi::vn_multi_kernel<S>, 32 * tu.vn_warps, 1, sms, s, tb.groups,
                        static_cast<const MultiCtl*>(tb.ctl), static_cast<const int32_t*>(tb.tile_group), list, pre);
}

template <typename S>
cudaError_t MultiLaunch<S>::syndrome(const MultiTables& tb, const MultiShape& sh, int cls, const MultiTuning& tu,
                                     int sms, cudaStream_t s) {
  const int32_t* list = tb.lists + size_t(cls) * sh.T;
  const int64_t* pre = tb.pre + size_t(sh.n_cls + cls) * (sh.T + 1);
  const int threads = 32 * tu.syn_warps;
  const int d = sh.cls_dmax[cls];
  const MultiCtl* ctl = tb.ctl;
  const int32_t* tg = tb.tile_group;
  if (d <= 8) return multi::persist(multi::syn_multi_kernel<8>, threads, 1, sms, s, tb.groups, ctl, tg, list, pre, cls);
  if (d <= 16) return multi::persist(multi::syn_multi_kernel<16>, threads, 1, sms, s, tb.groups, ctl, tg, list, pre, cls);
  if (d <= 32) return multi::persist(multi::syn_multi_kernel<32>, threads, 1, sms, s, tb.groups, ctl, tg, list, pre, cls);
  return multi::persist(multi::syn_multi_kernel<kMaxRowDeg>, threads, 1, sms, s, tb.groups, ctl, tg, list, pre, cls);
}

}  // namespace mbp
