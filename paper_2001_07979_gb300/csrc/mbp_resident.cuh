// The resident schedule of libmbp (MBP_SCHED_RESIDENT).
//
// One cooperative launch decodes the whole batch, a group of G tiles at a
// time: every block takes part in every step of the group's iterations
// (eq. 6, eq. 2, the stopping rule and retirement), the steps are separated by
// a grid-wide barrier, and the group's messages and posteriors are meant to
// stay in L2 from one iteration to the next. The barrier wait is bounded: a
// block that waits longer than the limit sets ctl->error and every block
// returns; the host reports MBP_ETIMEOUT.
//
// Templates over the message type M, instantiated in mbp_resident_<type>.cu
// (one file per type so they build in parallel).
#pragma once

#include <cmath>
#include <cstdlib>

#include "mbp_device.cuh"

namespace mbp {
namespace {

using namespace dev;

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
                                                       const uint32_t* __restrict__ yt, const M* __restrict__ ymag,
                                                       uint32_t* __restrict__ xh, const uint32_t* __restrict__ zt,
                                                       uint32_t* __restrict__ active, uint32_t* __restrict__ fail,
                                                       int32_t* __restrict__ iters, uint8_t* __restrict__ success,
                                                       uint8_t* __restrict__ synd_ok,
                                                       const int32_t* __restrict__ perm, ResidentCtl* ctl,
                                                       BarrierCfg bc) {
  unsigned gen = 0;
  const int warps = gridDim.x * (blockDim.x >> 5);
  const int gw = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const M d_lmax = Arith<M>::delta(l_max);
  const int row_groups = (c.m_tot + 31) / 32;
  __shared__ int last_block;

  // syndrome test of the group's hard decisions, then retirement by the last block to finish
  auto stop_test = [&](int g0, int gt, int t) -> bool {
    for (int it = gw; it < gt * row_groups; it += warps) {
      const int tile = g0 + it / row_groups;
      const uint32_t act = __ldcg(active + tile);
      if (act) syn_rows<DMAX, kPolCoherent>(c, tile, (it % row_groups) * 32, act, xh, n_tiles, zt, fail);
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
        any |= update_tile(g0 + i, F, c.u, t, max_iter, early_exit, active, fail, iters, success, synd_ok, perm) != 0;
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
      for (int it = gw; it < gt * c.m_tot; it += warps) {
        const int tile = g0 + it / c.m_tot;
        const uint32_t act = __ldcg(active + tile);
        if (act)
          cn_tile_row<M, M, DMAX, false, kPolCoherent>(c, tile, it % c.m_tot, act, t == 1, c2v, lsrc, yt, ymag, zt,
                                                    l_max, d_lmax, nullptr, 0.f);
      }
      if (!grid_sync(ctl, gen, bc)) return;
      for (int it = gw; it < gt * c.n; it += warps) {
        const int tile = g0 + it / c.n;
        const uint32_t act = __ldcg(active + tile);
        if (act) vn_node<M, M, kPolCoherent>(c, tile, it % c.n, act, c2v, lv, lp, yt, ymag, xh, n_tiles);
      }
      if (!grid_sync(ctl, gen, bc)) return;
      if (early_exit || t == max_iter) {
        if (!stop_test(g0, gt, t)) return;
        if (!*reinterpret_cast<volatile int*>(&ctl->any_active)) break;
      }
    }
  }
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
  const uint32_t* yt = st.yt;
  const M* ymag = static_cast<const M*>(st.chan_mag);
  uint32_t* xh = st.xh;
  const uint32_t* zt = st.zt;
  uint32_t* active = st.active;
  uint32_t* fail = st.fail;
  int32_t* iters = a.iters;
  uint8_t* success = a.success;
  uint8_t* synd_ok = a.synd_ok;
  const int32_t* perm = st.perm;
  ResidentCtl* ctl = static_cast<ResidentCtl*>(st.ctl);
  DevCode cc = c;
  const unsigned grid = unsigned(per_sm * sms);
  BarrierCfg bc{grid, kBarrierTimeout};
  // Test hook for the bounded-wait path: MBP_TEST_BARRIER_EXTRA_ARRIVALS makes every barrier wait for arrivals
  // that never come, and MBP_TEST_BARRIER_TIMEOUT_US shortens the wait limit.
  if (const char* ev = std::getenv("MBP_TEST_BARRIER_EXTRA_ARRIVALS")) bc.arrivals += unsigned(std::atoi(ev));
  if (const char* ev = std::getenv("MBP_TEST_BARRIER_TIMEOUT_US")) bc.timeout = std::atoll(ev) * 2000LL;
  void* args[] = {&cc, &F, &NT, &G, &max_iter, &early_exit, &lm, &c2v, &lv, &lp, &yt, &ymag, &xh, &zt, &active, &fail,
                  &iters, &success, &synd_ok, &perm, &ctl, &bc};
  return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(kern), dim3(grid), dim3(256), args, 0, s);
}

}  // namespace

// Tiles per group: as many as keep the group's messages, posteriors and
// decisions within 3/4 of L2 (0 = one tile does not fit).
template <typename M>
int resident_group(const DevCode& c, int n_tiles) {
  int dev = 0, l2 = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  const double per_tile = double(c.s_tot) * kLanes * sizeof(M) + 2.0 * c.n * kLanes * sizeof(M) +
                          4.0 * (2 * c.n + c.m_tot);
  int g = int(0.75 * l2 / per_tile);
  if (const char* ev = std::getenv("MBP_RESIDENT_GROUP_TILES")) g = std::atoi(ev);  // tuning override
  return g < 1 ? 0 : (g < n_tiles ? g : n_tiles);
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

}  // namespace mbp
