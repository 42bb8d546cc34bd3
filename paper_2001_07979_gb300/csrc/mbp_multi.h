// Internal declarations of the grouped decode (mbp_decode_multi and the
// MBP_SCHED_GRAPH schedule of the single-code entry points).
//
// A batch holds G groups; group g decodes F_g frames of its own code (n, R, u
// and QBER may all differ between groups) in the same interleaved layout as a
// single-code decode (tiles of kLanes frames). Tiles of all groups are numbered
// together ("global tiles"). Each iteration:
//   * one check-node kernel per degree class (the unroll bound of eq. 6 that
//     the group's largest check degree selects) over a device-built list of the
//     unfinished tiles of that class;
//   * one variable-node kernel (eq. 2) over every unfinished tile;
//   * one syndrome kernel per class (the stopping rule);
//   * one single-block retire kernel that retires finished frames, rebuilds the
//     lists with prefix sums of the rows / nodes they hold, advances the
//     iteration counter and decides whether another iteration runs.
// The kernels are persistent: a grid of (SMs x resident blocks), each warp
// stepping through the list's rows (or nodes) with a stride of all warps of
// the grid, so that the warps move together over one tile at a time (its
// posteriors stay in L2) and the work of an iteration is proportional to the
// frames still decoding. Alternatively ("grid kernels") each group runs the
// streaming schedule's kernels (one block per 8 rows or nodes of every tile;
// finished tiles' blocks return at once); the autotuner picks the faster of
// the two. The loop runs inside a CUDA graph whose WHILE node
// is driven by the retire kernel (no host round trip per iteration), or from
// the host (one launch per kernel and a read-back per iteration) when kernel
// accounting is on.
#pragma once

#include "mbp_internal.h"

namespace mbp {

constexpr int kMaxGroups = 256;
constexpr int kMaxClasses = 8;  // distinct check-degree classes in one batch

// Device-resident description of one group (in the workspace).
struct MultiGroup {
  DevCode c;
  DevState st;        // the group's decoder state (carved from the batch workspace)
  int32_t tile_base;  // global index of the group's first tile
  int32_t cls;        // degree class slot (0 .. n_cls - 1)
  // per-call outputs written by the retire kernel
  int32_t* iters;
  uint8_t* success;
  uint8_t* synd_ok;
};

// Control block of a batch (in the workspace).
struct MultiCtl {
  int32_t t;           // iteration the next retire kernel closes (0 = the test before iteration 1)
  int32_t max_iter;
  int32_t early_exit;
  int32_t cond;        // 1 while another iteration is to run (also the WHILE node's condition)
  int32_t n_all;       // unfinished tiles (entries of the variable-node list)
  int32_t n_ent[kMaxClasses];
  float l_max;  // clip in the decoder's internal LLR unit
};

// Launch shapes chosen by the autotuner (or the defaults).
struct MultiTuning {
  int32_t grid;         // 1: per-group grid kernels (the streaming schedule's), 0: persistent list kernels
  int32_t cn_warps;     // warps per block of the check-node kernels (2, 4 or 8)
  int32_t cn_waves;     // resident blocks per SM used, as a fraction of the maximum: 1 = all, 2 = half
  int32_t vn_warps;     // warps per block of the variable-node kernel
  int32_t syn_warps;    // warps per block of the syndrome kernels
};

// Device pointers of a batch's tables (all inside the workspace).
struct MultiTables {
  MultiGroup* groups;   // [G]
  MultiCtl* ctl;
  int32_t* tile_group;  // [T] group of each global tile
  int32_t* lists;       // [n_cls + 1][T]: class lists, then the all-tiles list
  int64_t* pre;         // [2 n_cls + 1][T + 1]: rows per class, syndrome warps per class, nodes (all)
};

// The conditions of the per-group IF nodes of a graph (grid kernels): group g's step runs while it has
// unfinished tiles. n = 0: no per-group conditions.
struct GroupConds {
  int32_t n;
  unsigned long long h[kMaxGroups];
};

struct MultiShape {
  int G, T, n_cls;
  int cls_dmax[kMaxClasses];  // unroll bound of each class slot
};

// kernels of one stored message type S (arithmetic in float), in mbp_multi_<type>.cu
template <typename S>
struct MultiLaunch {
  static cudaError_t build_lists(const MultiTables& tb, const MultiShape& sh, int retire, int in_graph,
                                 unsigned long long cond_handle, const GroupConds& gc, cudaStream_t s);
  static cudaError_t check(const MultiTables& tb, const MultiShape& sh, int cls, const MultiTuning& tu, int sms,
                           cudaStream_t s);
  static cudaError_t variable(const MultiTables& tb, const MultiShape& sh, const MultiTuning& tu, int sms,
                              cudaStream_t s);
  static cudaError_t syndrome(const MultiTables& tb, const MultiShape& sh, int cls, const MultiTuning& tu, int sms,
                              cudaStream_t s);
};

// degree class (unroll bound) of a code with largest check degree d
int multi_class_dmax(int d);

// set-up and output kernels of one group (mbp_kernels.cu), shared with the single-code driver
int group_setup(const DevCode& c, DevState& st, int msg_dtype, const DecodeArgs& a, cudaStream_t s);
int group_output(const DevCode& c, DevState& st, int msg_dtype, const DecodeArgs& a, cudaStream_t s);
void group_layout(const DevCode& c, int F, int msg_dtype, size_t* bytes);

// driver (mbp_multi.cpp); arguments validated by the entry points
int multi_check_opts(const mbp_opts* o);
int multi_workspace(const mbp_group* g, int G, const mbp_opts* o, bool host_io, size_t* bytes);
int multi_group_state(const mbp_group* g, int G, int index, const mbp_opts* o, bool host_io, DevState* st);
int multi_decode(const mbp_group* g, int G, int max_iter, const mbp_opts* o, bool host_io, cudaStream_t s);
int multi_autotune(const mbp_group* g, int G, int max_iter, const mbp_opts* o, mbp_tuning* best, cudaStream_t s);
int multi_set_tuning(const mbp_group* g, int G, const mbp_opts* o, const mbp_tuning* t);
void multi_release();
// Drop the cached graphs and tunings that name this code (before its handle is freed).
void multi_forget(const mbp_codes* h);

}  // namespace mbp
