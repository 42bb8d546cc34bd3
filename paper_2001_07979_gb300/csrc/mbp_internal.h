// Internal declarations of libmbp (not part of the C ABI).
//
// Device layout of the stacked code [H_1; ...; H_u] (Section 2: u matrices of
// size m_l x n sharing the n variable nodes):
//   * stacked row r = row_first[l] + j is row j of H_l (the CSR arrays);
//   * for the decoder the rows are put in (matrix, degree) order (position p;
//     matrix l's rows are positions row_pos[l] .. row_pos[l+1] - 1); the row at
//     position p owns the edge "slots" slice_base[p] .. slice_base[p+1] - 1,
//     slot slice_base[p] + k holding its edge k (column slot_col); row_mat and
//     row_local name the matrix and row of each position;
//   * kLanes = 32 frames ("lanes") are interleaved per tile, so that one edge
//     of a tile's frames is one contiguous vector; the tiles 2q and 2q + 1
//     share each message slot (an odd tile count gets an unused partner):
//     FP32 messages as [q][slot][2][lane] (two adjacent 128-byte lines, one
//     per tile), 2-byte messages (FP16/BF16) as [q][slot][lane][2] (one 32-bit
//     word holds a lane's message in both tiles, one 128-byte line per edge);
//     FP64 messages keep [tile][slot][lane] (256 bytes per edge);
//   * col_ptr/col_slot list, for every variable node, the slots of its edges in
//     stacked-row order (the order in which eq. (2) sums them).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>

#include "mbp.h"

namespace mbp {

constexpr int kLanes = 32;      // frames interleaved per tile (one warp lane each)
constexpr int kMaxU = 16;
constexpr int kMaxRowDeg = 64;
constexpr int kMaxDevices = 64;
constexpr int kMaxColDeg = 64;  // a variable node's edges over all u matrices
constexpr int kMaxVClasses = 8;  // variable-node degree classes with slot tables of their own
constexpr int kMaxQBits = 24;   // fixed-point accumulation: at most 2^-24 resolution
constexpr int kMinQBits = 12;   // and at least 2^-12

// Tiles whose messages of one edge are stored together: 2 for 2- and 4-byte
// messages (2-byte: one 128-byte line, the tiles interleaved lane by lane;
// 4-byte: two adjacent 128-byte lines, one per tile), else 1.
constexpr int msg_pair(size_t msg_bytes) { return msg_bytes <= 4 ? 2 : 1; }
// Tiles of message storage for n_tiles tiles (rounded up to whole pairs).
constexpr size_t msg_tiles(size_t n_tiles, size_t msg_bytes) {
  return (n_tiles + msg_pair(msg_bytes) - 1) / msg_pair(msg_bytes) * msg_pair(msg_bytes);
}

struct DevCode {
  int32_t n, u, m_tot;
  int32_t max_row_deg;
  int32_t min_row_deg;  // smallest degree of a check with edges (1 when there are none)
  int32_t max_col_deg;
  int64_t e_tot, s_tot;
  int32_t m[kMaxU];
  int32_t row_first[kMaxU + 1];  // first stacked row of each matrix (CSR order)
  int32_t row_pos[kMaxU + 1];    // first row position of each matrix (the decoder's order)
  const int32_t* slice_base;  // [m_tot + 1] first slot of each row position
  const int32_t* slot_col;    // [s_tot]
  const int32_t* col_ptr;     // [n + 1]
  const int32_t* col_slot;    // [e_tot]
  const int32_t* row_ptr;     // [m_tot + 1] stacked CSR
  const int32_t* col_idx;     // [e_tot]
  const int32_t* edge_slot;   // [e_tot] stacked CSR edge -> slot
  const uint8_t* row_mat;     // [m_tot] matrix l of the row at position p
  const int32_t* row_local;   // [m_tot] row index j inside H_l of the row at position p
  const int32_t* row_at;      // [m_tot] the position of stacked row r (the inverse of the two above)
  // Variable nodes grouped by their degree over all matrices (n_vclass = 0 when there are more classes than
  // kMaxVClasses): class k holds node positions vclass_first[k] .. vclass_first[k+1] - 1, all of degree
  // vclass_deg[k]; vnode gives the node at each position, and the class's slots (col_slot order, one row of
  // vclass_deg[k] per position) start at vslot + vclass_toff[k].
  int32_t n_vclass;
  int32_t vclass_deg[kMaxVClasses];
  int32_t vclass_first[kMaxVClasses + 1];
  int64_t vclass_toff[kMaxVClasses];
  const int32_t* vnode;       // [n]
  const int32_t* vslot;       // [e_tot]
  const int32_t* vrow;        // [e_tot] each vslot entry's row: position << 6 | degree - 1
};

// Per-call decoder state carved out of the caller's workspace.
struct DevState {
  int32_t F, n_tiles;
  void* c2v;          // message type: [n_tiles / 2][s_tot][2][kLanes] (4 bytes), [n_tiles / 2][s_tot][kLanes][2]
                      // (2 bytes), [n_tiles][s_tot][kLanes] (8 bytes); n_tiles rounded up to pairs (msg_tiles)
  void* lv;           // [n_tiles][n][kLanes] posterior L_V of eq. (2)
  void* lp;           // [n_tiles][n][kLanes] channel LLR L_P of general (LLR) inputs
  uint32_t* yt;       // [n_tiles][n] Bob's bits, bit lane, for BSC inputs; NULL when L_P comes from lp
  void* chan_mag;     // [n_tiles][kLanes] ln((1 - e)/e) per frame (internal unit) for BSC inputs
  int32_t* lacc;      // [n_tiles][n][kLanes] fixed-point sum of C2V per node (FP32 single pass), or NULL
  uint32_t* xh;       // [n][n_tiles] hard decisions, bit lane (node-major: a node's words of 32 tiles are
                      // one 128-byte line, which the stopping test reads per edge)
  uint32_t* zt;       // [n_tiles][m_tot] syndrome bits, bit lane
  uint32_t* ztt;      // [m_tot][n_tiles] the same words row-major, for the streaming stopping test
  uint32_t* active;   // [n_tiles] lanes still decoding
  uint32_t* fail;     // [n_tiles][u] lanes whose hard decision violates some check of H_l
  int32_t* counters;  // [4]: unfinished tiles, non-finite flag
  void* ctl;          // control block of the resident schedule (barrier, retirement)
  // Row form of the first iteration's messages (BSC inputs): the C2V of row p
  // (degree d) to a node is +-fmag[tile][d - 1][lane], with sign bit lane of
  // rsgn[p][tile] ^ yt[tile][node]
  void* fmag;         // [n_tiles][kMaxRowDeg][kLanes] arithmetic type (rounded to the message type)
  uint32_t* rsgn;     // [m_tot][n_tiles] (row-major)
  uint32_t* ppos;     // [n_tiles] the lanes whose channel magnitude ln((1 - e)/e) is positive (BSC inputs)
  // Frame order: the decoder's slot s = tile * kLanes + lane holds the caller's frame perm[s], and frame f sits
  // in slot slot_of[f]. BSC inputs are ordered by QBER (ties by index), so that the frames of a tile need similar
  // iteration counts and a tile retires close to when its frames do; LLR inputs keep their order.
  int32_t* perm;      // [n_tiles * kLanes] (entries past F unused)
  int32_t* slot_of;   // [n_tiles * kLanes]
  // staging for mbp_decode_bsc_host
  uint32_t* io_y;
  double* io_qber;
  uint32_t* io_z;
  uint32_t* io_xhat;
  int32_t* io_iters;
  uint8_t* io_success;
};

}  // namespace mbp

struct mbp_codes {
  mbp::DevCode d;
  void* dev_block;
  size_t dev_bytes;
  int device;
};

namespace mbp {

// error reporting (thread-local message)
int set_error(int code, const char* fmt, ...);
int cuda_error(cudaError_t e, const char* what);

// launchers (mbp_kernels.cu)
cudaError_t launch_syndrome(const DevCode& c, const uint32_t* x_bits, int F, uint32_t* z_bits, cudaStream_t s);
cudaError_t launch_bsc_llr(const uint32_t* y_bits, const double* qber, int F, int n, int dtype, void* llr,
                           cudaStream_t s);
size_t workspace_bytes(const DevCode& c, int F, int msg_dtype, bool host_io);
void carve_workspace(const DevCode& c, int F, int msg_dtype, bool host_io, void* base, DevState* st);

struct DecodeArgs {
  const void* llr;         // [F][n] or NULL when y_bits is used
  const uint32_t* y_bits;  // [F][W] (BSC entry)
  const double* qber;      // [F]   (BSC entry)
  const uint32_t* z_bits;
  int max_iter;
  int early_exit;
  int accumulate;
  int schedule;
  int rule;      // MBP_RULE_*: check-node rule
  int update;    // MBP_UPDATE_*: flooding or matrix by matrix
  int validate;
  double l_max;
  uint32_t* x_hat_bits;
  int32_t* iters;
  uint8_t* success;
  void* soft_out;
  uint8_t* synd_ok;
};

int decode(const DevCode& c, DevState& st, int msg_dtype, const DecodeArgs& a, cudaStream_t s);

// kernel accounting (mbp_profile_*), per host thread
void prof_enable(bool on);
bool prof_on();
void prof_begin(int family, cudaStream_t s);
void prof_end(int family, cudaStream_t s, int kernels);
int prof_get(int family, int64_t* launches, double* ms);
cudaError_t launch_export_c2v(const DevCode& c, const DevState& st, int msg_dtype, int frame, void* out,
                              cudaStream_t s);
// address of the library's fixed device scratch on the current device (mbp_decode_bsc_static)
int static_scratch(void** ptr);

// the iteration schedules: streaming (mbp_stream_<type>.cu) for arithmetic type M and stored message type S
// (float/float, double/double, float/__half, float/__nv_bfloat16), resident (mbp_resident.cu, M = S)
template <typename M, typename S>
int stream_iterations(const DevCode& c, DevState& st, const DecodeArgs& a, bool fixed, double l_max, float qscale,
                      float inv_qscale, cudaStream_t s);
// one flooding iteration of one group, no host synchronisation (grouped decode; float arithmetic); iter = 1,
// 2, 0 for a later iteration, or kStopTestOnly for the stopping test before iteration 1 alone
constexpr int kStopTestOnly = -1;
// Streams a step may fork onto while it is captured into a graph (independent launches then become parallel
// branches): the variable-node classes of a pass after the first run on aux[0], aux[1], joined back to the
// capturing stream through the events.
struct StreamFork {
  cudaStream_t aux[2];
  cudaEvent_t fork, join[2];
};
template <typename M, typename S>
cudaError_t stream_group_step(const DevCode& c, const DevState& st, int iter, double l_max, cudaStream_t s,
                              const StreamFork* fork = nullptr);
template <typename M>
int resident_group(const DevCode& c, int n_tiles);
template <typename M>
cudaError_t launch_resident_any(const DevCode& c, const DevState& st, const DecodeArgs& a, int G, double l_max,
                                cudaStream_t s);
size_t resident_ctl_bytes();
int resident_error(const void* ctl_host);

}  // namespace mbp
