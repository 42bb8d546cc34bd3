/*
 * mbp.h — C ABI of the GB300 multi-matrix belief-propagation (MBP) decoder.
 *
 * The library reconciles quantum-key frames as in arXiv 2001.07979: Bob holds
 * F frames y of n bits, Alice sends him, for each of u > 1 sparse parity-check
 * matrices H_1..H_u, the syndrome z^l = H_l x (mod 2) of her frame x
 * (Section 2, eq. 1). Bob decodes every frame with belief propagation on all u
 * matrices at once (Section 3A, Algorithm 1): flooding check-node updates
 * (eq. 6) and variable-node updates whose soft decision sums the messages of all
 * u matrices (eq. 2), then the hard decision and the stopping rule "H_l y = z^l
 * for every l" (Section 2), per frame.
 *
 * Conventions of every entry point:
 *  - Returns MBP_OK (0) or an MBP_E* status; mbp_last_error_string() then gives
 *    a message for the calling thread. No C++ exception crosses the ABI. A
 *    frame that fails to decode is not an error (success[f] = 0).
 *  - "device" pointers must be CUDA device (or managed) memory of the current
 *    device; they are owned by the caller and only read or written during the
 *    call's stream work. "host" pointers are ordinary host memory.
 *  - Bit vectors are packed in uint32 words, least significant bit first: bit i
 *    of a frame is bit (i & 31) of word (i >> 5); a frame of b bits takes
 *    ceil(b/32) words and unused high bits of its last word are zero on output
 *    and ignored on input.
 *  - Syndromes of F frames are laid out [u][F][ceil(m_l/32)]: all frames of
 *    matrix 1, then all frames of matrix 2, and so on.
 *  - LLRs are ln(P(bit = 0) / P(bit = 1)) (positive favours 0).
 *  - Work is issued on `stream` (NULL = the legacy default stream) and is
 *    stream-ordered. mbp_syndrome, mbp_bsc_llr, the NBP calls and the decode
 *    calls under the graph schedule (the default wherever it applies, see
 *    MBP_SCHED_AUTO) are asynchronous: they return once the work is queued, and
 *    the outputs are ready when `stream` reaches that point. The streaming and
 *    resident schedules read state back to the host during the call and return
 *    when decoding has finished; so do mbp_decode_bsc_host (it copies the
 *    outputs to host memory), mbp_autotune_multi, opts->validate = 1 (one
 *    read-back of the non-finite check) and kernel accounting.
 *  - Device pointers and the codes handle must belong to the device that is
 *    current when the call is made; a mismatch is MBP_EINVAL.
 */
#ifndef MBP_H
#define MBP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* mbp_stream_t; /* the same type as cudaStream_t */

enum {
  MBP_OK = 0,
  MBP_EINVAL = 1,       /* invalid argument: null pointer, bad size, malformed matrix, non-finite LLR */
  MBP_ENOMEM = 2,       /* host or device allocation inside mbp_create_codes failed */
  MBP_ECUDA = 3,        /* a CUDA runtime call or kernel launch failed */
  MBP_ETIMEOUT = 4,     /* a bounded device-side wait (grid barrier of the resident schedule) gave up */
  MBP_EUNSUPPORTED = 5  /* valid input outside this build's limits (e.g. a check of degree > 64) */
};

/*
 * Message storage precision of the decoder. F32 and F64 compute in the
 * precision they store. F16 and BF16 store every check-to-variable message
 * rounded to IEEE binary16 / bfloat16 (round to nearest even) and compute the
 * check-node update, the posteriors and eq. (2) in FP32; their results differ
 * from F32 by that rounding (relative 2^-11 / 2^-8 per stored message). The
 * LLR inputs and soft outputs of F16 and BF16 are float.
 */
enum { MBP_MSG_F32 = 0, MBP_MSG_F64 = 1, MBP_MSG_F16 = 2, MBP_MSG_BF16 = 3 };

/*
 * How the soft decision of eq. (2), L_V = L_P + sum of the node's C2V over all
 * u matrices, is accumulated:
 *  MBP_ACC_FLOAT  a second pass per iteration sums the node's messages in
 *                 floating point, in stacked-row order (H_1's checks first);
 *  MBP_ACC_FIXED  MBP_MSG_F32 only: the check-node pass adds every message's change,
 *                 rounded to a multiple of 2^-q, to a 32-bit integer sum per
 *                 node, so each message is read once per iteration. q is the
 *                 largest value <= 24 with (max node degree) x l_max x 2^q < 2^31
 *                 (q = 22 for degree 16 and l_max 20); integer addition makes
 *                 the result exact and independent of ordering. Needs q >= 12;
 *  MBP_ACC_AUTO   (default) FLOAT. On GB300 the L2 reductions of FIXED cost
 *                 more than the second read of the messages, so FIXED is an
 *                 option, not the default.
 */
enum { MBP_ACC_AUTO = 0, MBP_ACC_FLOAT = 1, MBP_ACC_FIXED = 2 };

/*
 * How the iterations are scheduled on the GPU (results are the same):
 *  MBP_SCHED_STREAMING  one kernel per step (check nodes, variable nodes,
 *                       syndrome test, retirement) per iteration over every
 *                       tile of 32 frames that is still decoding; messages
 *                       stream through HBM each iteration, and the host reads
 *                       the number of unfinished tiles after each iteration;
 *  MBP_SCHED_RESIDENT   one cooperative launch that takes the tiles a group at
 *                       a time, as many as keep the group's messages within
 *                       3/4 of L2, and runs all of a group's iterations with
 *                       grid-wide barriers between the steps; needs floating-
 *                       point accumulation and FP32 or FP64 storage. A barrier
 *                       that waits longer than about 2 s ends the decode with
 *                       MBP_ETIMEOUT;
 *  MBP_SCHED_GRAPH      the schedule of mbp_decode_multi with one group: the
 *                       streaming schedule's kernels (or, if mbp_autotune_multi
 *                       chose them, persistent kernels over a device-built list
 *                       of the unfinished tiles) with the iteration loop inside
 *                       a CUDA graph (a WHILE node that the retirement kernel
 *                       drives), so no host round trip per iteration and the
 *                       call returns once the work is queued; FP32, FP16 or
 *                       BF16 storage, floating-point accumulation, flooding
 *                       sum-product. The workspace layout differs from the
 *                       other schedules' (size it with the same opts). The
 *                       graph is built on the first call for each workspace,
 *                       frame count and input kind and then cached (at most
 *                       16; destroying a code drops the graphs that name it);
 *  MBP_SCHED_AUTO       (default) GRAPH where it applies (flooding sum-product
 *                       with FP32, FP16 or BF16 storage and floating-point
 *                       accumulation), STREAMING otherwise (FP64 storage,
 *                       fixed-point accumulation, min-sum, matrix-serial).
 */
enum { MBP_SCHED_AUTO = 0, MBP_SCHED_STREAMING = 1, MBP_SCHED_RESIDENT = 2, MBP_SCHED_GRAPH = 3 };

/*
 * Algorithm variants (they change the results; the defaults are the paper's
 * decoder). Check-node rule:
 *  MBP_RULE_SUM_PRODUCT  eq. (6), the exact sum-product combination (default);
 *  MBP_RULE_MIN_SUM      the min-sum approximation: sign as eq. (6), magnitude
 *                        the smallest magnitude among the other incoming
 *                        messages (float arithmetic: FP32, FP16 or BF16 storage).
 * Update order:
 *  MBP_UPDATE_FLOODING      every check of every matrix reads the previous
 *                           iteration's messages (default);
 *  MBP_UPDATE_MATRIX_SERIAL Algorithm 1's loop nesting taken literally: within
 *                           an iteration, H_1's checks then the soft decision of
 *                           eq. (2), then H_2's checks (reading that posterior)
 *                           and eq. (2), and so on; the stopping rule after all
 *                           u matrices.
 * Both variants run with the streaming schedule (AUTO, which then means
 * STREAMING, or STREAMING) and floating-point accumulation.
 */
enum { MBP_RULE_SUM_PRODUCT = 0, MBP_RULE_MIN_SUM = 1 };
enum { MBP_UPDATE_FLOODING = 0, MBP_UPDATE_MATRIX_SERIAL = 1 };

/* One binary m x n matrix in compressed sparse rows, host memory, 0-based. */
typedef struct {
  int32_t n, m, nnz;
  const int32_t* row_ptr; /* [m + 1], row_ptr[0] = 0, non-decreasing, row_ptr[m] = nnz */
  const int32_t* col_idx; /* [nnz], 0 <= col < n, no repeated column inside a row */
} mbp_csr;

/* The u matrices H_1..H_u uploaded to the device (immutable, thread-safe to share). */
typedef struct mbp_codes mbp_codes;

typedef struct {
  int32_t msg_dtype;      /* MBP_MSG_F32 (default), MBP_MSG_F64, MBP_MSG_F16 or MBP_MSG_BF16 */
  int32_t early_exit;     /* 1 (default): each frame stops at its first iteration whose hard
                             decision satisfies every syndrome, tested before iteration 1 too;
                             0: every frame runs exactly max_iter iterations */
  int32_t validate;       /* 1: reject non-finite input LLRs with MBP_EINVAL (one extra host sync) */
  int32_t host_io;        /* 1: also reserve workspace for the staging buffers of mbp_decode_bsc_host */
  double l_max;           /* clip of every message to [-l_max, l_max]; > 0, default 20 */
  void* workspace;        /* device, >= mbp_decode_workspace_size() bytes, 256-byte aligned; owned by
                             the caller; holds the decoder state, which stays readable after a
                             decode call (see mbp_export_c2v) until the next call that uses it */
  size_t workspace_bytes;
  void* soft_out;         /* optional device [F][n] posterior L_V of eq. (2) at the last iteration
                             each frame ran (double for F64, float for the others); NULL to skip */
  uint8_t* synd_ok;       /* optional device [F][u]: 1 where H_l x_hat = z^l for the output bits */
  int32_t accumulate;     /* MBP_ACC_AUTO (default), MBP_ACC_FLOAT or MBP_ACC_FIXED */
  int32_t schedule;       /* MBP_SCHED_AUTO (default), MBP_SCHED_STREAMING, MBP_SCHED_RESIDENT or MBP_SCHED_GRAPH */
  int32_t rule;           /* MBP_RULE_SUM_PRODUCT (default) or MBP_RULE_MIN_SUM */
  int32_t update;         /* MBP_UPDATE_FLOODING (default) or MBP_UPDATE_MATRIX_SERIAL */
} mbp_opts;

/* Fill *opts with the defaults above (F32, early exit, l_max 20, no workspace). */
void mbp_default_opts(mbp_opts* opts);

/* Message of the last failing call on this thread ("" if none). Never NULL. */
const char* mbp_last_error_string(void);

/* Library version: major * 10000 + minor * 100 + patch. */
int mbp_version(void);

/*
 * Upload u matrices H_1..H_u (Section 2: u > 1 matrices generated by PEG; u = 1
 * gives single-matrix BP). All must share n; m and nnz may differ. The library
 * copies the host arrays, validates them (MBP_EINVAL with *out = NULL on a
 * malformed matrix; MBP_EUNSUPPORTED for u > 16, a check of degree > 64 or a
 * variable node with more than 64 edges over all u matrices) and
 * builds its device layouts on the current device. Synchronous.
 */
int mbp_create_codes(const mbp_csr* H, int u, mbp_codes** out);

/* Free a handle from mbp_create_codes (NULL is accepted). Synchronizes the device. */
int mbp_destroy_codes(mbp_codes* codes);

/* Sizes of an uploaded code: any output pointer may be NULL. */
int mbp_codes_info(const mbp_codes* codes, int32_t* u, int32_t* n, int32_t* m_total, int64_t* edges,
                   int32_t* max_check_degree);

/*
 * eq. (1): z^l = H_l x (mod 2) for l = 1..u and F frames.
 * x_bits: device [F][ceil(n/32)]; z_bits: device [u][F][ceil(m_l/32)], written.
 */
int mbp_syndrome(const mbp_codes* codes, const uint32_t* x_bits, int F, uint32_t* z_bits, mbp_stream_t stream);

/*
 * Channel LLRs of a binary symmetric channel, eq. (5) (Section 3B) read as
 * P^1 = |y - e|, P^0 = 1 - |y - e|, i.e. L_P = (1 - 2 y) ln((1 - e) / e).
 * y_bits: device [F][ceil(n/32)]; qber: device [F], each in (0, 0.5];
 * llr: device [F][n] of float (dtype MBP_MSG_F32) or double (MBP_MSG_F64).
 * ln((1 - e)/e) is evaluated in double precision.
 */
int mbp_bsc_llr(const uint32_t* y_bits, const double* qber, int F, int n, int dtype, void* llr,
                mbp_stream_t stream);

/* Bytes of device workspace that a decode of F frames with these options needs. */
int mbp_decode_workspace_size(const mbp_codes* codes, int F, const mbp_opts* opts, size_t* bytes);

/*
 * Decode F frames (Algorithm 1, flooding over all u matrices):
 *   C2V starts at 0 (so V2C starts at L_P); each iteration every check of every
 *   matrix applies eq. (6) to V2C = clip(L_V - C2V_own) of the previous
 *   iteration, every variable forms L_V = L_P + sum over all matrices of its
 *   C2V (eq. 2), and the hard decision is bit = [L_V < 0]; the stopping rule
 *   is H_l x_hat = z^l for every l.
 * llr:     device [F][n], double for MBP_MSG_F64, float for the others.
 * z_bits:  device [u][F][ceil(m_l/32)] (Alice's syndromes).
 * max_iter >= 0.
 * Outputs (device): x_hat_bits [F][ceil(n/32)]; iters [F] = iterations run
 * (0 if the input already satisfied every syndrome, max_iter on failure);
 * success [F] = 1 iff the output satisfies every syndrome within max_iter.
 * On failure the output is the hard decision of the last iteration.
 * opts may be NULL only when F == 0. Asynchronous under the graph schedule
 * (the default for FP32, FP16 and BF16 storage); the streaming and resident
 * schedules return when the decode has finished.
 */
int mbp_decode_batch(const mbp_codes* codes, int F, const void* llr, const uint32_t* z_bits, int max_iter,
                     const mbp_opts* opts, uint32_t* x_hat_bits, int32_t* iters, uint8_t* success,
                     mbp_stream_t stream);

/*
 * mbp_decode_batch for BSC frames with the channel LLR of eq. (5) formed on the
 * device from Bob's bits: y_bits device [F][ceil(n/32)], qber device [F].
 * The decoder places the frames in its tiles of 32 in order of QBER (ties in
 * frame order; batches of up to 65,536 frames), so that the frames of a tile
 * need similar numbers of iterations and a tile stops close to when its frames
 * do. A frame's results do not depend on the other frames of the batch or on
 * their order, and every output is in the caller's frame order.
 */
int mbp_decode_bsc(const mbp_codes* codes, int F, const uint32_t* y_bits, const double* qber,
                   const uint32_t* z_bits, int max_iter, const mbp_opts* opts, uint32_t* x_hat_bits,
                   int32_t* iters, uint8_t* success, mbp_stream_t stream);

/*
 * mbp_decode_bsc with every input and output in HOST memory (page-locked
 * memory lets the copies run asynchronously; pageable memory also works). The
 * call copies y_bits [F][ceil(n/32)], qber [F] and z_bits [u][F][ceil(m_l/32)]
 * into staging buffers inside the workspace, decodes, and copies x_hat_bits,
 * iters and success back before it returns. opts->host_io must be 1 both here
 * and when the workspace was sized.
 */
int mbp_decode_bsc_host(const mbp_codes* codes, int F, const uint32_t* y_bits, const double* qber,
                        const uint32_t* z_bits, int max_iter, const mbp_opts* opts, uint32_t* x_hat_bits,
                        int32_t* iters, uint8_t* success, mbp_stream_t stream);

/*
 * mbp_decode_bsc_host without the final wait: the input copies, the decode and
 * the output copies are queued on `stream` and the call returns (once the
 * decode is queued, see MBP_SCHED_AUTO). The caller synchronises `stream` (or
 * an event recorded on it) before reading x_hat_bits, iters and success, and
 * before changing y_bits, qber or z_bits. The host buffers should be
 * page-locked (cudaHostAlloc / cudaHostRegister): copies from or to pageable
 * memory may wait for the stream. Calls on one stream with one workspace run in
 * order; calls that may overlap need workspaces of their own. This lets a
 * caller keep the GPU busy while it prepares the next batch: the copies of one
 * batch can run beside the decode of another on a second stream.
 */
int mbp_decode_bsc_host_async(const mbp_codes* codes, int F, const uint32_t* y_bits, const double* qber,
                              const uint32_t* z_bits, int max_iter, const mbp_opts* opts, uint32_t* x_hat_bits,
                              int32_t* iters, uint8_t* success, mbp_stream_t stream);

/*
 * Copy the check-to-variable messages of one frame, as left in the workspace
 * by the last decode with these opts, to c2v_out (device, [edges] in stacked
 * CSR order: H_1's edges row by row, then H_2's, ...; double for F64, float
 * for the others). Meant for inspection after an early_exit = 0 decode, where every
 * frame ran max_iter >= 1 iterations.
 */
int mbp_export_c2v(const mbp_codes* codes, int F, const mbp_opts* opts, int frame, void* c2v_out,
                   mbp_stream_t stream);

/*
 * Grouped decode of uneven frames. The paper splits a sifted key into k frames
 * of n bits that are decoded independently with one code (Section 3A); this
 * entry point decodes frames of several codes in one call: G groups; group g holds F_g
 * frames of its own code (n, rate, u and the QBER of each frame may all
 * differ between groups) with the same per-frame semantics as
 * mbp_decode_batch / mbp_decode_bsc. Every iteration runs either every
 * group's streaming-schedule kernels (grid kernels, the default unless
 * mbp_autotune_multi finds the other form faster; each group in a conditional
 * branch of its own, skipped once its frames have all finished), or one
 * persistent check-node kernel per check-degree class (at most 8 classes per
 * batch), one variable-node kernel and one syndrome kernel per class over the
 * frames of all groups that are still decoding; a single-block kernel retires
 * finished frames and sets the graph's conditions (and, for the persistent
 * kernels, rebuilds their work lists on the device). The loop is one CUDA
 * graph with a WHILE node (built on first use for each workspace, batch
 * shape, launch shape and group state, then cached by the library; destroying
 * a code drops the graphs that name it), so the call is asynchronous on
 * `stream`: it returns once the work is queued. opts->validate = 1 adds one host
 * synchronisation per group (the non-finite check), and while kernel
 * accounting (mbp_profile_enable) is on the loop is driven from the host with
 * one read-back per iteration.
 *
 * opts: msg_dtype F32 (default), F16 or BF16 (F64 gives MBP_EUNSUPPORTED);
 * accumulate AUTO or FLOAT; early_exit, l_max and validate as for
 * mbp_decode_batch; schedule, soft_out, synd_ok and host_io are ignored (the
 * per-group fields below replace them). workspace: device, 256-byte aligned,
 * >= mbp_multi_workspace_size() bytes for the same groups and opts.
 * At most 65535 tiles of 32 frames in all, and at most 256 groups.
 */
typedef struct {
  const mbp_codes* codes;  /* the group's code */
  int32_t F;               /* frames in the group (>= 0) */
  const void* llr;         /* device [F][n] float LLRs, or NULL to form eq. (5) from y_bits and qber */
  const uint32_t* y_bits;  /* device [F][ceil(n/32)] Bob's bits (used when llr is NULL) */
  const double* qber;      /* device [F] per-frame QBER in (0, 0.5] (used when llr is NULL) */
  const uint32_t* z_bits;  /* device [u][F][ceil(m_l/32)] Alice's syndromes */
  uint32_t* x_hat_bits;    /* device [F][ceil(n/32)], written */
  int32_t* iters;          /* device [F], written */
  uint8_t* success;        /* device [F], written */
  uint8_t* synd_ok;        /* optional device [F][u], written */
  void* soft_out;          /* optional device [F][n] float posterior L_V, written */
} mbp_group;

int mbp_multi_workspace_size(const mbp_group* groups, int G, const mbp_opts* opts, size_t* bytes);
int mbp_decode_multi(const mbp_group* groups, int G, int max_iter, const mbp_opts* opts, mbp_stream_t stream);

/*
 * Launch shapes of the grouped decode and the autotuner that picks them. The
 * paper chooses its thread-block split by measuring several for its frame
 * length (Section 3B, Table 1); mbp_autotune_multi makes that search on the
 * batch at hand: it decodes the batch with each
 * candidate (first the grid kernels against the persistent kernels; for the
 * persistent kernels then check-node blocks of 2, 4 or 8 warps on all or half
 * of the resident block slots, and variable-node and syndrome blocks of 2, 4
 * or 8 warps; a coordinate search), timing each with CUDA events on `stream`, and
 * keeps the fastest for later mbp_decode_multi calls with the same codes and
 * frame counts on this device and message type. The results of every shape
 * are identical; the outputs are left as a decode with the chosen shape
 * writes them. Blocks until done. best may be NULL.
 */
typedef struct {
  int32_t grid_kernels; /* 1: every group runs the streaming schedule's kernels (a block per 8 rows or nodes of
                           every tile); 0: persistent kernels over the device-built lists of unfinished tiles */
  int32_t cn_warps;   /* warps per block of the check-node kernels */
  int32_t cn_waves;   /* 1: every resident block slot of the SMs; 2: half of them */
  int32_t vn_warps;   /* warps per block of the variable-node kernel */
  int32_t syn_warps;  /* warps per block of the syndrome kernels */
  double ms;          /* measured time of one decode with this shape */
} mbp_tuning;

int mbp_autotune_multi(const mbp_group* groups, int G, int max_iter, const mbp_opts* opts, mbp_tuning* best,
                       mbp_stream_t stream);

/*
 * Set the launch shape that later mbp_decode_multi calls use for these codes and frame counts on the current
 * device and message type (as mbp_autotune_multi leaves it), e.g. one found by an earlier autotuning run.
 * cn_warps, vn_warps and syn_warps in {2, 4, 8}; cn_waves in {1, 2}; ms is ignored.
 */
int mbp_multi_set_tuning(const mbp_group* groups, int G, const mbp_opts* opts, const mbp_tuning* tuning);

/* Drop the library's cached graphs and tuned shapes (for example before freeing a workspace that a cached graph
 * refers to and allocating another at the same address; a graph never reads a workspace outside a decode call). */
int mbp_release_cached(void);

/*
 * Unrolled normalised BP with learnable scalars. The paper's decoder has no
 * learned parameters; this form unrolls T flooding iterations of the decoder
 * above (Algorithm 1 with eq. 6 and eq. 2, no early exit) and rescales every
 * check-to-variable message of matrix l at iteration t as
 *   C = alpha[t][l] * sgn(c) * max(|c| - beta[t][l], 0),
 * c being the message of eq. (6) clipped to l_max. alpha = 1, beta = 0 gives
 * the plain decoder's posteriors bit for bit. FP32 arithmetic; at most 32
 * edges per check.
 *
 * mbp_nbp_forward: llr device [F][n] float channel LLRs; z_bits device
 * [u][F][ceil(m_l/32)]; alpha, beta device [T][u] float (row t-1 for iteration
 * t; beta in LLR units); lv_out optional device [T][F][n] float, written: the
 * posterior L^t of eq. (2) after each iteration. The workspace (device,
 * 256-byte aligned, >= mbp_nbp_workspace_size bytes) keeps every iteration's
 * messages and posteriors (the checkpoints of the backward pass).
 *
 * mbp_nbp_backward: the gradient of J = sum_t sum_{f,i} grad_lv[t][f][i] L^t[f][i]
 * (grad_lv device [T][F][n]) with respect to alpha and beta (device [T][u]
 * float, written) and, if grad_llr is not NULL, the channel LLRs (device
 * [F][n] float, written). A hand-written adjoint that runs the iterations in
 * reverse from the checkpoints; it must follow mbp_nbp_forward with the same
 * codes, F, T, alpha, beta, l_max and workspace. Deterministic (no atomics).
 * Both calls are asynchronous on `stream`.
 */
int mbp_nbp_workspace_size(const mbp_codes* codes, int F, int T, size_t* bytes);
int mbp_nbp_forward(const mbp_codes* codes, int F, int T, const float* llr, const uint32_t* z_bits,
                    const float* alpha, const float* beta, double l_max, void* workspace, size_t workspace_bytes,
                    float* lv_out, mbp_stream_t stream);
int mbp_nbp_backward(const mbp_codes* codes, int F, int T, const float* alpha, const float* beta, double l_max,
                     const float* grad_lv, void* workspace, size_t workspace_bytes, float* grad_alpha,
                     float* grad_beta, float* grad_llr, mbp_stream_t stream);

/*
 * Allocation-free decode. The paper has no counterpart: this entry point
 * exists for callers that can pass device inputs and outputs but cannot call
 * cudaMalloc for a workspace, for example because another runtime owns the
 * device memory budget, or because an allocation (and the device
 * synchronization that cudaFree implies) is not allowed where they call from.
 *
 * It behaves like mbp_decode_bsc, but keeps the decoder state in a fixed
 * device array of MBP_STATIC_SCRATCH_BYTES inside this library instead of
 * opts->workspace. opts->workspace and opts->workspace_bytes are ignored, and
 * opts->host_io must be 0; opts->schedule MBP_SCHED_GRAPH gives MBP_EUNSUPPORTED
 * (instantiating a graph may allocate), and MBP_SCHED_AUTO runs the streaming
 * schedule, so the call returns when decoding has finished. opts->validate has
 * no effect here (BSC inputs carry no LLR array to check). The call allocates
 * nothing: no cudaMalloc, no cudaFree, no allocating library routine.
 *  - The array is created when the library's device code is loaded on a GPU.
 *    Every GPU that loads the library holds it until the process exits.
 *  - The array's device address is looked up once per device, with that device
 *    current, and cached. mbp_create_codes does this for the device it uploads
 *    to (which also loads the library's device code there), so the
 *    allocation-free calls that use those codes neither load code nor look the
 *    address up. Should that look-up have failed, the first allocation-free
 *    call on the device repeats it: make that call before starting any stream
 *    capture.
 *  - Sizes: a batch whose workspace (mbp_decode_workspace_size with the same
 *    opts) exceeds MBP_STATIC_SCRATCH_BYTES is rejected with MBP_EINVAL.
 *  - Every call shares the one array and leaves its contents behind. The
 *    decoder initialises everything it reads, so a call never sees the
 *    previous call's state. Two calls whose GPU work overlaps, for example on
 *    two streams or two host threads, race on the array and give undefined
 *    results: serialise them.
 */
#define MBP_STATIC_SCRATCH_BYTES (64u * 1024u * 1024u)
int mbp_decode_bsc_static(const mbp_codes* codes, int F, const uint32_t* y_bits, const double* qber,
                          const uint32_t* z_bits, int max_iter, const mbp_opts* opts, uint32_t* x_hat_bits,
                          int32_t* iters, uint8_t* success, mbp_stream_t stream);

/*
 * Kernel accounting for benchmarks (no counterpart in the paper). While
 * enabled on a host thread, the decode calls made by that thread record a CUDA
 * event pair on the call's stream around every kernel they launch and add the
 * elapsed device time to the kernel's family. mbp_profile_enable(1) clears the
 * totals; mbp_profile_get waits for the recorded events and returns the
 * launch count and summed milliseconds of one family.
 */
enum {
  MBP_KERNEL_CHECK = 0,     /* check-node update, eq. (6) */
  MBP_KERNEL_VARIABLE = 1,  /* variable-node update and hard decision, eq. (2) */
  MBP_KERNEL_SYNDROME = 2,  /* per-frame syndrome test of the hard decision */
  MBP_KERNEL_RETIRE = 3,    /* retire finished frames */
  MBP_KERNEL_SETUP = 4,     /* channel LLRs, syndrome bits and tile state into the workspace */
  MBP_KERNEL_OUTPUT = 5,    /* output bits and soft values */
  MBP_KERNEL_PERSISTENT = 6,/* the resident schedule's single kernel (all steps of every iteration) */
  MBP_KERNEL_CHECK_ROWS = 7,/* eq. (6) in iteration 1 of BSC inputs, kept in row form (one sign word per
                               check and one magnitude per check degree and frame), and in iteration 2,
                               which reads the previous messages from that form */
  MBP_KERNEL_FAMILIES = 8
};
int mbp_profile_enable(int on);
int mbp_profile_get(int family, int64_t* launches, double* milliseconds);

#ifdef __cplusplus
}
#endif

#endif /* MBP_H */
