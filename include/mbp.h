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
 *  - Work is issued on `stream` (NULL = the legacy default stream).
 *    mbp_syndrome and mbp_bsc_llr are asynchronous. The decode calls read a
 *    per-iteration count of unfinished frames back to the host, so they return
 *    only when decoding has finished on `stream`.
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
 *                       tile of 8 frames that is still decoding; messages
 *                       stream through HBM each iteration;
 *  MBP_SCHED_RESIDENT   one cooperative launch that takes the tiles a group at
 *                       a time, as many as keep the group's messages within
 *                       3/4 of L2, and runs all of a group's iterations with
 *                       grid-wide barriers between the steps; needs floating-
 *                       point accumulation. A barrier that waits longer than
 *                       about 2 s ends the decode with MBP_ETIMEOUT;
 *  MBP_SCHED_AUTO       (default) STREAMING, which measures faster on GB300
 *                       for the benchmark workload.
 */
enum { MBP_SCHED_AUTO = 0, MBP_SCHED_STREAMING = 1, MBP_SCHED_RESIDENT = 2 };

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
  int32_t schedule;       /* MBP_SCHED_AUTO (default), MBP_SCHED_STREAMING or MBP_SCHED_RESIDENT */
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
 * opts may be NULL only when F == 0. Blocks until the decode has finished.
 */
int mbp_decode_batch(const mbp_codes* codes, int F, const void* llr, const uint32_t* z_bits, int max_iter,
                     const mbp_opts* opts, uint32_t* x_hat_bits, int32_t* iters, uint8_t* success,
                     mbp_stream_t stream);

/*
 * mbp_decode_batch for BSC frames with the channel LLR of eq. (5) formed on the
 * device from Bob's bits: y_bits device [F][ceil(n/32)], qber device [F].
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
 * Copy the check-to-variable messages of one frame, as left in the workspace
 * by the last decode with these opts, to c2v_out (device, [edges] in stacked
 * CSR order: H_1's edges row by row, then H_2's, ...; double for F64, float
 * for the others). Meant for inspection after an early_exit = 0 decode, where every
 * frame ran max_iter >= 1 iterations.
 */
int mbp_export_c2v(const mbp_codes* codes, int F, const mbp_opts* opts, int frame, void* c2v_out,
                   mbp_stream_t stream);

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
 * opts->host_io must be 0. The call allocates nothing: no cudaMalloc, no
 * cudaFree, no allocating library routine.
 *  - The array is created when the library's device code is loaded on a GPU.
 *    Every GPU that loads the library holds it until the process exits.
 *  - The first call on each device looks up the array's device address, with
 *    that device current, and caches it. Make that first call before starting
 *    any stream capture.
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
  MBP_KERNEL_FAMILIES = 7
};
int mbp_profile_enable(int on);
int mbp_profile_get(int family, int64_t* launches, double* milliseconds);

#ifdef __cplusplus
}
#endif

#endif /* MBP_H */
