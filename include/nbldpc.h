/*
 * nbldpc.h -- min-max (MMA) decoding of non-binary LDPC codes over GF(2^p)
 * on NVIDIA GB300 (sm_103a).  C ABI: plain pointers and sizes only.
 *
 * The operation is Alg. 2 of "In-Memory Non-Binary LDPC Decoding"
 * (arXiv 2508.03567): flooding belief propagation with the min-max check-node
 * rule computed by forward/backward (F, B) matrices, variable-node sums with
 * min-normalization, an a-posteriori argmin decision and a syndrome test that
 * stops each frame early.  Messages are 8-bit unsigned integers; the only
 * saturation is min(255, .) after the variable-node normalization.
 *
 * Conventions shared by every entry point
 *  - Field: q = 2^p, 2 <= q <= 256.  Elements are the integers 0..q-1 in
 *    polynomial basis (bit i = coefficient of x^i); the primitive element is
 *    x = 2 (Sec. 2.1).
 *  - Reliabilities gamma[f][n][a] (uint8) are the initial LLR-like metrics of
 *    Alg. 2 (gamma_n(a) = ln(p(eta)/p(a)), quantized): smaller is more likely.
 *    Index a is the symbol value.  They are used as given (no renormalization).
 *  - Hard decisions take the lowest symbol on ties.  The stop test on the
 *    decision of iteration k-1 runs before iteration k; out_iters counts the
 *    completed check+variable passes (0 when the channel decision already
 *    satisfies every check and early_stop is set).
 *  - Every status is one of the NBLDPC_* codes below; nbldpc_status_string()
 *    describes it.  Errors detected on the host are returned before any GPU
 *    work is queued and leave the outputs untouched.
 */
#ifndef NBLDPC_H
#define NBLDPC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * Opaque code handle.  The code (H and its field) is fixed at create; the
 * launch configuration (tuning, message width, check-node schedule) changes
 * only through nbldpc_code_set_tuning, nbldpc_code_set_message_bits,
 * nbldpc_code_set_cnp_schedule and nbldpc_code_autotune, which must not run
 * concurrently with any other call on the same handle.
 */
typedef struct nbldpc_code nbldpc_code;

enum {
  NBLDPC_OK = 0,
  NBLDPC_ERR_ARG = -1,         /* null pointer, negative count, short workspace ... */
  NBLDPC_ERR_POLY = -2,        /* q not a power of two in [2,256] or polynomial not primitive of degree p */
  NBLDPC_ERR_H = -3,           /* malformed parity-check matrix */
  NBLDPC_ERR_CUDA = -4,        /* a CUDA call failed (also reports earlier asynchronous faults) */
  NBLDPC_ERR_NOMEM = -5,       /* device or host allocation failed inside nbldpc_code_create */
  NBLDPC_ERR_TIMEOUT = -6,     /* reserved: a bounded device-side wait expired */
  NBLDPC_ERR_UNSUPPORTED = -7  /* valid code outside the library's limits (see nbldpc_code_create) */
};

/*
 * Build a code handle from H given as CSR rows (Sec. 2.1: M x N sparse
 * parity-check matrix over GF(q); Tanner graph with M check and N variable
 * nodes; edge = non-zero entry).
 *
 *   q         field order, a power of two in [2, 256]
 *   prim_poly primitive polynomial including the x^p term (e.g. 0x11D for q = 256)
 *   n_cols    N, number of variable nodes (symbols per frame)
 *   n_rows    M, number of check nodes
 *   row_ptr   host, [n_rows+1], row_ptr[0] = 0, non-decreasing; nnz = row_ptr[n_rows]
 *   col_idx   host, [nnz], 0 <= col < n_cols, no column twice within a row
 *   coef      host, [nnz], 1 <= coef < q (the GF coefficient h_{m,n})
 *   out       receives the handle; set to NULL on failure
 *
 * Checks: every row has degree >= 2, every column degree >= 1.  Build limits
 * (NBLDPC_ERR_UNSUPPORTED beyond them): n_cols < 65535, nnz < 65535, row
 * degree <= 64, column degree <= 64, and the code description (3q + 2(M+1) +
 * 8 nnz + 2(N+1) bytes in 16-byte sections), the N decisions and one check
 * group's scratch per group must fit one block's shared memory (227 KB on
 * GB300: about N = 12000 for a (2,4) binary code).  The edge order within a
 * row does not change any output (the min-max convolution is commutative and
 * associative).
 *
 * The handle owns device copies of H, its variable-node view and the GF
 * exponent/logarithm tables, allocated on the device that is current at this
 * call; every later call that queues GPU work on the handle returns
 * NBLDPC_ERR_ARG (before queueing anything) unless that device is current.
 * Copies the host arrays; the caller keeps ownership of them.  Decodes may run
 * concurrently from several threads on one handle when each uses its own
 * workspace; the setters and the autotuner may not run alongside any other
 * call on the handle.
 */
int nbldpc_code_create(int q, uint32_t prim_poly, int n_cols, int n_rows, const int32_t *row_ptr,
                       const int32_t *col_idx, const uint8_t *coef, nbldpc_code **out);

/* Free a handle (NULL is accepted).  No decode on it may be in flight. */
void nbldpc_code_destroy(nbldpc_code *code);

/* Shape of a handle; any output pointer may be NULL. */
int nbldpc_code_info(const nbldpc_code *code, int *q, int *n, int *m, int *nnz);

/*
 * Device workspace nbldpc_decode needs for `frames` frames, in bytes (a
 * persistent grid sized to the current device keeps one message slot of
 * nnz*q bytes per resident block, so the size saturates for large batches).
 */
int nbldpc_decode_workspace_size(const nbldpc_code *code, int frames, size_t *bytes);

/*
 * Decode `frames` frames (Alg. 2), stream-ordered on `cuda_stream`
 * (a cudaStream_t; NULL = legacy default stream).  Returns after queueing.
 *
 *   gamma_dev      device, [frames][n_cols][q] uint8, read only
 *   max_iters      I_max >= 0 (0: channel decision only)
 *   early_stop     non-zero: stop a frame once its decision satisfies every check
 *   out_sym_dev    device, [frames][n_cols] uint8: decided symbols
 *   out_iters_dev  device, [frames] int32: iterations run
 *   out_ok_dev     device, [frames] uint8: 1 if the returned symbols satisfy every check
 *   workspace_dev  device, >= nbldpc_decode_workspace_size(code, frames) bytes,
 *                  16-byte aligned; scratch owned by the caller, contents
 *                  undefined after the call; one decode at a time per workspace
 *
 * All device buffers are owned by the caller and must stay valid until the
 * queued work completes.  frames == 0 queues nothing.  Each frame's outputs
 * depend only on that frame's gamma (not on the batch it is decoded in).
 */
int nbldpc_decode(const nbldpc_code *code, const uint8_t *gamma_dev, int frames, int max_iters,
                  int early_stop, uint8_t *out_sym_dev, int32_t *out_iters_dev, uint8_t *out_ok_dev,
                  void *workspace_dev, size_t workspace_bytes, void *cuda_stream);

/*
 * Device workspace nbldpc_decode_host needs when it streams the batch in
 * chunks of `chunk_frames` frames (two chunks in flight).
 */
int nbldpc_decode_host_workspace_size(const nbldpc_code *code, int chunk_frames, size_t *bytes);

/*
 * Same decode as nbldpc_decode, from and to HOST buffers: the batch is moved
 * in chunks of `chunk_frames` frames, the host-to-device copy of the next
 * chunk and the device-to-host copy of the previous one overlapping the
 * decode of the current chunk.  Pinned (page-locked) host buffers give
 * asynchronous copies; pageable ones work but serialize.
 *
 *   gamma_host     host, [frames][n_cols][q] uint8
 *   out_*_host     host, as in nbldpc_decode
 *   chunk_frames   frames per chunk (> 0)
 *   workspace_dev  device, >= nbldpc_decode_host_workspace_size(code, chunk_frames)
 *
 * Stream-ordered on `cuda_stream`: the host outputs are complete once that
 * stream has been synchronized.  Host and workspace buffers must stay valid
 * until then.
 */
int nbldpc_decode_host(const nbldpc_code *code, const uint8_t *gamma_host, int frames, int max_iters,
                       int early_stop, uint8_t *out_sym_host, int32_t *out_iters_host,
                       uint8_t *out_ok_host, int chunk_frames, void *workspace_dev,
                       size_t workspace_bytes, void *cuda_stream);

/*
 * ---- Mixed-code batches -------------------------------------------------
 * One persistent launch decodes the frames of up to NBLDPC_MAX_BATCH_JOBS
 * jobs, each with its own code (any q, N, degrees), reliabilities, iteration
 * limit and outputs.  The frames of all jobs form one work list; a block
 * slot takes the next frame as soon as its previous one has stopped (zero
 * syndrome or max_iters), so codes with different frame counts and frames
 * with different iteration counts share the GPU without idle tails.  Results
 * are identical to nbldpc_decode of each job on its own (frames are
 * independent); only the throughput differs.  The launch is a counter reset
 * plus one kernel on the caller's stream, so it can be captured in a CUDA
 * graph and replayed (same buffers) without host work.  This is the batching
 * form of the paper's multicodeword mapping (Sec. 4: one frame per processing
 * unit, no synchronization between frames), extended to mixed codes.
 */
#define NBLDPC_MAX_BATCH_JOBS 32

typedef struct nbldpc_job {
  const nbldpc_code *code;  /* all codes of a batch on the same device */
  const uint8_t *gamma_dev; /* [frames][n][q], 16-byte aligned */
  int frames;               /* >= 0 */
  int max_iters;            /* >= 0 */
  int early_stop;
  uint8_t *out_sym_dev;     /* [frames][n] */
  int32_t *out_iters_dev;   /* [frames] */
  uint8_t *out_ok_dev;      /* [frames] */
} nbldpc_job;

/* Device workspace for nbldpc_decode_batch with these jobs (their codes' current tuning). */
int nbldpc_decode_batch_workspace_size(const nbldpc_job *jobs, int n_jobs, size_t *bytes);

/*
 * Queue the batch on `cuda_stream`.  Each code decodes with its own layout
 * variant; the block is split into the smallest frames-per-block value among
 * the jobs' codes.  Errors: NBLDPC_ERR_ARG (n_jobs outside [1,
 * NBLDPC_MAX_BATCH_JOBS], bad pointers, short workspace), NBLDPC_ERR_UNSUPPORTED
 * (the combined shared-memory need exceeds the device), NBLDPC_ERR_CUDA.
 */
int nbldpc_decode_batch(const nbldpc_job *jobs, int n_jobs, void *workspace_dev, size_t workspace_bytes,
                        void *cuda_stream);

/*
 * ---- Tuning ----------------------------------------------------------------
 * Two knobs per code change speed, never results: the variant and the frames
 * decoded side by side in one 256-thread block (1, 2, 4 or 8; small codes
 * leave threads idle at 1).  Variant bit 0 is the layout (how the q x q
 * min-max work of one convolution is split between the lanes of a group and
 * their registers); bit 1 keeps each frame's messages in shared memory instead
 * of a workspace slot (variants 2 and 3: 8-bit messages, minimal schedule,
 * blocks of 384 threads with 1, 2 or 4 frames or of 256 threads with 8, and
 * the messages must fit beside the block's other shared data; otherwise
 * NBLDPC_ERR_UNSUPPORTED).  With one warp per frame (8 frames per block, or
 * any single-code launch whose frame slots are 32 threads) a GF(4) code of at
 * most 32 checks of degree <= 4 and columns of degree <= 2 is decoded by that
 * warp alone, with no block-wide barrier.
 * The workspace of such a code is 256 bytes.  Bit 2 (variants 4 and 5) prunes
 * the check-node convolutions: C(x) = min_y max(A(y), B(x ^ y)) equals the
 * minimum over the y with A(y) <= T for any T >= max_x C(x) (any other y gives
 * a maximum above C(x)), and likewise with A and B exchanged, so each
 * convolution folds in only the entries of one side below a bound it finds in
 * a few phases; the outputs are the same bit for bit.  Bit 2 needs a layout of
 * 32-lane groups (both layouts of GF(128) and GF(256), layout 0 of GF(64)),
 * 8-bit messages and the minimal schedule, and excludes bit 1 (otherwise
 * NBLDPC_ERR_UNSUPPORTED).  Mixed-code batches use the layout bit, and bit 2
 * for GF(128) and GF(256) codes.  nbldpc_code_create picks a default variant
 * per field order and a frames-per-block value from the code size;
 * nbldpc_code_autotune measures every valid pair on the caller's frames and
 * keeps the fastest.
 */
typedef struct nbldpc_tune_result {
  int variant;
  int frames_per_block;
  float ms;                 /* time of one decode of the tuning frames, fixed iterations */
} nbldpc_tune_result;

int nbldpc_code_get_tuning(const nbldpc_code *code, int *variant, int *frames_per_block);

/* Set the tuning by hand (variant 0..7, frames_per_block 1, 2, 4 or 8); NBLDPC_ERR_UNSUPPORTED if
 * that pair does not fit the device or the code.  Not concurrent with any other call on the same
 * handle (a decode reads the tuning).  Switching a code to 16-bit messages or to the Table 1
 * schedule keeps bit 0 of its variant only. */
int nbldpc_code_set_tuning(nbldpc_code *code, int variant, int frames_per_block);

/* Device workspace nbldpc_code_autotune needs for `frames` tuning frames. */
int nbldpc_code_autotune_workspace_size(const nbldpc_code *code, int frames, size_t *bytes);

/*
 * Time a fixed-iteration decode (max_iters >= 1, no early stop) of the
 * caller's `frames` frames gamma_dev for every valid (variant,
 * frames-per-block) pair (the fastest of three timed decodes after an untimed
 * one), keep the fastest pair, and report each measurement in
 * results[0 .. min(max_results, *n_results)).  Synchronous: returns after the
 * measurements (it waits on `cuda_stream`).  Not thread safe with respect to
 * other calls on the same handle.
 */
int nbldpc_code_autotune(nbldpc_code *code, const uint8_t *gamma_dev, int frames, int max_iters,
                         void *workspace_dev, size_t workspace_bytes, void *cuda_stream,
                         nbldpc_tune_result *results, int max_results, int *n_results);

/*
 * ---- Work counter --------------------------------------------------------------
 * With a counter set, every later decode of the code (single-code, batch job,
 * host-buffer and non-allocating decodes; not the autotuner's) adds to
 * *counter_dev, by device atomics in stream order, the number of pairs (x, y)
 * whose max(A(y), B(x ^ y)) its check-node convolutions evaluated: q^2 per
 * dense convolution, q per entry folded in by a pruned one.  The caller owns the
 * 8-byte-aligned device counter and clears it; NULL (the default) stops the
 * count.  Counting adds one atomic per frame and check group; leave it off
 * when timing.  Not concurrent with any other call on the same handle.
 */
int nbldpc_code_set_work_counter(nbldpc_code *code, unsigned long long *counter_dev);

/*
 * ---- Message width ---------------------------------------------------------
 * 8 bits (the default) keeps every message as one byte per symbol saturated at
 * 255 (the variable-node cap of the main reading).  16 bits keeps two bytes per
 * symbol saturated at 65535: the counterpart of the paper's comparison of
 * 8-bit and 32-bit integer messages (Sec. 5).  For column degree 2 and inputs
 * <= 63 a message grows by at most 63 per iteration, so within 1000
 * iterations the 16-bit cap is never reached and the results equal those of
 * unbounded integer messages.  Results depend on the width (through the cap);
 * each width is exact against the CPU oracle run with the same cap.  The
 * workspace doubles at 16 bits; mixed-code batches accept 8-bit codes only
 * (NBLDPC_ERR_UNSUPPORTED otherwise).
 */
/* bits: 8 or 16.  Not concurrent with any other call on the same handle. */
int nbldpc_code_set_message_bits(nbldpc_code *code, int bits);
int nbldpc_code_get_message_bits(const nbldpc_code *code, int *bits);

/*
 * ---- Check-node schedule ------------------------------------------------------
 *
 * The forward/backward check-node pass needs 3(d_c - 2) min-max convolutions
 * per check (F_1..F_{d_c-2}, B_{d_c-2}..B_1 and the d_c - 2 middle beta
 * values).  Table 1 of the paper counts F and B over d_c - 1 edges each,
 * 3 d_c - 4 convolutions: the two extra ones (F_{d_c-1} and B_0) feed no
 * message.  NBLDPC_CNP_TABLE1 computes them anyway, for timing the paper's
 * operation count; outputs are identical under both schedules.  Applies to
 * every later single-code decode of the code (a separate kernel); with 16-bit
 * messages, and in mixed-code batches, it returns NBLDPC_ERR_UNSUPPORTED.
 */
#define NBLDPC_CNP_MINIMAL 0
#define NBLDPC_CNP_TABLE1 1
/* Not concurrent with any other call on the same handle. */
int nbldpc_code_set_cnp_schedule(nbldpc_code *code, int schedule);
int nbldpc_code_get_cnp_schedule(const nbldpc_code *code, int *schedule);

/*
 * ---- FFT-based sum-product decoding (FFT-SPA, Alg. 1) -----------------------
 *
 * The paper's second decoder, in float arithmetic: messages are q symbol
 * probabilities per edge; the check node multiplies the Walsh-Hadamard
 * transforms (radix-2 transform over (Z_2)^p) of the permuted incoming
 * messages and transforms back (divided by q); the variable node multiplies
 * the channel probabilities with the other incoming messages and normalizes
 * the result to sum 1; the decision is the symbol of largest a-posteriori
 * product (lowest symbol on ties); the syndrome stop test precedes each
 * iteration as in Alg. 2.  A check-node output below zero (transform
 * rounding) is set to 0; a normalization whose sum is not positive gives the
 * uniform vector 1/q.
 *
 * Supported codes: column degree <= 8, and check degree <= 32 for q <= 64
 * (one lane per edge) or <= 8 for q = 128, 256 (a check's transformed
 * messages are spread over the registers of a lane group); other codes
 * return NBLDPC_ERR_UNSUPPORTED from both calls.
 */

/* Device workspace nbldpc_fftspa_decode needs for `frames` frames, in bytes
 * (one message slot of nnz*q floats per resident block, so the size
 * saturates for large batches). */
int nbldpc_fftspa_workspace_size(const nbldpc_code *code, int frames, size_t *bytes);

/*
 * Decode `frames` frames with FFT-SPA (Alg. 1), stream-ordered on
 * `cuda_stream` (a cudaStream_t; NULL = legacy default stream).  Returns
 * after queueing.
 *
 *   prob_dev       device, [frames][n_cols][q] float, 16-byte aligned, read
 *                  only: the channel probabilities p_n(x) of each symbol
 *                  (non-negative; each row is used as given, no
 *                  normalization is applied to it)
 *   max_iters      I_max >= 0 (0: channel decision only)
 *   early_stop     non-zero: stop a frame once its decision satisfies every check
 *   out_sym_dev    device, [frames][n_cols] uint8: decided symbols
 *   out_iters_dev  device, [frames] int32: iterations run
 *   out_ok_dev     device, [frames] uint8: 1 if the returned symbols satisfy every check
 *   out_app_dev    device, [frames][n_cols][q] float, 16-byte aligned, or
 *                  NULL: the a-posteriori vectors of the returned decision,
 *                  normalized to sum 1 (the channel probabilities, normalized,
 *                  when no iteration ran)
 *   workspace_dev  device, >= nbldpc_fftspa_workspace_size(code, frames)
 *                  bytes, 16-byte aligned; scratch owned by the caller,
 *                  contents undefined after the call; one decode at a time
 *                  per workspace
 *
 * All device buffers are owned by the caller and must stay valid until the
 * queued work completes.  frames == 0 queues nothing.  Each frame's outputs
 * depend only on that frame's probabilities.
 */
int nbldpc_fftspa_decode(const nbldpc_code *code, const float *prob_dev, int frames, int max_iters,
                         int early_stop, uint8_t *out_sym_dev, int32_t *out_iters_dev, uint8_t *out_ok_dev,
                         float *out_app_dev, void *workspace_dev, size_t workspace_bytes, void *cuda_stream);

/* Device workspace nbldpc_fftspa_decode_host needs for chunks of
 * `chunk_frames` frames, in bytes (two chunks of probabilities, outputs and
 * decoder workspace). */
int nbldpc_fftspa_decode_host_workspace_size(const nbldpc_code *code, int chunk_frames, size_t *bytes);

/*
 * nbldpc_fftspa_decode on HOST buffers: prob_host [frames][n_cols][q] float
 * (pinned memory lets the copies overlap), outputs out_sym_host
 * [frames][n_cols] uint8, out_iters_host [frames] int32, out_ok_host [frames]
 * uint8.  Frames move in chunks of `chunk_frames`: one chunk's host-to-device
 * copy, decode and device-to-host copies are queued on one of two streams (the
 * caller's stream and a stream owned by the code handle) so that copies and
 * decoding of consecutive chunks overlap, as in nbldpc_decode_host.
 * workspace_dev: device, >= nbldpc_fftspa_decode_host_workspace_size bytes,
 * 256-byte aligned.  Returns after queueing; the outputs are valid once
 * `cuda_stream` has completed.  One host decode at a time per handle.
 */
int nbldpc_fftspa_decode_host(const nbldpc_code *code, const float *prob_host, int frames, int max_iters,
                              int early_stop, uint8_t *out_sym_host, int32_t *out_iters_host, uint8_t *out_ok_host,
                              int chunk_frames, void *workspace_dev, size_t workspace_bytes, void *cuda_stream);

/*
 * Size of the fixed device array that nbldpc_decode_noalloc works in.
 */
#define NBLDPC_NOALLOC_SCRATCH_BYTES (32u << 20)

/*
 * nbldpc_decode without a workspace argument and without any allocation.
 * The paper has no counterpart; this entry point exists for callers that
 * cannot call cudaMalloc or hand over device scratch: for example a receiver
 * or plugin that must not allocate device memory once it is running, or code
 * that runs inside a framework whose allocator owns all device memory and
 * exposes no way to borrow scratch from it.
 *
 * Same arguments, semantics and results as nbldpc_decode, minus the
 * workspace.  The scratch is one file-scope device array of
 * NBLDPC_NOALLOC_SCRATCH_BYTES (32 MiB), created with the library's module on
 * every GPU that loads it and held until the process exits.  The array holds
 * the frame counter (cleared by each call, stream-ordered) and one message
 * slot of nnz*q bytes per resident block; when fewer slots fit than the
 * device can keep resident, the call launches fewer blocks (same results,
 * lower throughput).  A code whose slot alone exceeds the array is rejected
 * with NBLDPC_ERR_UNSUPPORTED before anything is queued.
 *
 * Every call looks up the array's address in the current device's context
 * (cudaGetSymbolAddress), so it stays valid across a context reset; the first
 * call on a device may load the library's device code there, so make that
 * first call before any stream capture.  Nothing is allocated by this
 * function: no cudaMalloc, no cudaFree, no allocating library routine.
 *
 * All calls share the one array, and each call leaves its own contents
 * there.  Calls whose work overlaps on the GPU (different streams, different
 * threads, or different handles) race on it and give undefined results;
 * serialize them, for instance by queueing them on one stream.
 */
int nbldpc_decode_noalloc(const nbldpc_code *code, const uint8_t *gamma_dev, int frames, int max_iters,
                          int early_stop, uint8_t *out_sym_dev, int32_t *out_iters_dev,
                          uint8_t *out_ok_dev, void *cuda_stream);

/*
 * ---- Serving: continuous batching of decode requests -------------------------
 *
 * A server queues requests (frames of one code in host memory), admits them in
 * arrival order while the device bytes they keep resident (reliabilities,
 * outputs, and the workspace of the launches in flight) fit a budget, and
 * launches the admitted requests as one mixed-code persistent decode
 * (nbldpc_decode_batch, up to max_jobs requests) as soon as one of its streams
 * is free; requests arriving meanwhile go into the next launch, concurrently
 * with the launches still in flight.  "Plain" mode is the reference point: one
 * stream, one fixed-iteration nbldpc_decode per request (early stop off).  A
 * request larger than the whole budget is admitted alone once nothing else is
 * resident.  Each frame decodes to the same outputs alone or in any mix.
 *
 * The scheduler runs inside nbldpc_server_poll (no thread, no device-side
 * wait); one host thread drives a server.  The device work goes through an
 * executor: the library's CUDA executor (nbldpc_server_create) or callbacks
 * (nbldpc_server_create_custom, e.g. a host fake that tests the scheduler
 * without a GPU).  The paper has no serving layer; this is the batching and
 * latency layer over Alg. 2 decodes.
 */
typedef struct nbldpc_request {
  const nbldpc_code *code;
  const uint8_t *gamma_host;      /* [frames][n_cols][q] uint8; pinned for asynchronous copies */
  int frames;                     /* >= 1 */
  int max_iters;                  /* I_max >= 0 */
  int early_stop;                 /* continuous mode only; plain mode decodes fixed iterations */
  uint8_t *out_sym_host;          /* [frames][n_cols], written by the time the request completes */
  int32_t *out_iters_host;        /* [frames] */
  uint8_t *out_ok_host;           /* [frames] */
  void *user;                     /* caller's tag, passed back to custom executors */
  uint64_t id;                    /* set by nbldpc_server_submit */
} nbldpc_request;

typedef struct nbldpc_server_executor {
  void *ctx;
  /* resident device bytes of one request while admitted or in flight */
  size_t (*request_bytes)(void *ctx, const nbldpc_request *req);
  /* workspace bytes of one launch of these requests */
  size_t (*launch_bytes)(void *ctx, const nbldpc_request *const *reqs, int n, int plain);
  /* queue copies in, the decode and copies out on stream index `stream`; a token for done/finish */
  int (*start)(void *ctx, const nbldpc_request *const *reqs, int n, int stream, int plain, uint64_t *token);
  /* 1: the launch and its copies completed, 0: not yet, < 0: error status (non-blocking) */
  int (*done)(void *ctx, uint64_t token);
  /* release what the launch holds (called once, after done returned 1) */
  int (*finish)(void *ctx, uint64_t token);
} nbldpc_server_executor;

typedef struct nbldpc_server_stats {
  size_t used_bytes;              /* admitted requests + launches in flight (their requests and workspace) */
  size_t peak_bytes;
  uint64_t launches, submitted, completed;
  int waiting, admitted, in_flight;
} nbldpc_server_stats;

typedef struct nbldpc_server nbldpc_server;

/* Server with the library's CUDA executor on the current device: `streams`
 * (>= 1) streams owned by the server, device buffers from the stream-ordered
 * allocator, budget_bytes of resident device memory, up to max_jobs
 * (1..NBLDPC_MAX_BATCH_JOBS) requests per launch; plain != 0: plain mode. */
int nbldpc_server_create(size_t budget_bytes, int streams, int max_jobs, int plain, nbldpc_server **out);

/* Server whose device work goes to `executor` (copied; its ctx must outlive the server). */
int nbldpc_server_create_custom(const nbldpc_server_executor *executor, size_t budget_bytes, int streams,
                                int max_jobs, int plain, nbldpc_server **out);

/* Queue a request (copied; its host buffers must stay valid until it completes); *id receives its id.
 * The CUDA executor needs code, gamma_host and the three output buffers (NBLDPC_ERR_ARG otherwise); a
 * custom executor's server checks only frames >= 1 and max_iters >= 0. */
int nbldpc_server_submit(nbldpc_server *server, const nbldpc_request *req, uint64_t *id);

/* One scheduling round: retire completed launches, admit, launch on free
 * streams; then write up to `capacity` ids of completed requests (in
 * completion order; the rest come with later calls) and their count. */
int nbldpc_server_poll(nbldpc_server *server, uint64_t *done_ids, int capacity, int *n_done);

int nbldpc_server_stats_get(const nbldpc_server *server, nbldpc_server_stats *stats);

/* Wait for launches in flight (their outputs are written), then free the server; NULL is accepted. */
void nbldpc_server_destroy(nbldpc_server *server);

/*
 * Number of decode-kernel launches the calls above queued since the library
 * was loaded (all threads, all handles).  Launch accounting for benchmarks.
 */
uint64_t nbldpc_kernel_launch_count(void);

/*
 * ---- Measurement: integer min/max throughput probe ----------------------------
 * The check-node pass of Alg. 2 is a chain of XOR min-max convolutions,
 * C(x) = min_y max(A(y), B(x ^ y)) (F, B and beta equations), computed here on
 * packed pairs of 16-bit values.  The probe runs the instruction forms of that
 * computation alone on every SM, so that a decode's measured min-max rate can
 * be set against the rate the hardware gives those instructions:
 *
 *   NBLDPC_PROBE_ALU           max.u16x2 / min.u16x2 on the integer ALU pipe
 *   NBLDPC_PROBE_FMA_k_8       k/8 of the maxima as b + relu(a - b) on the FMA
 *                              pipe (fma.rn.relu.f16x2 + add.rn.f16x2), the
 *                              rest as above (the decode kernels use 3/8 for
 *                              q <= 64 and 1/8 for q >= 128)
 *   NBLDPC_PROBE_FMA_3_8_SHFL  the 3/8 mix with its A operands exchanged by
 *                              shfl.xor, as in the convolution's inner loop
 *   NBLDPC_PROBE_CONV_64/256   the decode kernels' convolution itself (GF(64)
 *                              16-lane layout / GF(256) 32-lane layout) chained
 *                              on shared-memory vectors
 *
 * Queues one launch that fills the current device (resident blocks x SMs) and
 * runs `rounds` (>= 1) rounds per thread on `cuda_stream`; *pairs receives the
 * min-max pairs (one 16-bit maximum + one 16-bit minimum each) the launch
 * performs and *blocks the grid size (either may be NULL).  sink_dev: device,
 * one unsigned int the kernel may write (it keeps the results live; its value
 * is meaningless).  The caller times the launch (e.g. with events on the
 * stream).  NBLDPC_ERR_ARG for an unknown form, rounds < 1 or a NULL sink.
 */
enum {
  NBLDPC_PROBE_ALU = 0,
  NBLDPC_PROBE_FMA_1_8 = 1,
  NBLDPC_PROBE_FMA_3_8 = 2,
  NBLDPC_PROBE_FMA_4_8 = 3,
  NBLDPC_PROBE_FMA_3_8_SHFL = 4,
  NBLDPC_PROBE_CONV_64 = 5,
  NBLDPC_PROBE_CONV_256 = 6
};
int nbldpc_probe_minmax(int form, int rounds, unsigned int *sink_dev, double *pairs, int *blocks,
                        void *cuda_stream);

/* Static description of a status code (never NULL). */
const char *nbldpc_status_string(int status);

#ifdef __cplusplus
}
#endif

#endif /* NBLDPC_H */
