/*
 * ldpc.h — C ABI of the GB300 (sm_103a) layered min-sum LDPC decoder.
 *
 * The interface follows the paper's statement of the problem (Ling & Cautereels, "Fast
 * LDPC GPU Decoder for Cloud RAN"):
 *   Sec. II   a quasi-cyclic code is a base graph H_BG (M_bg x N_bg, K_b systematic
 *             columns) lifted by Z; rate is chosen by the number of base rows used; the
 *             first two information columns are punctured.
 *   Sec. III  the decoder consumes the demapper's bit LLRs L_b, iterates layered min-sum
 *             (check rule with a correction, posterior update, next message) and stops at
 *             a valid codeword or at the iteration cap.
 *   Sec. IV   many codewords are decoded in parallel across the GPU.
 *
 * Conventions
 *   - LLR = ln P(b=0)/P(b=1); hard decision bit = (L_v < 0); sgn(0) = +1.
 *   - Circulant shift: entry V >= 0 of the base table gives shift s = V mod Z; check row i
 *     of block (r, c) connects variable c*Z + ((i + s) mod Z).  -1 marks a zero block.
 *   - Channel LLRs of one codeword cover codeword positions [punct_cols*Z,
 *     punct_cols*Z + n_tx); every other used position starts at LLR 0.
 *   - Hard bits: the K = K_b*Z information bits (punctured ones included), packed
 *     LSB-first: bit j is bit (j & 7) of byte (j >> 3); ceil(K/8) bytes per codeword.
 *   - All device buffers are owned by the caller; the graph owns its own device tables.
 *   - Calls are asynchronous on `stream`: argument errors found on the host are returned
 *     at once; errors raised inside a kernel are written to the graph's device status word
 *     and returned by ldpc_graph_sync_status.
 *   - No exceptions cross this interface.  A graph may be used by several host threads
 *     for decodes on different streams at the same time.
 */
#ifndef LDPC_GB300_H
#define LDPC_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ldpc_graph *ldpc_graph_t;       /* opaque, device-resident tables */
typedef struct CUstream_st *ldpc_stream_t;     /* same type as cudaStream_t */

typedef enum {
    LDPC_OK = 0,
    LDPC_ERR_INVALID_ARG = 1,
    LDPC_ERR_UNSUPPORTED = 2,
    LDPC_ERR_OUT_OF_MEMORY = 3,
    LDPC_ERR_CUDA = 4,
    LDPC_ERR_TIMEOUT = 5
} ldpc_status;

typedef enum { LDPC_LLR_INT8 = 0, LDPC_LLR_FP16 = 1, LDPC_LLR_FP32 = 2 } ldpc_llr_type;
typedef enum {
    LDPC_NORMALISED = 0,
    LDPC_OFFSET = 1,
    LDPC_LEARNED = 2,
    LDPC_SUM_PRODUCT = 3      /* flooding decoder only (ldpc_decode_flooding) */
} ldpc_algo;

/* Decoder options.  Fill with ldpc_decode_opts_default() and change what you need.
 *   llr_type     element type of the channel LLRs, posteriors and messages.
 *   algo         check-node correction (Sec. III, the factor beta):
 *                  LDPC_NORMALISED  m' = alpha * m            (fp16 / fp32)
 *                  LDPC_OFFSET      m' = max(m - offset, 0)   (int8: offset_q LLR units)
 *                  LDPC_LEARNED     m' = beta[t][r] * max(m - gamma[t][r], 0)
 *   alpha        normalisation factor (default 0.75).
 *   offset       offset for fp16 / fp32 in LLR units (default 0).
 *   offset_q     offset for int8 in quantised units (default 1).
 *   n_rows       base rows used, 4 <= n_rows <= M_bg; 0 = all rows (rate, Sec. II).
 *   n_tx         channel LLRs per codeword; 0 = (K_b + n_rows - punct_cols) * Z.
 *   punct_cols   punctured leading columns (default 2, Sec. II).
 *   early_stop   1: stop a codeword when its syndrome is zero after a full iteration.
 *   cluster_size 1: one thread block per codeword.  2: one codeword per cluster of two
 *                thread blocks on two SMs, each block half of every layer's check rows
 *                (alpha = 2 threads per row pair), posterior updates exchanged through
 *                distributed shared memory after every layer; the latency mode for a lone
 *                codeword; int8 offset min-sum, Z a multiple of 4.  Results are identical.
 *   learned_params device float [max_iter][n_rows][2] = (beta, gamma) for LDPC_LEARNED.
 *   threads_per_row  the paper's alpha (Sec. IV): cooperating threads per check-row pair.
 *                1 = the high-throughput strategy (one thread per row pair, two codewords
 *                per thread block); 2 or 4 = the low-latency strategy (alpha threads split
 *                each row's circulants and combine min, sub-min and sign by a log2(alpha)
 *                step warp-shuffle reduce; one codeword per thread block); int8 only.
 *                0 = automatic: 1 when the batch exceeds the SM count; else 2 when the
 *                graph fits, unless only the batch kernel's compiled form (ldpc_pair_jit)
 *                is ready for the graph's row sequence and the low-latency kernel's is
 *                not (then 1).  Results are identical for every value. */
typedef struct {
    int llr_type;
    int algo;
    float alpha;
    float offset;
    int offset_q;
    int n_rows;
    int n_tx;
    int punct_cols;
    int early_stop;
    int cluster_size;
    const float *learned_params;
    int threads_per_row;
} ldpc_decode_opts;

/* Defaults: int8, offset min-sum with offset_q = 1, alpha = 0.75, all rows, n_tx from the
 * rows, punct_cols = 2, early_stop = 1, cluster_size = 1, no learned table,
 * threads_per_row = 0 (automatic). */
void ldpc_decode_opts_default(ldpc_decode_opts *opts);

/* Build a device-resident graph from a host base table (Sec. II).
 *   base_shift  host int16 [M_bg][N_bg], row-major; -1 = zero block, V >= 0 a circulant
 *               with shift V mod Z.  The table is copied; the caller keeps ownership.
 *               A decode that uses n_rows rows requires every non-zero entry of those
 *               rows to lie in a column < K_b + n_rows (checked per call).
 *   M_bg, N_bg  1 <= M_bg <= 64, 2 <= N_bg <= 128;  K_b >= 1;  1 <= Z <= 1024.
 *   out         receives the handle.
 * Returns LDPC_ERR_INVALID_ARG for bad shapes or values, LDPC_ERR_OUT_OF_MEMORY /
 * LDPC_ERR_CUDA if the device tables cannot be allocated or copied.  Synchronous. */
ldpc_status ldpc_graph_create(const int16_t *base_shift, int M_bg, int N_bg, int K_b, int Z,
                              ldpc_graph_t *out);

/* Release a graph (waits for the device to finish with it). */
ldpc_status ldpc_graph_destroy(ldpc_graph_t g);

/* Shape queries: edges (non-zero circulants) in the first n_rows rows (0 = all), and the
 * number of posterior entries (K_b + n_rows) * Z.  Return -1 on a bad argument. */
int ldpc_graph_edges(ldpc_graph_t g, int n_rows);
int ldpc_graph_vars(ldpc_graph_t g, int n_rows);

/* Decode a batch (Sec. III layered min-sum, Sec. IV batch parallel).
 *   llr_dev        device [batch][n_tx] of int8 / binary16 / float32 per opts->llr_type.
 *   batch          codewords (>= 0; 0 is a no-op).
 *   max_iter       iteration cap T, 1..64.
 *   stream         CUDA stream (NULL = legacy default stream).
 *   opts           NULL = defaults.
 *   hard_bits_dev  device uint8 [batch][ceil(K/8)] output.
 *   iters_dev      device int32 [batch] output: iterations executed (T without early stop).
 * Host-side argument errors return at once and launch nothing: LDPC_ERR_INVALID_ARG for a
 * threads_per_row other than 0, 1, 2, 4 or a cluster_size other than 1, 2;
 * LDPC_ERR_UNSUPPORTED for threads_per_row 2 or 4 or cluster_size 2 outside the int8 offset
 * decoder or for graphs they cannot hold (cluster_size 2 takes threads_per_row 0 or 2).
 * Returns after the launch. */
ldpc_status ldpc_decode(ldpc_graph_t g, const void *llr_dev, int batch, int max_iter,
                        ldpc_stream_t stream, const ldpc_decode_opts *opts,
                        uint8_t *hard_bits_dev, int32_t *iters_dev);

/* Batch decode through row maps (serving support; the paper has no counterpart): codeword
 * b of the batch reads channel LLR row in_rows_dev[b] of llr_dev and writes hard-bit row
 * out_rows_dev[b] of hard_bits_dev and entry out_rows_dev[b] of iters_dev, so requests
 * scattered over a device pool decode in one launch without a gather.
 *   in_rows_dev, out_rows_dev  device int32 [batch]; rows must lie inside the caller's
 *                              buffers, and out rows must be distinct.
 * Everything else as for ldpc_decode. */
ldpc_status ldpc_decode_rows(ldpc_graph_t g, const void *llr_dev, const int32_t *in_rows_dev,
                             const int32_t *out_rows_dev, int batch, int max_iter,
                             ldpc_stream_t stream, const ldpc_decode_opts *opts,
                             uint8_t *hard_bits_dev, int32_t *iters_dev);

/* As ldpc_decode_rows with the row maps in host memory (serving support): the library
 * copies them into a pinned staging buffer and uploads them on `stream` ahead of the
 * launch, so a slot's row-mapped batch is one call with no separate upload by the caller.
 *   in_rows_host, out_rows_host  host int32 [batch], read before the call returns (the
 *                                caller may reuse them at once); a negative row is
 *                                LDPC_ERR_INVALID_ARG.  Rows must lie inside the caller's
 *                                buffers and out rows must be distinct.
 * The staging buffers belong to the library, one pair per (device, stream), grown on demand
 * (LDPC_ERR_OUT_OF_MEMORY if that fails) and kept for the process's lifetime; a call waits
 * on the host for the previous upload on the same stream to finish before refilling them.
 * Everything else as for ldpc_decode. */
ldpc_status ldpc_decode_rows_host_maps(ldpc_graph_t g, const void *llr_dev,
                                       const int32_t *in_rows_host,
                                       const int32_t *out_rows_host, int batch, int max_iter,
                                       ldpc_stream_t stream, const ldpc_decode_opts *opts,
                                       uint8_t *hard_bits_dev, int32_t *iters_dev);

/* As ldpc_decode, and also writes the final posteriors and check-to-variable messages
 * (for parity tests):
 *   post_dev  device [batch][(K_b + n_rows) * Z] in the LLR type.
 *   c2v_dev   device [batch][E * Z] in the LLR type, edge-major: the message of edge e
 *             (edges ordered by row, then column) on check row i is at e*Z + i.
 * Either may be NULL. */
ldpc_status ldpc_decode_debug(ldpc_graph_t g, const void *llr_dev, int batch, int max_iter,
                              ldpc_stream_t stream, const ldpc_decode_opts *opts,
                              uint8_t *hard_bits_dev, int32_t *iters_dev, void *post_dev,
                              void *c2v_dev);

/* Host-buffer variant for callers whose data lives in host memory.
 *   llr_host        host [batch][n_tx] in the LLR type (pinned memory gives the fastest
 *                   copies; pageable memory works).
 *   hard_bits_host  host uint8 [batch][ceil(K/8)];  iters_host  host int32 [batch].
 * The graph keeps device staging buffers (grown on demand, reused across calls) and a copy
 * stream; the call copies the LLRs in on that stream in chunks (the first one codeword per
 * SM for int8 batches above two per SM, else two per SM; each next one up to 8 times the
 * previous, at most a few chunks), decodes each chunk on `stream` as soon as its copy has
 * landed (so later copies overlap earlier decodes), copies each chunk's results out on
 * `stream`, and returns after all results are in host memory.  Results equal those of
 * ldpc_decode on the same LLRs.  Calls on the same graph from several threads are
 * serialised.  Argument errors are those of ldpc_decode, found before anything is
 * allocated or copied; LDPC_ERR_OUT_OF_MEMORY if the staging buffers cannot be allocated. */
ldpc_status ldpc_decode_host(ldpc_graph_t g, const void *llr_host, int batch, int max_iter,
                             ldpc_stream_t stream, const ldpc_decode_opts *opts,
                             uint8_t *hard_bits_host, int32_t *iters_host);

/* One codeword of a heterogeneous work list (ldpc_decode_list).
 *   graph       its graph (any mix of graphs, lifting sizes and row counts in one list)
 *   llr         device [n_tx] int8 channel LLRs
 *   hard_bits   device uint8 [ceil(K_b*Z/8)] output (LSB-first)
 *   iters       device int32 [1] output
 *   n_rows      base rows used (0 = all); n_tx: transmitted LLRs (0 = from n_rows);
 *   max_iter    iteration cap, 1..64. */
typedef struct {
    ldpc_graph_t graph;
    const void *llr;
    uint8_t *hard_bits;
    int32_t *iters;
    int n_rows;
    int n_tx;
    int max_iter;
} ldpc_work_item;

/* Decode a heterogeneous list of codewords in one launch (Sec. III decoding, Sec. IV many
 * codewords in parallel; the serving path).  int8 offset min-sum with offset_q = 1 and
 * punct_cols = 2 (opts: early_stop is honoured, llr_type must be INT8, algo OFFSET).
 * Each item needs even Z <= 384 and row degrees 2..20 (LDPC_ERR_UNSUPPORTED otherwise).
 * opts->threads_per_row picks the kernel: 0 (default) the low-latency strategy of Sec. IV
 * (2 threads per row pair, one persistent block per SM) when every item fits it, else one
 * thread per row pair; 1 forces the latter, 2 the former (LDPC_ERR_UNSUPPORTED when an
 * item does not fit it); 4 is LDPC_ERR_UNSUPPORTED, other values LDPC_ERR_INVALID_ARG.
 * Results are the same whichever kernel runs.
 * Thread blocks take items dynamically, largest first.  The library keeps a per-stream
 * device work table and work counter (allocated on first use, grown on demand, released
 * at exit); the host item array is copied before the call returns, so it may be reused.
 * Asynchronous on `stream`. */
ldpc_status ldpc_decode_list(const ldpc_work_item *items, int n_items, ldpc_stream_t stream,
                             const ldpc_decode_opts *opts);

/* Same as ldpc_decode_list, for callers that cannot allocate device memory (code running
 * inside another framework's memory pool, behind a fixed memory map, or on a path where a
 * cudaMalloc would synchronise the device).  The paper has no counterpart: this is a
 * deployment variant of the work-list decode.
 *   - Allocates nothing: no cudaMalloc / cudaFree / pinned host memory / heap.  The work
 *     table and the work counter live in a static device array inside the library, sized
 *     for at most 2048 items; every GPU that loads the library keeps it until exit.
 *     Longer lists return LDPC_ERR_INVALID_ARG.
 *   - The first call on a device looks up the array's device address (once per device,
 *     with that device current); make that first call before any stream capture.
 *   - Every call shares the one array: calls whose work overlaps on the GPU (different
 *     streams, or no ordering between them) race and may decode the wrong items.  The
 *     counter is cleared by each call.
 *   - The table is uploaded from pageable memory, so the call may wait for the stream's
 *     earlier work before it returns.
 * Outputs, supported shapes and the kernel choice (opts->threads_per_row) are those of
 * ldpc_decode_list. */
ldpc_status ldpc_decode_list_noalloc(const ldpc_work_item *items, int n_items,
                                     ldpc_stream_t stream, const ldpc_decode_opts *opts);

/* ---- Learned min-sum (training support) ------------------------------------------
 * A per-(iteration, base row) extension of the min-sum correction factor of Sec. III:
 * m' = beta[t][r] * max(m - gamma[t][r], 0), binary32 arithmetic, T iterations, no early
 * stop.  Loss-agnostic: the forward pass returns the final posteriors, the backward pass
 * takes dLoss/dposteriors and returns dLoss/d(beta, gamma) per codeword (and optionally
 * dLoss/dLLR), by reverse mode through the unrolled layers with the subgradient of each
 * min routed to the edge that attains it and signs held constant.
 *
 * Workspace: caller-owned device memory of ldpc_learned_workspace_floats(g, batch, T,
 * n_rows) floats; the forward pass writes the per-iteration checkpoints there and the
 * backward pass of the same batch reads them (and uses the rest as scratch). */
size_t ldpc_learned_workspace_floats(ldpc_graph_t g, int batch, int T, int n_rows);

/*   llr_dev      device float [batch][n_tx] channel LLRs
 *   params_dev   device float [T][n_rows][2] (beta, gamma)
 *   post_dev     device float [batch][(K_b + n_rows) * Z] output posteriors
 *   n_rows       0 = all rows; n_tx: 0 = from n_rows (punct_cols = 2). */
ldpc_status ldpc_learned_forward(ldpc_graph_t g, const float *llr_dev, int batch, int T,
                                 int n_rows, int n_tx, const float *params_dev,
                                 ldpc_stream_t stream, float *post_dev, float *workspace_dev);

/*   grad_post_dev    device float [batch][(K_b + n_rows) * Z]: dLoss/dposteriors
 *   grad_params_dev  device float [batch][T][n_rows][2] output (per codeword)
 *   grad_llr_dev     device float [batch][n_tx] output, or NULL */
ldpc_status ldpc_learned_backward(ldpc_graph_t g, const float *grad_post_dev, int batch, int T,
                                  int n_rows, int n_tx, const float *params_dev,
                                  ldpc_stream_t stream, float *workspace_dev,
                                  float *grad_params_dev, float *grad_llr_dev);

/* Per-iteration variants, for a loss over the posteriors after every iteration.
 *   post_iter_dev       device float [T][batch][(K_b + n_rows) * Z] output: slice t holds
 *                       the posteriors after iteration t + 1 (slice T-1 = final posteriors)
 *   grad_post_iter_dev  device float [T][batch][(K_b + n_rows) * Z]: dLoss/d(slice t)
 * Other arguments, the workspace contract and the outputs are those of
 * ldpc_learned_forward / ldpc_learned_backward.  The reverse sweep adds the adjoint of
 * slice t when it reaches the end of iteration t + 1, so grad_params is the gradient of
 * the loss summed over all slices.  detach != 0 resets the adjoints at every iteration
 * boundary instead: the parameters of iteration t + 1 then get the partial derivative of
 * slice t's own loss term (exact for that term; later terms' contributions are dropped) and
 * grad_llr only the contribution through iteration 1.  Not in the paper (training support,
 * like the functions above). */
ldpc_status ldpc_learned_forward_iter(ldpc_graph_t g, const float *llr_dev, int batch, int T,
                                      int n_rows, int n_tx, const float *params_dev,
                                      ldpc_stream_t stream, float *post_iter_dev,
                                      float *workspace_dev);
ldpc_status ldpc_learned_backward_iter(ldpc_graph_t g, const float *grad_post_iter_dev,
                                       int batch, int T, int n_rows, int n_tx,
                                       const float *params_dev, ldpc_stream_t stream,
                                       float *workspace_dev, float *grad_params_dev,
                                       float *grad_llr_dev, int detach);

/* ---- Flooding schedule (the comparison baseline of Sec. V) -------------------------
 * Every check row of every used base row is updated from the posteriors of the previous
 * iteration; then every posterior is recomputed as its channel LLR plus its incoming
 * messages summed in base-row order (the posterior equation of Sec. III); then the
 * syndrome test of ldpc_decode.  fp32 LLRs only (opts->llr_type must be LDPC_LLR_FP32);
 * opts->algo selects min-sum with LDPC_NORMALISED / LDPC_OFFSET, or LDPC_SUM_PRODUCT: the
 * exact tanh rule (Sec. III), evaluated in binary64 with the product over the other edges
 * clamped to +-(1 - 1e-15) before atanh.  Other options as for ldpc_decode.
 *   llr_dev        device float [batch][n_tx]
 *   bits_dev, iters_dev  as for ldpc_decode
 *   post_dev       device float [batch][(K_b + n_rows) * Z] final posteriors, or NULL
 *   workspace_dev  caller-owned device memory of ldpc_flooding_workspace_floats(g, batch,
 *                  n_rows) floats (the check-to-variable messages); overwritten.
 * Errors: LDPC_ERR_INVALID_ARG for bad arguments, LDPC_ERR_UNSUPPORTED for shapes beyond
 * 1024 edges, row degree 24 or the shared-memory size of one codeword's posteriors. */
size_t ldpc_flooding_workspace_floats(ldpc_graph_t g, int batch, int n_rows);
ldpc_status ldpc_decode_flooding(ldpc_graph_t g, const float *llr_dev, int batch, int max_iter,
                                 ldpc_stream_t stream, const ldpc_decode_opts *opts,
                                 uint8_t *hard_bits_dev, int32_t *iters_dev, float *post_dev,
                                 float *workspace_dev);

/* Self-test of the bounded device waits (no counterpart in the paper): launches a kernel
 * that waits on a shared-memory barrier armed for a transfer that is never issued, with at
 * most spin_limit polls (1 .. the decoders' own limit, 4 194 304), and returns the status
 * that wait produced: LDPC_ERR_TIMEOUT when it gave up as designed (the decoders then
 * record the same code in the graph's status word and return), LDPC_ERR_INVALID_ARG for a
 * bad limit, LDPC_ERR_CUDA on a launch error.  Nothing stays in flight; the context remains
 * usable.  cycles_out (host, may be NULL) receives the SM cycles the wait took.
 * Synchronous on `stream`. */
ldpc_status ldpc_selftest_wait_timeout(unsigned int spin_limit, ldpc_stream_t stream,
                                       unsigned long long *cycles_out);

/* Wait for the graph's outstanding work on `stream` and return (then clear) the device
 * status word: LDPC_OK, or the first error a kernel reported (e.g. LDPC_ERR_TIMEOUT). */
ldpc_status ldpc_graph_sync_status(ldpc_graph_t g, ldpc_stream_t stream);

/* Human-readable name of a status code (static string). */
const char *ldpc_status_string(ldpc_status s);

/* Number of kernels this library has launched since it was loaded (all threads). */
uint64_t ldpc_launch_count(void);

/* Device and pinned-host allocations the library has made since it was loaded (graph
 * tables, per-stream workspaces, staging buffers), all threads.  Monotone; a
 * diagnostic. */
uint64_t ldpc_alloc_count(void);

/* The 8-bit batch kernel (threads_per_row 1; the layered schedule of Sec. III), the
 * low-latency kernel (threads_per_row 2 and 4) and the binary16 kernel compiled at run time
 * for the degree sequence of the rows a decode uses, so that the layers of an iteration run
 * as straight-line code instead of one indirect branch per row.  Compiling
 * (NVRTC) takes a few seconds of host time per new degree sequence; the module is then
 * kept for the process's lifetime.  Results are bit-identical to the generic kernel's,
 * which runs whenever no compiled kernel is ready.
 *   mode 0: off.
 *   mode 1 (the default): a new sequence is compiled on a background thread; decodes use
 *           the generic kernel until it is ready.
 *   mode 2: the decode that meets a new sequence compiles it and waits (for throughput
 *           runs: compile during warm-up).
 *   mode 3: no change; wait until no background compilation runs.  A process must not
 *           exit while one runs (the compiler's exit-time cleanup may run under it): call
 *           this first (the Python binding does so when the interpreter exits).
 *   any other value: no change.
 * Returns the mode before the call (bits 0-1), plus 4 once a kernel has been compiled and
 * loaded and 8 once a compilation or load has failed since the library was loaded.
 * Process-wide; never fails. */
int ldpc_pair_jit(int mode);

/* Compile (and wait for) the 8-bit kernels of ldpc_pair_jit (the batch kernel and the
 * low-latency kernel at alpha 2 and 4) for a degree sequence:
 * row_degrees (host, n_rows entries, each 2..20) are the degrees of the rows a decode will
 * use, in order.  Host work only (no CUDA call; the first decode with the sequence loads
 * the module), so a throughput run can compile before its warm-up.  Returns LDPC_OK
 * (compiled now or earlier), LDPC_ERR_INVALID_ARG for a bad sequence, LDPC_ERR_UNSUPPORTED
 * when the compilation failed (decodes then use the generic kernel). */
ldpc_status ldpc_pair_jit_prepare(const int *row_degrees, int n_rows);

/* Compile the low-latency work-list kernel of ldpc_decode_list for a set of row sequences
 * (a server's graphs and rates): sequence q has n_rows[q] rows whose degrees (2..20) follow
 * those of sequence q - 1 in row_degrees (host arrays).  An item whose graph's first n_rows
 * rows have one of these degree sequences then runs its layers as straight-line code
 * instead of one indirect branch per row; other items run the generic row loop in the same
 * launch.  Results are identical either way.  Host work only (NVRTC, seconds); the next
 * ldpc_decode_list call loads the module and later calls use it.  n_seqs = 0 stops using
 * compiled list kernels.  Returns LDPC_OK, LDPC_ERR_INVALID_ARG (bad sequences, more than
 * 64 of them), LDPC_ERR_UNSUPPORTED (the compilation failed: lists keep the kernel they
 * had).  ldpc_decode_list_noalloc always uses the generic kernel. */
ldpc_status ldpc_list_jit_prepare(const int *row_degrees, const int *n_rows, int n_seqs);

#ifdef __cplusplus
}
#endif

#endif /* LDPC_GB300_H */
