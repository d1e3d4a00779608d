// Internal definitions shared by the C-ABI entry points and the decoder kernels.
#pragma once

#include <atomic>
#include <cstdint>
#include <functional>
#include <mutex>
#include <string>
#include <vector>
#include <cuda_runtime.h>

#include "../../include/ldpc.h"
#include "ldpc_params.h"

namespace ldpc {

constexpr int kMaxRows = 64;
constexpr int kMaxCols = 128;
constexpr int kMaxZ = 1024;
constexpr int kMaxIter = 64;
constexpr int kMaxEdges = kMaxRows * kMaxCols;

// Host-side graph object behind ldpc_graph_t.
struct Graph {
    int M_bg = 0, N_bg = 0, K_b = 0, Z = 0;
    int E_total = 0;
    int row_ptr[kMaxRows + 1] = {};      // edges of row r: [row_ptr[r], row_ptr[r+1])
    int max_col_upto[kMaxRows + 1] = {}; // largest column referenced by rows < r
    int max_deg_upto[kMaxRows + 1] = {}; // largest row degree among rows < r
    int min_deg_upto[kMaxRows + 1] = {}; // smallest row degree among rows < r
    int slots2_upto[kMaxRows + 1] = {};  // sum of ceil(degree / 2) over rows < r
    uint32_t h_edges[kMaxEdges] = {};    // (column << 16) | (shift mod Z), row by row
    uint32_t *d_edges = nullptr;         // device copy of h_edges
    int *d_row_ptr = nullptr;            // device [M_bg + 1]
    int *d_status = nullptr;             // device status word (ldpc_status of the first error)
    int device = 0;
    // staging buffers of ldpc_decode_host (guarded by host_mu): device copies of the
    // inputs and outputs, a copy stream, and one event per chunk of the pipelined upload
    std::mutex host_mu;
    void *d_stage = nullptr;
    size_t stage_bytes = 0;
    cudaStream_t copy_stream = nullptr;
    static constexpr int kHostChunks = 16;
    cudaEvent_t chunk_ev[kHostChunks] = {};
    // work counters of the batch kernel: one pair per stream that decodes with the graph
    // (zero between launches; the last block of a launch resets its pair)
    static constexpr int kQueues = 64;
    std::mutex q_mu;
    int *d_queues = nullptr;              // device [kQueues][2]
    cudaStream_t q_stream[kQueues] = {};
    int n_queues = 0;
    // per row count: (generation of a compiled list module << 32) | (1 + the case of this
    // graph's row sequence in it, 0 = none); list_jit.cu
    std::atomic<uint64_t> list_seq[kMaxRows + 1] = {};
};

// The work-counter pair of `g` for decodes on `stream`, or null when every slot is taken
// (the kernel then falls back to a fixed assignment of codewords to blocks).
int *graph_queue(Graph *g, cudaStream_t stream);

// Launch entry for the layered decoder (decode_layered.cu).  Returns LDPC_OK or an error
// found while configuring the launch.
ldpc_status launch_layered(const DecodeParams &p, int llr_type, cudaStream_t stream);

// Two codewords per thread (one per binary16 lane), one check row per thread, messages in
// Tensor Memory, per-lane stopping and refill (decode_tmem_pair.cu).
bool pair_supported(const DecodeParams &p, int llr_type, int max_deg, size_t smem_optin);
ldpc_status launch_pair(const DecodeParams &p, cudaStream_t stream);
// The batch kernel compiled at run time for the row sequence of p (pair_jit.cu), as a
// launchable kernel handle, or null (compilation off or failed: the generic kernel runs).
const void *pair_jit_kernel(const DecodeParams &p);

// One codeword per cluster of two blocks on two SMs, each block half of the row pairs,
// posterior updates exchanged through distributed shared memory (decode_cluster.cu).
bool cluster_supported(const DecodeParams &p, int llr_type, int max_deg, size_t smem_optin);
ldpc_status launch_cluster(const DecodeParams &p, cudaStream_t stream);

// One-codeword kernel with A = 2 or 4 cooperating threads per row pair, messages in
// Tensor Memory (decode_tmem_ll.cu): the low-latency strategy.
bool tmem_ll_supported(const DecodeParams &p, int llr_type, int max_deg, int A,
                       size_t smem_optin);
ldpc_status launch_tmem_ll(const DecodeParams &p, int A, cudaStream_t stream);
// tmem_ll_kernel compiled at run time for the row sequence of p (list_jit.cu), or null;
// ll_jit_prepare compiles it for a degree sequence and waits (host work only).
const void *ll_jit_kernel(const DecodeParams &p, int A);
bool ll_jit_prepare(const std::vector<int> &deg, int A);

// Row-pair fp16x2 kernel for 8-bit offset min-sum, messages in shared memory
// (decode_rowpair.cu).
bool rowpair_supported(const DecodeParams &p, int llr_type, int max_deg, size_t smem_optin);
ldpc_status launch_rowpair(const DecodeParams &p, int max_deg, cudaStream_t stream);

// binary16 decoder with messages in Tensor Memory, all three corrections
// (decode_tmem16.cu).
bool tmem16_supported(const DecodeParams &p, int llr_type, int max_deg, size_t smem_optin);
ldpc_status launch_tmem16(const DecodeParams &p, cudaStream_t stream);
// The binary16 kernel compiled at run time for the row sequence of p and a block shape
// (t16_jit.cu), or null (compilation off, pending or failed: the generic kernel runs).
const void *t16_jit_kernel(const DecodeParams &p, int cw, bool hybrid);

// Flooding-schedule decoder, fp32 min-sum or sum-product (decode_flooding.cu); ws holds
// the messages of every codeword.
size_t flooding_ws_floats_per_cw(int E, int Z);
ldpc_status launch_flooding(const DecodeParams &p, float *ws, cudaStream_t stream);

// Learned min-sum forward / backward (decode_learned.cu); ws holds the checkpoints.
size_t learned_ws_floats_per_cw(int N, int EZ, int T);
ldpc_status launch_learned(const DecodeParams &dp, int T, const float *params, const float *llr,
                           float *post, const float *grad_post, float *grad_params,
                           float *grad_llr, float *ws, bool backward, cudaStream_t stream,
                           float *post_iter = nullptr, const float *grad_post_iter = nullptr,
                           int detach = 0);

// Work-list decode (decode_rowpair.cu): items are taken dynamically through *d_counter,
// which must be zero at launch.
bool list_item_supported(int Z, int E, int n_rows, int max_deg);
size_t list_item_smem_bytes(int E, int n_rows, int n_cols, int Z);
// The work list with the low-latency strategy (decode_tmem_ll.cu): alpha = 2 threads per
// row pair, messages in Tensor Memory; slots2 = sum of ceil(degree / 2) over the item's rows.
bool list_ll_item_supported(int Z, int E, int n_rows, int max_deg, int slots2);
size_t list_ll_smem_bytes(int E, int n_cols, int Z, int n_tx);
// kernel: a compiled list kernel (list_jit_kernel), or null for the generic one.
ldpc_status launch_list_ll(const ListItem *d_items, int n_items, int *d_counter, size_t smem,
                           int early_stop, cudaStream_t stream, const void *kernel = nullptr);
// Work-list kernels compiled for a set of row sequences (list_jit.cu): the module new
// work lists use (null: none prepared), its kernel, and the case of a graph's first n_rows
// rows in it (-1: not among its sequences, the item takes the generic row loop).
// NVRTC front end (jit_common.cu): the fixed-width type prelude of a runtime-compiled
// source, and source to cubin for sm_103a (empty on failure; host work only).
const char *jit_prelude();
std::vector<char> jit_compile(const std::string &src, const char *name);
// Registry of runtime-compiled kernels (jit_common.cu), one per key: the kernel `kernel`
// of the module built from source() (compiled in the background, or waited for in mode 2;
// null while not ready, when compilation is off or failed); jit_prepare compiles and waits
// without loading.  Mode 0 off, 1 background (default), 2 blocking; jit_set_mode returns the
// previous mode plus 4 once a kernel has loaded and 8 once a compilation or load failed.
int jit_mode();
int jit_set_mode(int mode);
const void *jit_kernel(const std::string &key, const std::function<std::string()> &source,
                       const char *name, const char *kernel);
bool jit_prepare(const std::string &key, const std::function<std::string()> &source,
                 const char *name);
struct ListModule;
const ListModule *list_jit_active();
const void *list_jit_kernel(const ListModule *m);
int list_jit_seq(const ListModule *m, Graph *g, int n_rows);
ldpc_status launch_list(const ListItem *d_items, int n_items, int *d_counter, size_t smem,
                        int early_stop, cudaStream_t stream);

// Work-list decode whose work table and counter sit in a static device array
// (decode_rowpair.cu); h_items is sorted host-side already; ll selects the low-latency
// list kernel (smem is then its request).
constexpr int kNoAllocMaxItems = 2048;
ldpc_status launch_list_noalloc(const ListItem *h_items, int n_items, size_t smem,
                                int early_stop, bool ll, cudaStream_t stream);

void count_launch();

// Every device and pinned-host allocation the library makes goes through these two
// (counted, exported through ldpc_alloc_count()).
cudaError_t dev_alloc(void **p, size_t bytes);
cudaError_t pinned_alloc(void **p, size_t bytes);

// Launch set-up kept off the per-call path: a kernel's dynamic shared-memory limit is set
// only when a launch asks for a different amount than the last one on this device, and
// occupancy answers are remembered per (kernel, device, threads, dynamic shared memory).
// Both return what the CUDA runtime call they stand for would have returned.
cudaError_t set_dyn_smem(const void *kernel, size_t smem);
cudaError_t blocks_per_sm(int *per_sm, const void *kernel, int threads, size_t smem);

}  // namespace ldpc
