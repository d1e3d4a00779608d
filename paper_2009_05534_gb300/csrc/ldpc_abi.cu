// C-ABI entry points: graph construction (paper Sec. II code model) and the decode calls
// (Sec. III layered min-sum over a batch, Sec. IV).  Host-side validation only; all
// decoding work runs in the kernels of decode_layered.cu.
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <tuple>
#include <utility>
#include <vector>

#include "ldpc_internal.h"

namespace ldpc {

static std::atomic<uint64_t> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

static std::atomic<uint64_t> g_allocs{0};
cudaError_t dev_alloc(void **p, size_t bytes) {
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    return cudaMalloc(p, bytes);
}
cudaError_t pinned_alloc(void **p, size_t bytes) {
    g_allocs.fetch_add(1, std::memory_order_relaxed);
    return cudaMallocHost(p, bytes);
}

static std::mutex g_attr_mu;
static std::map<std::pair<const void *, int>, size_t> g_dyn_smem;
static std::map<std::tuple<const void *, int, int, size_t>, int> g_occupancy;

cudaError_t set_dyn_smem(const void *kernel, size_t smem) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_attr_mu);
    const auto key = std::make_pair(kernel, dev);
    const auto it = g_dyn_smem.find(key);
    if (it != g_dyn_smem.end() && it->second == smem) return cudaSuccess;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        g_dyn_smem[key] = smem;
    else
        g_dyn_smem.erase(key);
    return e;
}

cudaError_t blocks_per_sm(int *per_sm, const void *kernel, int threads, size_t smem) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_attr_mu);
    const auto key = std::make_tuple(kernel, dev, threads, smem);
    const auto it = g_occupancy.find(key);
    if (it != g_occupancy.end()) {
        *per_sm = it->second;
        return cudaSuccess;
    }
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kernel, threads, smem);
    if (e == cudaSuccess) g_occupancy[key] = *per_sm;
    return e;
}

// Per-(device, stream) workspace of the work-list decode: device work table + counter, and
// a pinned host staging copy of the table guarded by an event.
struct ListWorkspace {
    ListItem *d_items = nullptr;
    int *d_counter = nullptr;
    ListItem *h_items = nullptr;
    size_t cap = 0;
    cudaEvent_t copied = nullptr;
    // row maps of ldpc_decode_rows_host_maps: [in rows | out rows], pinned and device
    int32_t *d_maps = nullptr;
    int32_t *h_maps = nullptr;
    size_t map_cap = 0;             // codewords
    cudaEvent_t maps_copied = nullptr;
};
static std::mutex g_ws_mu;
static std::map<std::pair<int, cudaStream_t>, ListWorkspace> g_ws;

int *graph_queue(Graph *g, cudaStream_t stream) {
    std::lock_guard<std::mutex> lk(g->q_mu);
    for (int k = 0; k < g->n_queues; ++k)
        if (g->q_stream[k] == stream) return g->d_queues + 2 * k;
    if (g->n_queues == Graph::kQueues) return nullptr;
    g->q_stream[g->n_queues] = stream;
    return g->d_queues + 2 * g->n_queues++;
}

}  // namespace ldpc

using ldpc::Graph;

extern "C" {

void ldpc_decode_opts_default(ldpc_decode_opts *o) {
    if (!o) return;
    o->llr_type = LDPC_LLR_INT8;
    o->algo = LDPC_OFFSET;
    o->alpha = 0.75f;
    o->offset = 0.0f;
    o->offset_q = 1;
    o->n_rows = 0;
    o->n_tx = 0;
    o->punct_cols = 2;
    o->early_stop = 1;
    o->cluster_size = 1;
    o->threads_per_row = 0;
    o->learned_params = nullptr;
}

const char *ldpc_status_string(ldpc_status s) {
    switch (s) {
    case LDPC_OK: return "LDPC_OK";
    case LDPC_ERR_INVALID_ARG: return "LDPC_ERR_INVALID_ARG";
    case LDPC_ERR_UNSUPPORTED: return "LDPC_ERR_UNSUPPORTED";
    case LDPC_ERR_OUT_OF_MEMORY: return "LDPC_ERR_OUT_OF_MEMORY";
    case LDPC_ERR_CUDA: return "LDPC_ERR_CUDA";
    case LDPC_ERR_TIMEOUT: return "LDPC_ERR_TIMEOUT";
    }
    return "LDPC_ERR_UNKNOWN";
}

uint64_t ldpc_launch_count(void) { return ldpc::g_launches.load(); }

uint64_t ldpc_alloc_count(void) { return ldpc::g_allocs.load(); }

ldpc_status ldpc_graph_create(const int16_t *base, int M_bg, int N_bg, int K_b, int Z,
                              ldpc_graph_t *out) {
    if (!out) return LDPC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!base || M_bg < 1 || M_bg > ldpc::kMaxRows || N_bg < 2 || N_bg > ldpc::kMaxCols ||
        K_b < 1 || K_b >= N_bg || Z < 1 || Z > ldpc::kMaxZ)
        return LDPC_ERR_INVALID_ARG;
    int E = 0;
    for (int k = 0; k < M_bg * N_bg; ++k) {
        if (base[k] < -1) return LDPC_ERR_INVALID_ARG;
        if (base[k] >= 0) ++E;
    }
    if (E == 0) return LDPC_ERR_INVALID_ARG;
    Graph *g = new (std::nothrow) Graph;
    if (!g) return LDPC_ERR_OUT_OF_MEMORY;
    g->M_bg = M_bg;
    g->N_bg = N_bg;
    g->K_b = K_b;
    g->Z = Z;
    g->E_total = E;
    uint32_t *h_edges = g->h_edges;
    int e = 0, maxc = -1, maxd = 0, mind = 1 << 30, slots2 = 0;
    for (int r = 0; r < M_bg; ++r) {
        g->row_ptr[r] = e;
        g->max_col_upto[r] = maxc;
        g->max_deg_upto[r] = maxd;
        g->min_deg_upto[r] = mind;
        g->slots2_upto[r] = slots2;
        int d = 0;
        for (int c = 0; c < N_bg; ++c) {
            const int v = base[r * N_bg + c];
            if (v < 0) continue;
            h_edges[e++] = ((uint32_t)c << 16) | (uint32_t)(v % Z);
            if (c > maxc) maxc = c;
            ++d;
        }
        if (d > maxd) maxd = d;
        if (d < mind) mind = d;
        slots2 += (d + 1) / 2;
    }
    g->slots2_upto[M_bg] = slots2;
    g->row_ptr[M_bg] = e;
    g->max_col_upto[M_bg] = maxc;
    g->max_deg_upto[M_bg] = maxd;
    g->min_deg_upto[M_bg] = mind;
    cudaGetDevice(&g->device);
    ldpc_status st = LDPC_OK;
    const size_t q_bytes = sizeof(int) * 2 * Graph::kQueues;
    if (ldpc::dev_alloc((void **)&g->d_edges, sizeof(uint32_t) * E) != cudaSuccess ||
        ldpc::dev_alloc((void **)&g->d_row_ptr, sizeof(int) * (M_bg + 1)) != cudaSuccess ||
        ldpc::dev_alloc((void **)&g->d_status, sizeof(int)) != cudaSuccess ||
        ldpc::dev_alloc((void **)&g->d_queues, q_bytes) != cudaSuccess) {
        st = LDPC_ERR_OUT_OF_MEMORY;
    } else if (cudaMemcpy(g->d_edges, h_edges, sizeof(uint32_t) * E, cudaMemcpyHostToDevice) !=
                   cudaSuccess ||
               cudaMemcpy(g->d_row_ptr, g->row_ptr, sizeof(int) * (M_bg + 1),
                          cudaMemcpyHostToDevice) != cudaSuccess ||
               cudaMemset(g->d_status, 0, sizeof(int)) != cudaSuccess ||
               cudaMemset(g->d_queues, 0, q_bytes) != cudaSuccess) {
        st = LDPC_ERR_CUDA;
    }
    if (st != LDPC_OK) {
        cudaGetLastError();
        cudaFree(g->d_edges);
        cudaFree(g->d_row_ptr);
        cudaFree(g->d_status);
        cudaFree(g->d_queues);
        delete g;
        return st;
    }
    *out = reinterpret_cast<ldpc_graph_t>(g);
    return LDPC_OK;
}

ldpc_status ldpc_graph_destroy(ldpc_graph_t h) {
    if (!h) return LDPC_ERR_INVALID_ARG;
    Graph *g = reinterpret_cast<Graph *>(h);
    cudaDeviceSynchronize();
    cudaFree(g->d_edges);
    cudaFree(g->d_row_ptr);
    cudaFree(g->d_status);
    cudaFree(g->d_queues);
    cudaFree(g->d_stage);
    for (int k = 0; k < Graph::kHostChunks; ++k)
        if (g->chunk_ev[k]) cudaEventDestroy(g->chunk_ev[k]);
    if (g->copy_stream) cudaStreamDestroy(g->copy_stream);
    delete g;
    return LDPC_OK;
}

int ldpc_graph_edges(ldpc_graph_t h, int n_rows) {
    if (!h) return -1;
    Graph *g = reinterpret_cast<Graph *>(h);
    if (n_rows == 0) n_rows = g->M_bg;
    if (n_rows < 1 || n_rows > g->M_bg) return -1;
    return g->row_ptr[n_rows];
}

int ldpc_graph_vars(ldpc_graph_t h, int n_rows) {
    if (!h) return -1;
    Graph *g = reinterpret_cast<Graph *>(h);
    if (n_rows == 0) n_rows = g->M_bg;
    if (n_rows < 1 || n_rows > g->M_bg) return -1;
    return (g->K_b + n_rows) * g->Z;
}

// Validates the arguments of a batch decode and fills the kernel parameters; *empty is
// set for a zero batch (nothing to launch).  flooding: the flooding decoder's rules.
static ldpc_status decode_params(ldpc_graph_t h, const void *llr, int batch, int max_iter,
                                 const ldpc_decode_opts *opts, uint8_t *bits, int32_t *iters,
                                 void *post, void *c2v, bool flooding, ldpc::DecodeParams *out,
                                 ldpc_decode_opts *o_out, bool *empty) {
    *empty = false;
    if (!h) return LDPC_ERR_INVALID_ARG;
    Graph *g = reinterpret_cast<Graph *>(h);
    ldpc_decode_opts o;
    if (opts)
        o = *opts;
    else
        ldpc_decode_opts_default(&o);
    if (batch < 0 || max_iter < 1 || max_iter > ldpc::kMaxIter) return LDPC_ERR_INVALID_ARG;
    if (o.llr_type < LDPC_LLR_INT8 || o.llr_type > LDPC_LLR_FP32) return LDPC_ERR_INVALID_ARG;
    if (o.algo < LDPC_NORMALISED || o.algo > LDPC_SUM_PRODUCT) return LDPC_ERR_INVALID_ARG;
    if (flooding) {
        if (o.llr_type != LDPC_LLR_FP32 || o.algo == LDPC_LEARNED) return LDPC_ERR_UNSUPPORTED;
    } else if (o.algo == LDPC_SUM_PRODUCT) {
        return LDPC_ERR_UNSUPPORTED;
    }
    if (o.llr_type == LDPC_LLR_INT8 && o.algo != LDPC_OFFSET) return LDPC_ERR_UNSUPPORTED;
    if (o.algo == LDPC_LEARNED && !o.learned_params) return LDPC_ERR_INVALID_ARG;
    if (o.cluster_size != 1 && o.cluster_size != 2) return LDPC_ERR_INVALID_ARG;
    if (o.cluster_size == 2 &&
        (o.llr_type != LDPC_LLR_INT8 || flooding || (o.threads_per_row != 0 && o.threads_per_row != 2)))
        return LDPC_ERR_UNSUPPORTED;
    if (o.threads_per_row != 0 && o.threads_per_row != 1 && o.threads_per_row != 2 &&
        o.threads_per_row != 4)
        return LDPC_ERR_INVALID_ARG;
    if (o.threads_per_row > 1 && (o.llr_type != LDPC_LLR_INT8 || flooding))
        return LDPC_ERR_UNSUPPORTED;
    const int n_rows = o.n_rows == 0 ? g->M_bg : o.n_rows;
    if (n_rows < 1 || n_rows > g->M_bg) return LDPC_ERR_INVALID_ARG;
    const int n_cols = g->K_b + n_rows;
    if (n_cols > g->N_bg || g->max_col_upto[n_rows] >= n_cols) return LDPC_ERR_INVALID_ARG;
    // every used check row needs two edges (a min over the other edges must exist)
    if (g->min_deg_upto[n_rows] < 2) return LDPC_ERR_UNSUPPORTED;
    if (o.punct_cols < 0 || o.punct_cols > n_cols) return LDPC_ERR_INVALID_ARG;
    const int n_tx = o.n_tx == 0 ? (n_cols - o.punct_cols) * g->Z : o.n_tx;
    // (written without a sum that a huge n_tx could overflow)
    if (n_tx < 0 || n_tx > (n_cols - o.punct_cols) * g->Z) return LDPC_ERR_INVALID_ARG;
    if (batch == 0) {
        *empty = true;
        return LDPC_OK;
    }
    if (!llr || !bits || !iters) return LDPC_ERR_INVALID_ARG;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != g->device) return LDPC_ERR_INVALID_ARG;

    ldpc::DecodeParams &p = *out;
    p.edges = g->d_edges;
    p.row_ptr = g->d_row_ptr;
    p.h_edges = g->h_edges;
    p.h_row_ptr = g->row_ptr;
    p.n_rows = n_rows;
    p.E = g->row_ptr[n_rows];
    p.Z = g->Z;
    p.n_cols = n_cols;
    p.K_b = g->K_b;
    p.max_deg = g->max_deg_upto[n_rows];
    p.punct = o.punct_cols;
    p.n_tx = n_tx;
    p.max_iter = max_iter;
    p.early_stop = o.early_stop ? 1 : 0;
    p.batch = batch;
    p.algo = o.algo;
    p.alpha = o.alpha;
    p.offset = o.offset;
    p.offset_q = o.offset_q;
    p.learned = o.learned_params;
    p.llr = llr;
    p.bits = bits;
    p.iters = iters;
    p.post = post;
    p.c2v = c2v;
    p.status = g->d_status;
    p.in_rows = nullptr;
    p.out_rows = nullptr;
    p.threads_per_row = o.threads_per_row;
    p.cluster_size = o.cluster_size;
    p.queue = nullptr;
    *o_out = o;
    return LDPC_OK;
}

static ldpc_status decode_common(ldpc_graph_t h, const void *llr, int batch, int max_iter,
                                 ldpc_stream_t stream, const ldpc_decode_opts *opts,
                                 uint8_t *bits, int32_t *iters, void *post, void *c2v) {
    ldpc::DecodeParams p;
    ldpc_decode_opts o;
    bool empty = false;
    const ldpc_status st = decode_params(h, llr, batch, max_iter, opts, bits, iters, post, c2v,
                                         false, &p, &o, &empty);
    if (st != LDPC_OK || empty) return st;
    p.queue = ldpc::graph_queue(reinterpret_cast<Graph *>(h), reinterpret_cast<cudaStream_t>(stream));
    return ldpc::launch_layered(p, o.llr_type, reinterpret_cast<cudaStream_t>(stream));
}

ldpc_status ldpc_decode(ldpc_graph_t g, const void *llr_dev, int batch, int max_iter,
                        ldpc_stream_t stream, const ldpc_decode_opts *opts,
                        uint8_t *hard_bits_dev, int32_t *iters_dev) {
    return decode_common(g, llr_dev, batch, max_iter, stream, opts, hard_bits_dev, iters_dev,
                         nullptr, nullptr);
}

ldpc_status ldpc_decode_rows(ldpc_graph_t g, const void *llr_dev, const int32_t *in_rows_dev,
                             const int32_t *out_rows_dev, int batch, int max_iter,
                             ldpc_stream_t stream, const ldpc_decode_opts *opts,
                             uint8_t *hard_bits_dev, int32_t *iters_dev) {
    ldpc::DecodeParams p;
    ldpc_decode_opts o;
    bool empty = false;
    const ldpc_status st = decode_params(g, llr_dev, batch, max_iter, opts, hard_bits_dev,
                                         iters_dev, nullptr, nullptr, false, &p, &o, &empty);
    if (st != LDPC_OK || empty) return st;
    if (!in_rows_dev || !out_rows_dev) return LDPC_ERR_INVALID_ARG;
    p.in_rows = in_rows_dev;
    p.out_rows = out_rows_dev;
    p.queue = ldpc::graph_queue(reinterpret_cast<Graph *>(g), reinterpret_cast<cudaStream_t>(stream));
    return ldpc::launch_layered(p, o.llr_type, reinterpret_cast<cudaStream_t>(stream));
}

ldpc_status ldpc_decode_rows_host_maps(ldpc_graph_t g, const void *llr_dev,
                                       const int32_t *in_rows_host,
                                       const int32_t *out_rows_host, int batch, int max_iter,
                                       ldpc_stream_t stream, const ldpc_decode_opts *opts,
                                       uint8_t *hard_bits_dev, int32_t *iters_dev) {
    ldpc::DecodeParams p;
    ldpc_decode_opts o;
    bool empty = false;
    const ldpc_status st = decode_params(g, llr_dev, batch, max_iter, opts, hard_bits_dev,
                                         iters_dev, nullptr, nullptr, false, &p, &o, &empty);
    if (st != LDPC_OK || empty) return st;
    if (!in_rows_host || !out_rows_host) return LDPC_ERR_INVALID_ARG;
    for (int b = 0; b < batch; ++b)
        if (in_rows_host[b] < 0 || out_rows_host[b] < 0) return LDPC_ERR_INVALID_ARG;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LDPC_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lk(ldpc::g_ws_mu);
    ldpc::ListWorkspace &ws = ldpc::g_ws[std::make_pair(dev, s)];
    if (ws.map_cap < (size_t)batch) {
        if (ws.maps_copied) cudaEventSynchronize(ws.maps_copied);
        cudaFree(ws.d_maps);
        cudaFreeHost(ws.h_maps);
        ws.d_maps = nullptr;
        ws.h_maps = nullptr;
        ws.map_cap = 0;
        size_t cap = 256;
        while (cap < (size_t)batch) cap *= 2;
        if (ldpc::dev_alloc((void **)&ws.d_maps, 2 * cap * sizeof(int32_t)) != cudaSuccess ||
            ldpc::pinned_alloc((void **)&ws.h_maps, 2 * cap * sizeof(int32_t)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(ws.d_maps);
            cudaFreeHost(ws.h_maps);
            ws.d_maps = nullptr;
            ws.h_maps = nullptr;
            return LDPC_ERR_OUT_OF_MEMORY;
        }
        ws.map_cap = cap;
    }
    if (!ws.maps_copied &&
        cudaEventCreateWithFlags(&ws.maps_copied, cudaEventDisableTiming) != cudaSuccess)
        return LDPC_ERR_CUDA;
    // the pinned staging copy may still feed the previous call's upload; the device copy is
    // ordered after the previous launch on this stream
    if (cudaEventSynchronize(ws.maps_copied) != cudaSuccess) return LDPC_ERR_CUDA;
    std::memcpy(ws.h_maps, in_rows_host, (size_t)batch * sizeof(int32_t));
    std::memcpy(ws.h_maps + batch, out_rows_host, (size_t)batch * sizeof(int32_t));
    if (cudaMemcpyAsync(ws.d_maps, ws.h_maps, 2 * (size_t)batch * sizeof(int32_t),
                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaEventRecord(ws.maps_copied, s) != cudaSuccess)
        return LDPC_ERR_CUDA;
    p.in_rows = ws.d_maps;
    p.out_rows = ws.d_maps + batch;
    p.queue = ldpc::graph_queue(reinterpret_cast<Graph *>(g), s);
    return ldpc::launch_layered(p, o.llr_type, s);
}

ldpc_status ldpc_decode_debug(ldpc_graph_t g, const void *llr_dev, int batch, int max_iter,
                              ldpc_stream_t stream, const ldpc_decode_opts *opts,
                              uint8_t *hard_bits_dev, int32_t *iters_dev, void *post_dev,
                              void *c2v_dev) {
    return decode_common(g, llr_dev, batch, max_iter, stream, opts, hard_bits_dev, iters_dev,
                         post_dev, c2v_dev);
}

ldpc_status ldpc_decode_host(ldpc_graph_t h, const void *llr_host, int batch, int max_iter,
                             ldpc_stream_t stream, const ldpc_decode_opts *opts,
                             uint8_t *hard_bits_host, int32_t *iters_host) {
    if (!h) return LDPC_ERR_INVALID_ARG;
    Graph *g = reinterpret_cast<Graph *>(h);
    ldpc_decode_opts o;
    if (opts)
        o = *opts;
    else
        ldpc_decode_opts_default(&o);
    // every argument is checked before anything is allocated or copied (the decode's own
    // checks; the pointers here are host pointers, which it only tests for null)
    {
        ldpc::DecodeParams pv;
        ldpc_decode_opts ov;
        bool empty = false;
        const ldpc_status st = decode_params(h, llr_host, batch, max_iter, &o, hard_bits_host,
                                             iters_host, nullptr, nullptr, false, &pv, &ov,
                                             &empty);
        if (st != LDPC_OK || empty) return st;
    }
    const int n_rows = o.n_rows == 0 ? g->M_bg : o.n_rows;
    if (n_rows < 1 || n_rows > g->M_bg || o.punct_cols < 0) return LDPC_ERR_INVALID_ARG;
    const int n_cols = g->K_b + n_rows;
    const int n_tx = o.n_tx == 0 ? (n_cols - o.punct_cols) * g->Z : o.n_tx;
    if (n_tx < 0) return LDPC_ERR_INVALID_ARG;
    const size_t esz = o.llr_type == LDPC_LLR_INT8 ? 1 : (o.llr_type == LDPC_LLR_FP16 ? 2 : 4);
    const size_t nbytes = (size_t)(g->K_b * g->Z + 7) / 8;
    const size_t in_b = (size_t)batch * n_tx * esz;
    const size_t bits_b = (size_t)batch * nbytes;
    const size_t it_b = (size_t)batch * sizeof(int32_t);
    auto up = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t need = up(in_b) + up(bits_b) + up(it_b);
    std::lock_guard<std::mutex> lk(g->host_mu);
    if (need > g->stage_bytes) {
        cudaFree(g->d_stage);
        g->d_stage = nullptr;
        g->stage_bytes = 0;
        if (ldpc::dev_alloc((void **)&g->d_stage, need) != cudaSuccess) {
            cudaGetLastError();
            return LDPC_ERR_OUT_OF_MEMORY;
        }
        g->stage_bytes = need;
    }
    if (!g->copy_stream) {
        if (cudaStreamCreateWithFlags(&g->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
            return LDPC_ERR_CUDA;
        for (int k = 0; k < Graph::kHostChunks; ++k)
            if (cudaEventCreateWithFlags(&g->chunk_ev[k], cudaEventDisableTiming) != cudaSuccess)
                return LDPC_ERR_CUDA;
    }
    char *base = (char *)g->d_stage;
    char *d_llr = base;
    uint8_t *d_bits = (uint8_t *)(base + up(in_b));
    int32_t *d_it = (int32_t *)(base + up(in_b) + up(bits_b));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    // Pipeline: the inputs go up in chunks on the graph's copy stream, and the decode of
    // chunk k waits only for chunk k's upload, so later uploads overlap earlier decodes;
    // each chunk's outputs come back on `stream` right after its decode.  Chunks grow
    // geometrically (up to 8 times the previous one): an upload is more than ten times
    // faster than the decode of the same codewords, so each still hides behind the decode
    // before it, and the batch kernel, which balances codewords over the SMs by itself,
    // runs as few launches as that allows (each launch pays its own ramp-up and last round).
    int dev = 0, n_sm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
    // chunk k covers codewords [start[k], start[k + 1]); for int8 the first chunk is one
    // codeword per SM (decoded by the low-latency kernel in about the time of a full
    // round), which halves the upload that nothing overlaps
    int start[Graph::kHostChunks + 1];
    int n_chunks = 0;
    {
        int chunk = (o.llr_type == LDPC_LLR_INT8 && batch > 2 * n_sm) ? n_sm : 2 * n_sm;
        start[0] = 0;
        int b = 0;
        while (b < batch) {
            // the last chunk takes the rest
            const int rest = batch - b;
            const int c = (n_chunks + 1 == Graph::kHostChunks || chunk >= rest) ? rest : chunk;
            b += c;
            start[++n_chunks] = b;
            chunk = c > batch / 8 ? batch : 8 * c;
        }
    }
    for (int k = 0; k < n_chunks; ++k) {
        const size_t b0 = (size_t)start[k];
        const size_t nb = (size_t)(start[k + 1] - start[k]);
        if (cudaMemcpyAsync(d_llr + b0 * n_tx * esz, (const char *)llr_host + b0 * n_tx * esz,
                            nb * n_tx * esz, cudaMemcpyHostToDevice,
                            g->copy_stream) != cudaSuccess ||
            cudaEventRecord(g->chunk_ev[k], g->copy_stream) != cudaSuccess)
            return LDPC_ERR_CUDA;
    }
    for (int k = 0; k < n_chunks; ++k) {
        const size_t b0 = (size_t)start[k];
        const int nb = start[k + 1] - start[k];
        if (cudaStreamWaitEvent(s, g->chunk_ev[k], 0) != cudaSuccess) return LDPC_ERR_CUDA;
        ldpc_status st = decode_common(h, d_llr + b0 * n_tx * esz, nb, max_iter, stream, &o,
                                       d_bits + b0 * nbytes, d_it + b0, nullptr, nullptr);
        if (st != LDPC_OK) {
            cudaStreamSynchronize(g->copy_stream);
            cudaStreamSynchronize(s);
            return st;
        }
        if (cudaMemcpyAsync(hard_bits_host + b0 * nbytes, d_bits + b0 * nbytes, nb * nbytes,
                            cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(iters_host + b0, d_it + b0, nb * sizeof(int32_t),
                            cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return LDPC_ERR_CUDA;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess) return LDPC_ERR_CUDA;
    return LDPC_OK;
}

ldpc_status ldpc_decode_list(const ldpc_work_item *items, int n_items, ldpc_stream_t stream,
                             const ldpc_decode_opts *opts) {
    if (n_items < 0 || (n_items > 0 && !items)) return LDPC_ERR_INVALID_ARG;
    ldpc_decode_opts o;
    if (opts)
        o = *opts;
    else
        ldpc_decode_opts_default(&o);
    if (o.llr_type != LDPC_LLR_INT8 || o.algo != LDPC_OFFSET || o.offset_q != 1 ||
        o.punct_cols != 2 || o.cluster_size != 1)
        return LDPC_ERR_UNSUPPORTED;
    if (o.threads_per_row < 0 || o.threads_per_row > 4 || o.threads_per_row == 3)
        return LDPC_ERR_INVALID_ARG;
    if (o.threads_per_row == 4) return LDPC_ERR_UNSUPPORTED;
    if (n_items == 0) return LDPC_OK;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LDPC_ERR_CUDA;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    std::vector<std::pair<double, ldpc::ListItem>> v;
    v.reserve((size_t)n_items);
    size_t smem = 0, smem_ll = 0;
    bool ll_ok = o.threads_per_row != 1;
    // the compiled list kernel of the graphs' row sequences, if one has been prepared
    const ldpc::ListModule *lm = ll_ok ? ldpc::list_jit_active() : nullptr;
    for (int k = 0; k < n_items; ++k) {
        const ldpc_work_item &w = items[k];
        if (!w.graph || !w.llr || !w.hard_bits || !w.iters) return LDPC_ERR_INVALID_ARG;
        Graph *g = reinterpret_cast<Graph *>(w.graph);
        if (g->device != dev) return LDPC_ERR_INVALID_ARG;
        const int n_rows = w.n_rows == 0 ? g->M_bg : w.n_rows;
        if (n_rows < 1 || n_rows > g->M_bg || w.max_iter < 1 || w.max_iter > ldpc::kMaxIter)
            return LDPC_ERR_INVALID_ARG;
        const int n_cols = g->K_b + n_rows;
        if (n_cols > g->N_bg || g->max_col_upto[n_rows] >= n_cols) return LDPC_ERR_INVALID_ARG;
        const int n_tx = w.n_tx == 0 ? (n_cols - 2) * g->Z : w.n_tx;
        if (n_tx < 0 || n_tx > (n_cols - 2) * g->Z) return LDPC_ERR_INVALID_ARG;
        const int E = g->row_ptr[n_rows];
        if (g->min_deg_upto[n_rows] < 2 ||
            !ldpc::list_item_supported(g->Z, E, n_rows, g->max_deg_upto[n_rows]))
            return LDPC_ERR_UNSUPPORTED;
        ldpc::ListItem it;
        it.edges = g->d_edges;
        it.row_ptr = g->d_row_ptr;
        it.llr = static_cast<const int8_t *>(w.llr);
        it.bits = w.hard_bits;
        it.iters = w.iters;
        it.Z = g->Z;
        it.K_b = g->K_b;
        it.n_rows = n_rows;
        it.n_cols = n_cols;
        it.E = E;
        it.n_tx = n_tx;
        it.punct = 2;
        it.max_iter = w.max_iter;
        it.seq = ldpc::list_jit_seq(lm, g, n_rows);
        smem = std::max(smem, ldpc::list_item_smem_bytes(E, n_rows, n_cols, g->Z));
        ll_ok = ll_ok && ldpc::list_ll_item_supported(g->Z, E, n_rows, g->max_deg_upto[n_rows],
                                                      g->slots2_upto[n_rows]);
        smem_ll = std::max(smem_ll, ldpc::list_ll_smem_bytes(E, n_cols, g->Z, n_tx));
        v.emplace_back((double)E * g->Z * w.max_iter, it);
    }
    ll_ok = ll_ok && smem_ll <= (size_t)optin;
    if (o.threads_per_row == 2 && !ll_ok) return LDPC_ERR_UNSUPPORTED;
    // largest items first: the dynamic work counter then balances the tail
    std::stable_sort(v.begin(), v.end(),
                     [](const auto &a, const auto &b) { return a.first > b.first; });
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    std::lock_guard<std::mutex> lk(ldpc::g_ws_mu);
    ldpc::ListWorkspace &ws = ldpc::g_ws[std::make_pair(dev, s)];
    if (ws.cap < (size_t)n_items) {
        if (ws.copied) cudaEventSynchronize(ws.copied);
        cudaFree(ws.d_items);
        cudaFreeHost(ws.h_items);
        ws.d_items = nullptr;
        ws.h_items = nullptr;
        ws.cap = 0;
        size_t cap = 256;
        while (cap < (size_t)n_items) cap *= 2;
        if (ldpc::dev_alloc((void **)&ws.d_items, cap * sizeof(ldpc::ListItem)) != cudaSuccess ||
            ldpc::pinned_alloc((void **)&ws.h_items, cap * sizeof(ldpc::ListItem)) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(ws.d_items);
            cudaFreeHost(ws.h_items);
            ws.d_items = nullptr;
            ws.h_items = nullptr;
            return LDPC_ERR_OUT_OF_MEMORY;
        }
        ws.cap = cap;
    }
    if (!ws.d_counter && ldpc::dev_alloc((void **)&ws.d_counter, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return LDPC_ERR_OUT_OF_MEMORY;
    }
    if (!ws.copied && cudaEventCreateWithFlags(&ws.copied, cudaEventDisableTiming) != cudaSuccess)
        return LDPC_ERR_CUDA;
    // the pinned staging copy may still feed the previous call's upload
    if (cudaEventSynchronize(ws.copied) != cudaSuccess) return LDPC_ERR_CUDA;
    for (int k = 0; k < n_items; ++k) ws.h_items[k] = v[(size_t)k].second;
    if (cudaMemcpyAsync(ws.d_items, ws.h_items, (size_t)n_items * sizeof(ldpc::ListItem),
                        cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaEventRecord(ws.copied, s) != cudaSuccess ||
        cudaMemsetAsync(ws.d_counter, 0, sizeof(int), s) != cudaSuccess)
        return LDPC_ERR_CUDA;
    if (ll_ok)
        return ldpc::launch_list_ll(ws.d_items, n_items, ws.d_counter, smem_ll,
                                    o.early_stop ? 1 : 0, s, ldpc::list_jit_kernel(lm));
    return ldpc::launch_list(ws.d_items, n_items, ws.d_counter, smem, o.early_stop ? 1 : 0, s);
}

// Validation for the allocation-free work list: writes the device items into the caller's
// fixed arrays and the launch order (largest work first) into order[0..n).
static ldpc_status prepare_list_noalloc(const ldpc_work_item *items, int n_items,
                                const ldpc_decode_opts *opts, ldpc::ListItem *out,
                                int *order, double *work, size_t *smem_out, int *early_stop,
                                size_t *smem_ll_out, bool *ll_out) {
    ldpc_decode_opts o;
    if (opts)
        o = *opts;
    else
        ldpc_decode_opts_default(&o);
    if (o.llr_type != LDPC_LLR_INT8 || o.algo != LDPC_OFFSET || o.offset_q != 1 ||
        o.punct_cols != 2 || o.cluster_size != 1)
        return LDPC_ERR_UNSUPPORTED;
    if (o.threads_per_row < 0 || o.threads_per_row > 4 || o.threads_per_row == 3)
        return LDPC_ERR_INVALID_ARG;
    if (o.threads_per_row == 4) return LDPC_ERR_UNSUPPORTED;
    *early_stop = o.early_stop ? 1 : 0;
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return LDPC_ERR_CUDA;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    size_t smem = 0, smem_ll = 0;
    bool ll_ok = o.threads_per_row != 1;
    for (int k = 0; k < n_items; ++k) {
        const ldpc_work_item &w = items[k];
        if (!w.graph || !w.llr || !w.hard_bits || !w.iters) return LDPC_ERR_INVALID_ARG;
        Graph *g = reinterpret_cast<Graph *>(w.graph);
        if (g->device != dev) return LDPC_ERR_INVALID_ARG;
        const int n_rows = w.n_rows == 0 ? g->M_bg : w.n_rows;
        if (n_rows < 1 || n_rows > g->M_bg || w.max_iter < 1 || w.max_iter > ldpc::kMaxIter)
            return LDPC_ERR_INVALID_ARG;
        const int n_cols = g->K_b + n_rows;
        if (n_cols > g->N_bg || g->max_col_upto[n_rows] >= n_cols) return LDPC_ERR_INVALID_ARG;
        const int n_tx = w.n_tx == 0 ? (n_cols - 2) * g->Z : w.n_tx;
        if (n_tx < 0 || n_tx > (n_cols - 2) * g->Z) return LDPC_ERR_INVALID_ARG;
        const int E = g->row_ptr[n_rows];
        if (g->min_deg_upto[n_rows] < 2 ||
            !ldpc::list_item_supported(g->Z, E, n_rows, g->max_deg_upto[n_rows]))
            return LDPC_ERR_UNSUPPORTED;
        ldpc::ListItem &it = out[k];
        it.edges = g->d_edges;
        it.row_ptr = g->d_row_ptr;
        it.llr = static_cast<const int8_t *>(w.llr);
        it.bits = w.hard_bits;
        it.iters = w.iters;
        it.Z = g->Z;
        it.K_b = g->K_b;
        it.n_rows = n_rows;
        it.n_cols = n_cols;
        it.E = E;
        it.n_tx = n_tx;
        it.punct = 2;
        it.max_iter = w.max_iter;
        it.seq = -1;                             // the generic list kernels only
        smem = std::max(smem, ldpc::list_item_smem_bytes(E, n_rows, n_cols, g->Z));
        ll_ok = ll_ok && ldpc::list_ll_item_supported(g->Z, E, n_rows, g->max_deg_upto[n_rows],
                                                      g->slots2_upto[n_rows]);
        smem_ll = std::max(smem_ll, ldpc::list_ll_smem_bytes(E, n_cols, g->Z, n_tx));
        order[k] = k;
        work[k] = (double)E * g->Z * w.max_iter;
    }
    // largest items first (ties keep list order): the dynamic work counter then balances
    // the tail.  std::sort works in place, so this path allocates nothing.
    std::sort(order, order + n_items, [work](int a, int b) {
        return work[a] > work[b] || (work[a] == work[b] && a < b);
    });
    ll_ok = ll_ok && smem_ll <= (size_t)optin;
    if (o.threads_per_row == 2 && !ll_ok) return LDPC_ERR_UNSUPPORTED;
    *smem_out = smem;
    *smem_ll_out = smem_ll;
    *ll_out = ll_ok;
    return LDPC_OK;
}

ldpc_status ldpc_decode_list_noalloc(const ldpc_work_item *items, int n_items,
                                     ldpc_stream_t stream, const ldpc_decode_opts *opts) {
    if (n_items < 0 || (n_items > 0 && !items)) return LDPC_ERR_INVALID_ARG;
    if (n_items > ldpc::kNoAllocMaxItems) return LDPC_ERR_INVALID_ARG;   // beyond the array
    if (n_items == 0) return LDPC_OK;
    // host-side working arrays are fixed-size statics: nothing on this path allocates
    static std::mutex mu;
    static ldpc::ListItem raw[ldpc::kNoAllocMaxItems], sorted[ldpc::kNoAllocMaxItems];
    static int order[ldpc::kNoAllocMaxItems];
    static double work[ldpc::kNoAllocMaxItems];
    std::lock_guard<std::mutex> lk(mu);
    size_t smem = 0, smem_ll = 0;
    int early_stop = 1;
    bool ll = false;
    ldpc_status st = prepare_list_noalloc(items, n_items, opts, raw, order, work, &smem,
                                          &early_stop, &smem_ll, &ll);
    if (st != LDPC_OK) return st;
    for (int k = 0; k < n_items; ++k) sorted[k] = raw[order[k]];
    return ldpc::launch_list_noalloc(sorted, n_items, ll ? smem_ll : smem, early_stop, ll,
                                     reinterpret_cast<cudaStream_t>(stream));
}

static ldpc_status learned_common(ldpc_graph_t h, int batch, int T, int n_rows_in, int n_tx_in,
                                  ldpc::DecodeParams *p) {
    if (!h || batch < 0 || T < 1 || T > ldpc::kMaxIter) return LDPC_ERR_INVALID_ARG;
    Graph *g = reinterpret_cast<Graph *>(h);
    const int n_rows = n_rows_in == 0 ? g->M_bg : n_rows_in;
    if (n_rows < 1 || n_rows > g->M_bg) return LDPC_ERR_INVALID_ARG;
    const int n_cols = g->K_b + n_rows;
    if (n_cols > g->N_bg || g->max_col_upto[n_rows] >= n_cols) return LDPC_ERR_INVALID_ARG;
    if (g->min_deg_upto[n_rows] < 2) return LDPC_ERR_UNSUPPORTED;
    const int n_tx = n_tx_in == 0 ? (n_cols - 2) * g->Z : n_tx_in;
    if (n_tx < 0 || n_tx > (n_cols - 2) * g->Z) return LDPC_ERR_INVALID_ARG;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != g->device) return LDPC_ERR_INVALID_ARG;
    std::memset(p, 0, sizeof(*p));
    p->edges = g->d_edges;
    p->row_ptr = g->d_row_ptr;
    p->h_edges = g->h_edges;
    p->h_row_ptr = g->row_ptr;
    p->n_rows = n_rows;
    p->E = g->row_ptr[n_rows];
    p->Z = g->Z;
    p->n_cols = n_cols;
    p->K_b = g->K_b;
    p->max_deg = g->max_deg_upto[n_rows];
    p->punct = 2;
    p->n_tx = n_tx;
    p->max_iter = T;
    p->batch = batch;
    p->algo = LDPC_LEARNED;
    p->status = g->d_status;
    return LDPC_OK;
}

size_t ldpc_learned_workspace_floats(ldpc_graph_t h, int batch, int T, int n_rows) {
    ldpc::DecodeParams p;
    if (learned_common(h, batch, T, n_rows, 0, &p) != LDPC_OK) return 0;
    return (size_t)batch * ldpc::learned_ws_floats_per_cw(p.n_cols * p.Z, p.E * p.Z, T);
}

ldpc_status ldpc_learned_forward(ldpc_graph_t h, const float *llr, int batch, int T, int n_rows,
                                 int n_tx, const float *params, ldpc_stream_t stream, float *post,
                                 float *ws) {
    ldpc::DecodeParams p;
    ldpc_status st = learned_common(h, batch, T, n_rows, n_tx, &p);
    if (st != LDPC_OK) return st;
    if (batch == 0) return LDPC_OK;
    if (!llr || !params || !post || !ws) return LDPC_ERR_INVALID_ARG;
    return ldpc::launch_learned(p, T, params, llr, post, nullptr, nullptr, nullptr, ws, false,
                                reinterpret_cast<cudaStream_t>(stream));
}

ldpc_status ldpc_learned_backward(ldpc_graph_t h, const float *grad_post, int batch, int T,
                                  int n_rows, int n_tx, const float *params, ldpc_stream_t stream,
                                  float *ws, float *grad_params, float *grad_llr) {
    ldpc::DecodeParams p;
    ldpc_status st = learned_common(h, batch, T, n_rows, n_tx, &p);
    if (st != LDPC_OK) return st;
    if (batch == 0) return LDPC_OK;
    if (!grad_post || !params || !ws || !grad_params) return LDPC_ERR_INVALID_ARG;
    return ldpc::launch_learned(p, T, params, nullptr, nullptr, grad_post, grad_params, grad_llr,
                                ws, true, reinterpret_cast<cudaStream_t>(stream));
}

ldpc_status ldpc_learned_forward_iter(ldpc_graph_t h, const float *llr, int batch, int T,
                                      int n_rows, int n_tx, const float *params,
                                      ldpc_stream_t stream, float *post_iter, float *ws) {
    ldpc::DecodeParams p;
    ldpc_status st = learned_common(h, batch, T, n_rows, n_tx, &p);
    if (st != LDPC_OK) return st;
    if (batch == 0) return LDPC_OK;
    if (!llr || !params || !post_iter || !ws) return LDPC_ERR_INVALID_ARG;
    return ldpc::launch_learned(p, T, params, llr, nullptr, nullptr, nullptr, nullptr, ws, false,
                                reinterpret_cast<cudaStream_t>(stream), post_iter, nullptr);
}

ldpc_status ldpc_learned_backward_iter(ldpc_graph_t h, const float *grad_post_iter, int batch,
                                       int T, int n_rows, int n_tx, const float *params,
                                       ldpc_stream_t stream, float *ws, float *grad_params,
                                       float *grad_llr, int detach) {
    ldpc::DecodeParams p;
    ldpc_status st = learned_common(h, batch, T, n_rows, n_tx, &p);
    if (st != LDPC_OK) return st;
    if (batch == 0) return LDPC_OK;
    if (!grad_post_iter || !params || !ws || !grad_params) return LDPC_ERR_INVALID_ARG;
    return ldpc::launch_learned(p, T, params, nullptr, nullptr, nullptr, grad_params, grad_llr,
                                ws, true, reinterpret_cast<cudaStream_t>(stream), nullptr,
                                grad_post_iter, detach ? 1 : 0);
}

size_t ldpc_flooding_workspace_floats(ldpc_graph_t h, int batch, int n_rows) {
    if (!h || batch < 0) return 0;
    Graph *g = reinterpret_cast<Graph *>(h);
    const int r = n_rows == 0 ? g->M_bg : n_rows;
    if (r < 1 || r > g->M_bg) return 0;
    return (size_t)batch * ldpc::flooding_ws_floats_per_cw(g->row_ptr[r], g->Z);
}

ldpc_status ldpc_decode_flooding(ldpc_graph_t h, const float *llr, int batch, int max_iter,
                                 ldpc_stream_t stream, const ldpc_decode_opts *opts,
                                 uint8_t *bits, int32_t *iters, float *post, float *ws) {
    ldpc::DecodeParams p;
    ldpc_decode_opts o;
    bool empty = false;
    const ldpc_status st = decode_params(h, llr, batch, max_iter, opts, bits, iters, post,
                                         nullptr, true, &p, &o, &empty);
    if (st != LDPC_OK || empty) return st;
    if (!ws) return LDPC_ERR_INVALID_ARG;
    return ldpc::launch_flooding(p, ws, reinterpret_cast<cudaStream_t>(stream));
}

ldpc_status ldpc_graph_sync_status(ldpc_graph_t h, ldpc_stream_t stream) {
    if (!h) return LDPC_ERR_INVALID_ARG;
    Graph *g = reinterpret_cast<Graph *>(h);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int v = 0;
    if (cudaMemcpyAsync(&v, g->d_status, sizeof(int), cudaMemcpyDeviceToHost, s) !=
            cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return LDPC_ERR_CUDA;
    if (v != 0) {
        if (cudaMemsetAsync(g->d_status, 0, sizeof(int), s) != cudaSuccess) return LDPC_ERR_CUDA;
        cudaStreamSynchronize(s);
    }
    return (ldpc_status)v;
}

}  // extern "C"
