// Work-list kernels compiled at run time for a set of row sequences, and the one-codeword
// low-latency kernel compiled for one sequence (ll_jit_kernel, at the end: a lone
// BG1-shaped Z=384 codeword at 10 iterations 230 -> 162 us at alpha 2, 282 -> 206 us at
// alpha 4, bit-identical).  A serving slot's work
// list mixes base graphs, lifting sizes and rates, and the slot lasts as long as its
// largest item decoded alone by the low-latency list kernel (ll_kernel.cuh).  That kernel
// dispatches once per row on the row's degree; compiled with the row sequences of the
// graphs a server uses (LDPC_LL_SEQS), an item whose sequence is among them runs its layers
// as straight-line code, selected once per iteration, and any other item runs the generic
// row loop in the same launch.
//
// ldpc_list_jit_prepare compiles one module for a set of degree sequences (NVRTC, host
// work only) and makes it the next one; the following list launch loads it
// (cudaLibraryLoadData, valid in every context) and from then on work lists use it.  Loaded
// modules are kept for the process's lifetime, so a launch that chose a module keeps it
// even if another is prepared meanwhile.  Each graph remembers, per row count, the index
// of its sequence in the current module (one 64-bit word: module generation and index), so
// building a work list costs a lookup per item only when the module has changed.
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "f16x2.h"
#include "ldpc_internal.h"

namespace ldpc {

struct ListModule {
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kernel = nullptr;
    uint32_t generation = 0;
    std::map<std::string, int> index;     // degree-sequence key -> case of LDPC_LL_SEQS
};

namespace {

struct ListRegistry {
    std::mutex mu;                        // guards every member below
    std::mutex compile_mu;                // one compilation at a time
    const ListModule *active = nullptr;   // loaded, used by new work lists
    std::vector<char> pending;            // compiled, not loaded yet
    std::map<std::string, int> pending_index;
    bool clear = false;                   // a prepare with no sequences: stop using modules
    uint32_t generations = 0;
};
ListRegistry &registry() {
    static ListRegistry *r = new ListRegistry;   // never destroyed
    return *r;
}

constexpr int kA = 2;                     // cooperating threads per row pair (list kernel)

std::string key_of(const int *deg, int n) {
    std::string key;
    for (int r = 0; r < n; ++r) {
        key += std::to_string(deg[r]);
        key += ',';
    }
    return key;
}

// The rows of one sequence for A cooperating threads per row pair, as `macro`(D, P, s0, e0)
// entries; a block of up to four rows repeated back to back (same degrees, same slot
// parities) becomes a loop over its repetitions.
std::string ll_rows(const std::vector<int> &deg, int A, const char *macro) {
    const int n = (int)deg.size();
    std::vector<int> e0(n + 1, 0), s0(n + 1, 0);
    for (int r = 0; r < n; ++r) {
        e0[r + 1] = e0[r] + deg[r];
        s0[r + 1] = s0[r] + (deg[r] + A - 1) / A;
    }
    auto same = [&](int a, int b, int L) {
        for (int t = 0; t < L; ++t)
            if (a + t >= n || b + t >= n || deg[a + t] != deg[b + t] ||
                ((s0[a + t] ^ s0[b + t]) & 1))
                return false;
        return true;
    };
    auto row = [&](int r, const std::string &ds, const std::string &de) {
        return std::string(" ") + macro + "(" + std::to_string(deg[r]) + ", " +
               std::to_string(s0[r] & 1) + ", (" + std::to_string(s0[r]) + ds + "), (" +
               std::to_string(e0[r]) + de + "))";
    };
    std::string s;
    int r = 0;
    while (r < n) {
        int bestL = 0, bestK = 0, bestSave = 0;
        for (int L = 1; L <= 4 && r + 2 * L <= n; ++L) {
            int k = 1;
            while (r + (k + 1) * L <= n && same(r, r + k * L, L)) ++k;
            const int save = (k - 1) * (e0[r + L] - e0[r]);
            if (k >= 2 && save > bestSave) {
                bestL = L;
                bestK = k;
                bestSave = save;
            }
        }
        if (bestK >= 2) {
            const std::string ds = " + u_ * " + std::to_string(s0[r + bestL] - s0[r]);
            const std::string de = " + u_ * " + std::to_string(e0[r + bestL] - e0[r]);
            s += " _Pragma(\"unroll 1\") for (int u_ = 0; u_ < " + std::to_string(bestK) +
                 "; ++u_) {";
            for (int t = 0; t < bestL; ++t) s += row(r + t, ds, de);
            s += " }";
            r += bestL * bestK;
        } else {
            s += row(r, "", "");
            ++r;
        }
    }
    return s;
}

// One `case` of the list kernel: the rows of one sequence (A = 2).
std::string case_source(int c, const std::vector<int> &deg) {
    return " case " + std::to_string(c) + ":" + ll_rows(deg, kA, "LDPC_LLQ") + " break;";
}

std::vector<char> compile_list(const std::vector<std::vector<int>> &seqs) {
    std::string src(jit_prelude());
    src += "#define LDPC_LL_SEQS";
    for (size_t c = 0; c < seqs.size(); ++c) src += case_source((int)c, seqs[c]);
    src += "\n#include \"ll_kernel.cuh\"\n";
    return jit_compile(src, "ldpc_list_rows.cu");
}

}  // namespace

const ListModule *list_jit_active() {
    ListRegistry &R = registry();
    std::lock_guard<std::mutex> lk(R.mu);
    if (R.clear) {
        R.clear = false;
        R.active = nullptr;
    }
    if (!R.pending.empty()) {
        auto *m = new ListModule;             // kept for the process's lifetime
        bool ok = cudaLibraryLoadData(&m->lib, R.pending.data(), nullptr, nullptr, 0, nullptr,
                                      nullptr, 0) == cudaSuccess;
        if (ok && cudaLibraryGetKernel(&m->kernel, m->lib, "list_ll_kernel") != cudaSuccess) {
            cudaLibraryUnload(m->lib);
            ok = false;
        }
        if (ok) {
            m->index = std::move(R.pending_index);
            m->generation = ++R.generations;
            R.active = m;
        } else {
            cudaGetLastError();
            delete m;
        }
        R.pending.clear();
        R.pending.shrink_to_fit();
        R.pending_index.clear();
    }
    return R.active;
}

const void *list_jit_kernel(const ListModule *m) {
    return m ? reinterpret_cast<const void *>(m->kernel) : nullptr;
}

int list_jit_seq(const ListModule *m, Graph *g, int n_rows) {
    if (!m) return -1;
    std::atomic<uint64_t> &slot = g->list_seq[n_rows];
    const uint64_t v = slot.load(std::memory_order_relaxed);
    if ((uint32_t)(v >> 32) == m->generation) return (int)(uint32_t)v - 1;
    std::vector<int> deg((size_t)n_rows);
    for (int r = 0; r < n_rows; ++r) deg[(size_t)r] = g->row_ptr[r + 1] - g->row_ptr[r];
    const auto it = m->index.find(key_of(deg.data(), n_rows));
    const int seq = it == m->index.end() ? -1 : it->second;
    slot.store(((uint64_t)m->generation << 32) | (uint32_t)(seq + 1), std::memory_order_relaxed);
    return seq;
}

}  // namespace ldpc

extern "C" ldpc_status ldpc_list_jit_prepare(const int *row_degrees, const int *n_rows,
                                             int n_seqs) {
    ldpc::ListRegistry &R = ldpc::registry();
    if (n_seqs == 0) {
        std::lock_guard<std::mutex> lk(R.mu);
        R.pending.clear();
        R.pending_index.clear();
        R.clear = true;
        return LDPC_OK;
    }
    if (!row_degrees || !n_rows || n_seqs < 0 || n_seqs > 64) return LDPC_ERR_INVALID_ARG;
    std::vector<std::vector<int>> seqs;
    std::map<std::string, int> index;
    int off = 0;
    for (int q = 0; q < n_seqs; ++q) {
        const int n = n_rows[q];
        if (n < 1 || n > ldpc::kMaxRows) return LDPC_ERR_INVALID_ARG;
        std::vector<int> deg(row_degrees + off, row_degrees + off + n);
        off += n;
        int E = 0;
        for (const int d : deg) {
            if (d < 2 || d > ldpc::h2::kMaxDeg) return LDPC_ERR_INVALID_ARG;
            E += d;
        }
        if (E > ldpc::kMaxEdges) return LDPC_ERR_INVALID_ARG;
        const std::string key = ldpc::key_of(deg.data(), n);
        if (index.count(key)) continue;          // a repeated sequence needs one case
        index[key] = (int)seqs.size();
        seqs.push_back(std::move(deg));
    }
    std::vector<char> cubin;
    {
        std::lock_guard<std::mutex> ck(R.compile_mu);
        cubin = ldpc::compile_list(seqs);
    }
    if (cubin.empty()) return LDPC_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(R.mu);
    R.pending = std::move(cubin);
    R.pending_index = std::move(index);
    R.clear = false;
    return LDPC_OK;
}

namespace ldpc {

namespace {

std::string ll_key(const std::vector<int> &deg, int A) {
    std::string key = "ll:" + std::to_string(A) + ":";
    for (const int d : deg) {
        key += std::to_string(d);
        key += ',';
    }
    return key;
}

std::string ll_source(const std::vector<int> &deg, int A) {
    return std::string(jit_prelude()) + "#define LDPC_LL_A " + std::to_string(A) +
           "\n#define LDPC_LL_ROWS" + ll_rows(deg, A, "LDPC_LLR") +
           "\n#include \"ll_kernel.cuh\"\n";
}

}  // namespace

// The one-codeword low-latency kernel compiled for the row sequence of p and A cooperating
// threads per row pair (registry of jit_common.cu; ldpc_pair_jit's mode applies), or null.
const void *ll_jit_kernel(const DecodeParams &p, int A) {
    if (jit_mode() == 0) return nullptr;
    std::vector<int> deg((size_t)p.n_rows);
    for (int r = 0; r < p.n_rows; ++r) deg[(size_t)r] = p.h_row_ptr[r + 1] - p.h_row_ptr[r];
    return jit_kernel(ll_key(deg, A), [&deg, A] { return ll_source(deg, A); },
                      "ldpc_ll_rows.cu", "tmem_ll_kernel");
}

bool ll_jit_prepare(const std::vector<int> &deg, int A) {
    return jit_prepare(ll_key(deg, A), [&deg, A] { return ll_source(deg, A); },
                       "ldpc_ll_rows.cu");
}

}  // namespace ldpc
