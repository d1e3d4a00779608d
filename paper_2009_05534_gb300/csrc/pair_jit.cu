// Per-graph batch kernels compiled at run time.  The batch kernel (pair_kernel.cuh) walks
// the layers of an iteration with one indirect branch per row on the row's degree and the
// parity of its first edge; compiled with the graph's row sequence written out
// (LDPC_PAIR_ROWS), the same kernel runs the layers as straight-line code (measured 19 %
// less time per headline launch, bit-identical results).  The row sequence depends only on
// the degrees of the rows a decode uses, so one module serves every graph and lifting size
// with that degree sequence: the shifts and columns stay in the kernel's parameter table.
//
// Modules are built with NVRTC from the kernel headers embedded at build time
// (ldpc_jit_sources.h, written by build.py), loaded with cudaLibraryLoadData (valid in
// every context of the process) and kept for the process's lifetime.  Compiling takes a
// few seconds of host time, so by default it runs on a background thread (host code only:
// the thread makes no CUDA call) and the generic kernel serves the degree sequence until
// the module is ready; the first launch after that loads it.  In the blocking mode the
// launch that meets a new sequence compiles and loads it itself.  A compile or load that
// fails marks its sequence, and the generic kernel runs instead.
#include <atomic>
#include <condition_variable>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include <nvrtc.h>

#include "f16x2.h"
#include "ldpc_internal.h"
#include "ldpc_jit_sources.h"

namespace ldpc {
namespace {

enum JitState { kCompiling, kCompiled, kLoaded, kFailed };

struct JitEntry {
    JitState state = kCompiling;
    std::vector<char> cubin;          // kCompiled: the module image, not loaded yet
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kernel = nullptr;    // kLoaded
};

// Never destroyed: a background compile may still run while the process exits.
struct JitRegistry {
    std::mutex mu;
    std::condition_variable cv;
    std::map<std::string, JitEntry> entries;   // key: the degrees of the used rows
};
JitRegistry &registry() {
    static JitRegistry *r = new JitRegistry;
    return *r;
}

std::atomic<int> g_jit_mode{1};      // 0 off, 1 background compile, 2 blocking compile
std::atomic<int> g_jit_built{0}, g_jit_failed{0};

// fixed-width types for the runtime compiler, which has no libc headers
const char kPrelude[] =
    "typedef signed char int8_t;\n"
    "typedef unsigned char uint8_t;\n"
    "typedef short int16_t;\n"
    "typedef unsigned short uint16_t;\n"
    "typedef int int32_t;\n"
    "typedef unsigned int uint32_t;\n"
    "typedef long long int64_t;\n"
    "typedef unsigned long long uint64_t;\n"
    "typedef unsigned long size_t;\n"
    "typedef unsigned long uintptr_t;\n";

// The source of one module: the prelude, the row sequence and the kernel header.  A block
// of up to 4 rows repeated back to back (same degrees, same first-edge parities) becomes a
// loop over its repetitions, the block that saves the most edges of code first: the
// straight-line layer loop is about 22 instructions per edge, its instruction fetch grows
// with its length, and the loops shorten it by a quarter on the BG1-shaped table (3 % less
// time per headline launch, measured).
std::string module_source(const std::vector<int> &deg) {
    std::string s(kPrelude);
    s += "#define LDPC_PAIR_ROWS";
    const int n = (int)deg.size();
    std::vector<int> e0s(n + 1, 0);
    for (int r = 0; r < n; ++r) e0s[r + 1] = e0s[r] + deg[r];
    auto same = [&](int a, int b, int L) {
        for (int t = 0; t < L; ++t)
            if (a + t >= n || b + t >= n || deg[a + t] != deg[b + t] ||
                ((e0s[a + t] ^ e0s[b + t]) & 1))
                return false;
        return true;
    };
    int r = 0;
    while (r < n) {
        int bestL = 0, bestK = 0, bestSave = 0;
        for (int L = 1; L <= 4 && r + 2 * L <= n; ++L) {
            int k = 1;
            while (r + (k + 1) * L <= n && same(r, r + k * L, L)) ++k;
            const int save = (k - 1) * (e0s[r + L] - e0s[r]);
            if (k >= 2 && save > bestSave) {
                bestL = L;
                bestK = k;
                bestSave = save;
            }
        }
        if (bestK >= 2) {
            const int S = e0s[r + bestL] - e0s[r];
            s += " _Pragma(\"unroll 1\") for (int u_ = 0; u_ < " + std::to_string(bestK) +
                 "; ++u_) {";
            for (int t = 0; t < bestL; ++t)
                s += " LDPC_PQ(" + std::to_string(deg[r + t]) + ", " +
                     std::to_string(e0s[r + t] & 1) + ", (" + std::to_string(e0s[r + t]) +
                     " + u_ * " + std::to_string(S) + "))";
            s += " }";
            r += bestL * bestK;
        } else {
            s += " LDPC_PQ(" + std::to_string(deg[r]) + ", " + std::to_string(e0s[r] & 1) +
                 ", " + std::to_string(e0s[r]) + ")";
            ++r;
        }
    }
    s += "\n#include \"pair_kernel.cuh\"\n";
    return s;
}

// NVRTC: source to cubin (host only).  Empty on failure.
std::vector<char> compile_module(const std::vector<int> &deg) {
    const std::string src = module_source(deg);
    std::vector<const char *> names, texts;
    for (const auto &f : jitsrc::kFiles) {
        names.push_back(f.name);
        texts.push_back(f.text);
    }
    std::vector<char> cubin;
    nvrtcProgram prog;
    if (nvrtcCreateProgram(&prog, src.c_str(), "ldpc_pair_rows.cu", (int)names.size(),
                           texts.data(), names.data()) != NVRTC_SUCCESS)
        return cubin;
    const char *opts[] = {"--gpu-architecture=sm_103a", "-std=c++17"};
    if (nvrtcCompileProgram(prog, 2, opts) == NVRTC_SUCCESS) {
        size_t n = 0;
        if (nvrtcGetCUBINSize(prog, &n) == NVRTC_SUCCESS && n > 0) {
            cubin.resize(n);
            if (nvrtcGetCUBIN(prog, cubin.data()) != NVRTC_SUCCESS) cubin.clear();
        }
    }
    nvrtcDestroyProgram(&prog);
    return cubin;
}

// kCompiled -> kLoaded or kFailed, on the launching thread (lock held).
void load_module(JitEntry &e) {
    bool ok = cudaLibraryLoadData(&e.lib, e.cubin.data(), nullptr, nullptr, 0, nullptr,
                                  nullptr, 0) == cudaSuccess;
    if (ok && cudaLibraryGetKernel(&e.kernel, e.lib, "pair_kernel") != cudaSuccess) {
        cudaLibraryUnload(e.lib);
        ok = false;
    }
    if (!ok) cudaGetLastError();
    e.cubin.clear();
    e.cubin.shrink_to_fit();
    e.state = ok ? kLoaded : kFailed;
    (ok ? g_jit_built : g_jit_failed).fetch_add(1);
}

// the compile result into the registry (lock taken here)
void finish_compile(const std::string &key, std::vector<char> cubin) {
    JitRegistry &R = registry();
    std::lock_guard<std::mutex> lk(R.mu);
    JitEntry &e = R.entries[key];
    if (cubin.empty()) {
        e.state = kFailed;
        g_jit_failed.fetch_add(1);
    } else {
        e.cubin = std::move(cubin);
        e.state = kCompiled;
    }
    R.cv.notify_all();
}

}  // namespace

namespace {

std::string degree_key(const std::vector<int> &deg) {
    std::string key;
    for (const int d : deg) {
        key += std::to_string(d);
        key += ',';
    }
    return key;
}

// The registry entry of a degree sequence, created (and its compile started: on a
// background thread unless wait) when absent; with wait, returns once it is compiled or
// has failed.  Lock held on entry and exit.
JitEntry *entry_for(std::unique_lock<std::mutex> &lk, const std::vector<int> &deg, bool wait) {
    JitRegistry &R = registry();
    const std::string key = degree_key(deg);
    auto it = R.entries.find(key);
    if (it == R.entries.end()) {
        R.entries[key].state = kCompiling;
        if (wait) {
            lk.unlock();
            finish_compile(key, compile_module(deg));
            lk.lock();
        } else {
            try {
                std::thread([key, deg] { finish_compile(key, compile_module(deg)); }).detach();
            } catch (...) {                  // no thread: this sequence keeps the generic kernel
                R.entries[key].state = kFailed;
                g_jit_failed.fetch_add(1);
            }
        }
        it = R.entries.find(key);
    }
    JitEntry *e = &it->second;
    if (wait) R.cv.wait(lk, [e] { return e->state != kCompiling; });
    return e;
}

}  // namespace

const void *pair_jit_kernel(const DecodeParams &p) {
    const int mode = g_jit_mode.load(std::memory_order_relaxed);
    if (mode == 0) return nullptr;
    std::vector<int> deg((size_t)p.n_rows);
    for (int r = 0; r < p.n_rows; ++r) deg[(size_t)r] = p.h_row_ptr[r + 1] - p.h_row_ptr[r];
    std::unique_lock<std::mutex> lk(registry().mu);
    JitEntry *e = entry_for(lk, deg, mode == 2);
    if (e->state == kCompiled) load_module(*e);
    return e->state == kLoaded ? reinterpret_cast<const void *>(e->kernel) : nullptr;
}

}  // namespace ldpc

extern "C" int ldpc_pair_jit(int mode) {
    const int prev = ldpc::g_jit_mode.load();
    if (mode >= 0 && mode <= 2) ldpc::g_jit_mode.store(mode);
    return prev | (ldpc::g_jit_built.load() > 0 ? 4 : 0) |
           (ldpc::g_jit_failed.load() > 0 ? 8 : 0);
}

extern "C" ldpc_status ldpc_pair_jit_prepare(const int *row_degrees, int n_rows) {
    if (!row_degrees || n_rows < 1 || n_rows > ldpc::kMaxRows) return LDPC_ERR_INVALID_ARG;
    std::vector<int> deg((size_t)n_rows);
    int E = 0;
    for (int r = 0; r < n_rows; ++r) {
        deg[(size_t)r] = row_degrees[r];
        if (row_degrees[r] < 2 || row_degrees[r] > ldpc::h2::kMaxDeg) return LDPC_ERR_INVALID_ARG;
        E += row_degrees[r];
    }
    if (E > ldpc::kMaxEdges) return LDPC_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(ldpc::registry().mu);
    const ldpc::JitEntry *e = ldpc::entry_for(lk, deg, true);
    return e->state == ldpc::kFailed ? LDPC_ERR_UNSUPPORTED : LDPC_OK;
}
