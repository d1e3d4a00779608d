// NVRTC front end shared by the runtime-compiled kernels of pair_jit.cu, list_jit.cu and
// t16_jit.cu: one source (the fixed-width type prelude, the caller's macros, the kernel
// header) to a cubin for sm_103a, with the kernel headers embedded at build time
// (ldpc_jit_sources.h); and the registry of compiled kernels, which loads their modules on
// the launching thread.
#include <string>
#include <vector>

#include <nvrtc.h>

#include "ldpc_internal.h"
#include "ldpc_jit_sources.h"

namespace ldpc {

const char *jit_prelude() {
    return "typedef signed char int8_t;\n"
           "typedef unsigned char uint8_t;\n"
           "typedef short int16_t;\n"
           "typedef unsigned short uint16_t;\n"
           "typedef int int32_t;\n"
           "typedef unsigned int uint32_t;\n"
           "typedef long long int64_t;\n"
           "typedef unsigned long long uint64_t;\n"
           "typedef unsigned long size_t;\n"
           "typedef unsigned long uintptr_t;\n";
}

std::vector<char> jit_compile(const std::string &src, const char *name) {
    std::vector<const char *> names, texts;
    for (const auto &f : jitsrc::kFiles) {
        names.push_back(f.name);
        texts.push_back(f.text);
    }
    std::vector<char> cubin;
    nvrtcProgram prog;
    if (nvrtcCreateProgram(&prog, src.c_str(), name, (int)names.size(), texts.data(),
                           names.data()) != NVRTC_SUCCESS)
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

}  // namespace ldpc

// ------------------------------------------------------------------ kernel registry
//
// Kernels compiled at run time, one per key (the caller's description of what the module
// is specialised on), kept for the process's lifetime.  A missing key is compiled on a
// background thread (host work only: the thread makes no CUDA call) or, with wait, by the
// caller; the first launch after the compilation loads the module on the launching thread.

#include <atomic>
#include <condition_variable>
#include <map>
#include <mutex>
#include <thread>

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
    std::map<std::string, JitEntry> entries;
};
JitRegistry &registry() {
    static JitRegistry *r = new JitRegistry;
    return *r;
}

// Background compilations in flight.  A process must not exit while one runs: the runtime
// compiler's own exit-time cleanup can run first and tear its state down under the thread.
// ldpc_pair_jit(3) waits for them (the Python binding calls it from an interpreter exit
// hook, which runs before any C exit handler); the destructor waits as well, for the exit
// orders where it runs first.
struct JitThreads {
    std::mutex mu;
    std::condition_variable cv;
    int running = 0;
    ~JitThreads() {
        std::unique_lock<std::mutex> lk(mu);
        cv.wait(lk, [this] { return running == 0; });
    }
};
JitThreads &threads() {
    static JitThreads t;
    return t;
}

std::atomic<int> g_mode{1};          // 0 off, 1 background compile, 2 blocking compile
std::atomic<int> g_built{0}, g_failed{0};

// kCompiled -> kLoaded or kFailed, on the launching thread (lock held).
void load_module(JitEntry &e, const char *kernel) {
    bool ok = cudaLibraryLoadData(&e.lib, e.cubin.data(), nullptr, nullptr, 0, nullptr,
                                  nullptr, 0) == cudaSuccess;
    if (ok && cudaLibraryGetKernel(&e.kernel, e.lib, kernel) != cudaSuccess) {
        cudaLibraryUnload(e.lib);
        ok = false;
    }
    if (!ok) cudaGetLastError();
    e.cubin.clear();
    e.cubin.shrink_to_fit();
    e.state = ok ? kLoaded : kFailed;
    (ok ? g_built : g_failed).fetch_add(1);
}

// the compile result into the registry (lock taken here)
void finish_compile(const std::string &key, std::vector<char> cubin) {
    JitRegistry &R = registry();
    std::lock_guard<std::mutex> lk(R.mu);
    JitEntry &e = R.entries[key];
    if (cubin.empty()) {
        e.state = kFailed;
        g_failed.fetch_add(1);
    } else {
        e.cubin = std::move(cubin);
        e.state = kCompiled;
    }
    R.cv.notify_all();
}

// The entry of key, created (and its compilation started: on a background thread unless
// wait) when absent; with wait, returns once it is compiled or has failed.  Lock held on
// entry and exit.
JitEntry *entry_for(std::unique_lock<std::mutex> &lk, const std::string &key,
                    const std::function<std::string()> &source, const char *name, bool wait) {
    JitRegistry &R = registry();
    auto it = R.entries.find(key);
    if (it == R.entries.end()) {
        R.entries[key].state = kCompiling;
        if (wait) {
            lk.unlock();
            finish_compile(key, jit_compile(source(), name));
            lk.lock();
        } else {
            JitThreads &T = threads();
            {
                std::lock_guard<std::mutex> tl(T.mu);
                ++T.running;
            }
            try {
                std::string src = source();
                std::string nm(name);
                std::thread([key, src, nm, &T] {
                    finish_compile(key, jit_compile(src, nm.c_str()));
                    std::lock_guard<std::mutex> tl(T.mu);
                    --T.running;
                    T.cv.notify_all();
                }).detach();
            } catch (...) {                  // no thread: this key keeps the generic kernel
                R.entries[key].state = kFailed;
                g_failed.fetch_add(1);
                std::lock_guard<std::mutex> tl(T.mu);
                --T.running;
            }
        }
        it = R.entries.find(key);
    }
    JitEntry *e = &it->second;
    if (wait) R.cv.wait(lk, [e] { return e->state != kCompiling; });
    return e;
}

}  // namespace

int jit_mode() { return g_mode.load(std::memory_order_relaxed); }

int jit_set_mode(int mode) {
    const int prev = g_mode.load();
    if (mode >= 0 && mode <= 2) g_mode.store(mode);
    if (mode == 3) {                         // wait for the background compilations
        JitThreads &T = threads();
        std::unique_lock<std::mutex> lk(T.mu);
        T.cv.wait(lk, [&T] { return T.running == 0; });
    }
    return prev | (g_built.load() > 0 ? 4 : 0) | (g_failed.load() > 0 ? 8 : 0);
}

const void *jit_kernel(const std::string &key, const std::function<std::string()> &source,
                       const char *name, const char *kernel) {
    const int mode = jit_mode();
    if (mode == 0) return nullptr;
    std::unique_lock<std::mutex> lk(registry().mu);
    JitEntry *e = entry_for(lk, key, source, name, mode == 2);
    if (e->state == kCompiled) load_module(*e, kernel);
    return e->state == kLoaded ? reinterpret_cast<const void *>(e->kernel) : nullptr;
}

bool jit_prepare(const std::string &key, const std::function<std::string()> &source,
                 const char *name) {
    std::unique_lock<std::mutex> lk(registry().mu);
    return entry_for(lk, key, source, name, true)->state != kFailed;
}

}  // namespace ldpc
