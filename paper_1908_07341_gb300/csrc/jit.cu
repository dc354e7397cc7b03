// jit.cu -- half-step sweeps compiled at run time for one threshold table.
//
// The draw compares each random plane with the threshold bit of the site's
// class (device.cuh, apply_planes).  With the three thresholds known when
// the kernel is compiled, every plane's class mask becomes a constant and
// folds into the logic: the sweep then needs fewer instructions and
// registers than the generic kernel, which reads the masks from its
// parameters.  This file compiles the sweep kernels' own source text (the
// headers are embedded at build time) with NVRTC for sm_103a, once per
// (launch shape, threshold table, device), and launches the result through
// the runtime's library API.  After the first compile of the process (which
// runs on the calling thread), compiles run on a background thread, so a
// launch does not wait for them (unless the blocking mode asks to): until the
// specialised kernel is ready, and whenever NVRTC cannot be loaded or the
// compile fails, the caller launches the generic kernel, which computes the
// same spins and sums.
#include <dlfcn.h>
#include <pthread.h>
#include <nvrtc.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "shaken.h"
#include "internal.h"
#include "sweep.cuh"
#include "jit_sources.inc"   // generated by build.py: kJitSourceCount, kJitSourceNames, kJitSourceTexts

namespace shk {

std::atomic<int> g_jit_mode{1};

namespace {

// NVRTC entry points, loaded with dlopen so that the library does not
// depend on NVRTC at link time.
struct Nvrtc {
    decltype(&nvrtcCreateProgram) create = nullptr;
    decltype(&nvrtcAddNameExpression) add_name = nullptr;
    decltype(&nvrtcCompileProgram) compile = nullptr;
    decltype(&nvrtcGetProgramLogSize) log_size = nullptr;
    decltype(&nvrtcGetProgramLog) log = nullptr;
    decltype(&nvrtcGetLoweredName) lowered = nullptr;
    decltype(&nvrtcGetCUBINSize) cubin_size = nullptr;
    decltype(&nvrtcGetCUBIN) cubin = nullptr;
    decltype(&nvrtcDestroyProgram) destroy = nullptr;
    bool ok = false;
};

const Nvrtc& nvrtc() {
    static Nvrtc n;
    static std::once_flag once;
    std::call_once(once, [] {
        void* h = nullptr;
        std::string home;
        if (const char* c = std::getenv("CUDA_HOME")) home = std::string(c) + "/lib64/libnvrtc.so.13";
        for (const char* name : {"libnvrtc.so.13", "libnvrtc.so", home.c_str(), "/usr/local/cuda/lib64/libnvrtc.so.13"}) {
            if (*name) h = dlopen(name, RTLD_NOW | RTLD_LOCAL);
            if (h) break;
        }
        if (!h) return;
        n.create = reinterpret_cast<decltype(n.create)>(dlsym(h, "nvrtcCreateProgram"));
        n.add_name = reinterpret_cast<decltype(n.add_name)>(dlsym(h, "nvrtcAddNameExpression"));
        n.compile = reinterpret_cast<decltype(n.compile)>(dlsym(h, "nvrtcCompileProgram"));
        n.log_size = reinterpret_cast<decltype(n.log_size)>(dlsym(h, "nvrtcGetProgramLogSize"));
        n.log = reinterpret_cast<decltype(n.log)>(dlsym(h, "nvrtcGetProgramLog"));
        n.lowered = reinterpret_cast<decltype(n.lowered)>(dlsym(h, "nvrtcGetLoweredName"));
        n.cubin_size = reinterpret_cast<decltype(n.cubin_size)>(dlsym(h, "nvrtcGetCUBINSize"));
        n.cubin = reinterpret_cast<decltype(n.cubin)>(dlsym(h, "nvrtcGetCUBIN"));
        n.destroy = reinterpret_cast<decltype(n.destroy)>(dlsym(h, "nvrtcDestroyProgram"));
        n.ok = n.create && n.add_name && n.compile && n.log_size && n.log && n.lowered && n.cubin_size &&
               n.cubin && n.destroy;
    });
    return n;
}

// One (kernel pair, threshold table) entry.  The compile (NVRTC, host only)
// runs on a background thread and leaves a cubin; each device loads it on a
// launching thread, at its first launch there.
struct JitEntry {
    enum State { kQueued, kCompiled, kFailed };
    State state = kQueued;
    std::string e[2];
    uint32_t U[3] = {0, 0, 0};
    int block = 0;
    std::vector<char> cubin;
    std::string lowered[2];
    struct Loaded {
        bool ok = false;
        cudaLibrary_t lib = nullptr;
        cudaKernel_t k[2] = {nullptr, nullptr};
        int per_sm[2] = {0, 0};
    };
    std::map<int, Loaded> dev;   // by device ordinal
};

using Key = std::tuple<std::string, uint32_t, uint32_t, uint32_t>;

std::mutex g_mu;                          // guards everything below
std::condition_variable g_cv;             // signalled when an entry leaves kQueued, or on stop
std::map<Key, JitEntry*> g_cache;         // entries live for the life of the process
std::deque<JitEntry*> g_queue;
std::thread* g_worker = nullptr;
bool g_stop = false;
std::string g_last_log;
double g_compile_s = 0.0;                 // host seconds spent compiling, all entries

constexpr size_t kMaxQueued = 2;          // launches queue no table beyond this (generic kernel meanwhile)
constexpr size_t kMaxEntries = 512;       // bound on compiled tables per process
constexpr std::chrono::seconds kWaitLimit(120);   // longest blocking wait for one compile

// NVRTC compile of the entry's two kernels with its thresholds as
// constants; fills cubin and the lowered names, or returns false with the
// compiler log.
bool compile_cubin(JitEntry* en, std::string* log_out) {
    const Nvrtc& n = nvrtc();
    if (!n.ok) {
        *log_out = "NVRTC could not be loaded";
        return false;
    }
    nvrtcProgram prog = nullptr;
    const char* src = "#include \"sweep_kernels.cuh\"\n#include \"checkerboard.cuh\"\n";
    if (n.create(&prog, src, "shk_jit.cu", kJitSourceCount, kJitSourceTexts, kJitSourceNames) != NVRTC_SUCCESS) {
        *log_out = "nvrtcCreateProgram failed";
        return false;
    }
    bool ok = n.add_name(prog, en->e[0].c_str()) == NVRTC_SUCCESS && n.add_name(prog, en->e[1].c_str()) == NVRTC_SUCCESS;
    char d0[48], d1[48], d2[48];
    std::snprintf(d0, sizeof d0, "-DSHK_JIT_U0=%uu", en->U[0]);
    std::snprintf(d1, sizeof d1, "-DSHK_JIT_U1=%uu", en->U[1]);
    std::snprintf(d2, sizeof d2, "-DSHK_JIT_U2=%uu", en->U[2]);
    const char* opts[] = {"--gpu-architecture=sm_103a", "-std=c++17", d0, d1, d2};
    if (ok && n.compile(prog, 5, opts) != NVRTC_SUCCESS) {
        size_t sz = 0;
        n.log_size(prog, &sz);
        std::string log(sz, '\0');
        if (sz) n.log(prog, &log[0]);
        *log_out = log.empty() ? std::string("nvrtcCompileProgram failed") : log;
        ok = false;
    }
    if (ok) {
        const char* low[2] = {nullptr, nullptr};
        size_t sz = 0;
        ok = n.lowered(prog, en->e[0].c_str(), &low[0]) == NVRTC_SUCCESS &&
             n.lowered(prog, en->e[1].c_str(), &low[1]) == NVRTC_SUCCESS && n.cubin_size(prog, &sz) == NVRTC_SUCCESS &&
             sz > 0;
        if (ok) {
            en->lowered[0] = low[0];
            en->lowered[1] = low[1];
            en->cubin.resize(sz);
            ok = n.cubin(prog, en->cubin.data()) == NVRTC_SUCCESS;
        }
        if (!ok) *log_out = "reading the compiled program failed";
    }
    n.destroy(&prog);
    return ok;
}

void worker_main() {
    std::unique_lock<std::mutex> lock(g_mu);
    for (;;) {
        g_cv.wait(lock, [] { return g_stop || !g_queue.empty(); });
        if (g_stop) return;
        JitEntry* en = g_queue.front();
        g_queue.pop_front();
        lock.unlock();
        std::string log;
        const auto t0 = std::chrono::steady_clock::now();
        const bool ok = compile_cubin(en, &log);
        const double dt = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        lock.lock();
        g_compile_s += dt;
        en->state = ok ? JitEntry::kCompiled : JitEntry::kFailed;
        if (!ok) g_last_log = log;
        g_cv.notify_all();
    }
}

// Lets a compile in flight finish and stops the worker; idempotent.  Runs at
// process exit (registered after NVRTC's own teardown, so before it), and
// from shk_specialize_shutdown.
void stop_worker() {
    std::thread* t = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_mu);
        g_stop = true;
        t = g_worker;
    }
    g_cv.notify_all();
    if (t && t->joinable()) t->join();
}

// fork(): the child has no worker thread.  The parent holds g_mu across the
// fork so that the child's copy is consistent; the child stops run-time
// compilation (its requests run generic, and blocking waits return).
void atfork_prepare() { g_mu.lock(); }
void atfork_parent() { g_mu.unlock(); }
void atfork_child() {
    g_stop = true;
    g_worker = nullptr;
    g_mu.unlock();
}

// The entry of (e0, U), queued for compile when new.  force: queue even past
// kMaxQueued.  Null when no entry can be made (stopping, too many entries,
// queue full, no NVRTC).  Called with g_mu held.
JitEntry* find_or_queue(const char* e0, const char* e1, int block, const uint32_t U[3], bool force) {
    const Key key = std::make_tuple(std::string(e0), U[0], U[1], U[2]);
    auto it = g_cache.find(key);
    if (it != g_cache.end()) return it->second;
    if (g_stop || g_cache.size() >= kMaxEntries || (!force && g_queue.size() >= kMaxQueued)) return nullptr;
    if (!nvrtc().ok) {
        g_last_log = "NVRTC could not be loaded";
        return nullptr;
    }
    JitEntry* en = new (std::nothrow) JitEntry;
    if (en == nullptr) return nullptr;
    en->e[0] = e0;
    en->e[1] = e1;
    std::copy(U, U + 3, en->U);
    en->block = block;
    g_cache.emplace(key, en);
    if (g_worker == nullptr) {
        // The first compile of the process runs here, on the calling thread.
        // NVRTC builds internal state on first use and registers its teardown
        // at exit then; registering stop_worker only afterwards makes it run
        // before that teardown, so an exit during a later background compile
        // waits for it instead of tearing NVRTC down under it (which crashed).
        std::string log;
        const auto t0 = std::chrono::steady_clock::now();
        const bool ok = compile_cubin(en, &log);
        g_compile_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        en->state = ok ? JitEntry::kCompiled : JitEntry::kFailed;
        if (!ok) g_last_log = log;
        std::atexit(stop_worker);
        pthread_atfork(atfork_prepare, atfork_parent, atfork_child);
        try {
            g_worker = new std::thread(worker_main);
        } catch (...) {
            g_stop = true;          // no background compiles: tables not yet compiled run generic
            g_last_log = "could not start the compile thread";
        }
        return en;
    }
    g_queue.push_back(en);
    g_cv.notify_all();
    return en;
}

// The kernels of a compiled entry on device dev, loaded now if needed (on
// the calling thread); null if loading failed.  Called with g_mu held.
const JitEntry::Loaded* loaded_on(JitEntry* en, int dev) {
    auto it = en->dev.find(dev);
    if (it != en->dev.end()) return it->second.ok ? &it->second : nullptr;
    JitEntry::Loaded& l = en->dev[dev];
    if (cudaLibraryLoadData(&l.lib, en->cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0) != cudaSuccess) {
        cudaGetLastError();
        g_last_log = "cudaLibraryLoadData failed";
        return nullptr;
    }
    for (int h = 0; h < 2; ++h) {
        if (cudaLibraryGetKernel(&l.k[h], l.lib, en->lowered[h].c_str()) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&l.per_sm[h], reinterpret_cast<const void*>(l.k[h]),
                                                          en->block, 0) != cudaSuccess) {
            cudaGetLastError();
            g_last_log = "loading a compiled kernel failed";
            return nullptr;
        }
        if (l.per_sm[h] <= 0) l.per_sm[h] = 1;
    }
    l.ok = true;
    return &l;
}

}  // namespace

// The three class thresholds U[n'] = T[3 + n'] recovered from the plane masks
// of the draw parameters (bit 31-b of U0 is m0[b], U1 and U2 follow from the
// differences).
static void thresholds_of(const DrawParams& P, uint32_t U[3]) {
    U[0] = U[1] = U[2] = 0;
    for (int b = 0; b < 32; ++b) {
        const uint32_t m0 = P.m0[b] & 1u, m1 = m0 ^ (P.d01[b] & 1u), m2 = m1 ^ (P.d12[b] & 1u);
        U[0] |= m0 << (31 - b);
        U[1] |= m1 << (31 - b);
        U[2] |= m2 << (31 - b);
    }
}

// Launches half `half` of a sweep compiled for a's threshold table; returns
// false (nothing launched) when no run-time compiled kernel is ready, so that
// the caller launches the generic one.  The first request for a table queues
// its compile; in blocking mode it also waits for it.
bool jit_launch(const char* e0, const char* e1, int block, int half, uint32_t work_items, const SweepArgs& a,
                cudaStream_t st, cudaError_t* err, bool loaded_only, int waves) {
#ifdef SHK_DEBUG_BOUNDS
    (void)e0, (void)e1, (void)block, (void)half, (void)work_items, (void)a, (void)st, (void)err, (void)loaded_only,
        (void)waves;
    return false;   // the bounds-checked build checks the generic kernels
#else
    const int mode = g_jit_mode.load();
    if (mode == 0 || e0 == nullptr || e1 == nullptr) return false;
    uint32_t U[3];
    thresholds_of(a.P, U);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    const JitEntry::Loaded* l = nullptr;
    if (loaded_only) {
        // only a kernel that an earlier launch on this device has loaded:
        // no compile is queued, run or waited for, and no module is loaded
        std::lock_guard<std::mutex> lock(g_mu);
        auto it = g_cache.find(std::make_tuple(std::string(e0), U[0], U[1], U[2]));
        if (it == g_cache.end() || it->second->state != JitEntry::kCompiled) return false;
        auto d = it->second->dev.find(dev);
        if (d == it->second->dev.end() || !d->second.ok) return false;
        l = &d->second;
    } else {
        std::unique_lock<std::mutex> lock(g_mu);
        JitEntry* en = find_or_queue(e0, e1, block, U, mode == 2);
        if (en == nullptr) return false;
        // blocking mode waits for the compile, at most kWaitLimit (the generic kernel runs after that)
        if (mode == 2) g_cv.wait_for(lock, kWaitLimit, [en] { return en->state != JitEntry::kQueued || g_stop; });
        if (en->state != JitEntry::kCompiled) return false;
        if (en->dev.find(dev) == en->dev.end()) {
            // loading a module is not allowed while the stream is being
            // captured into a graph: launch generic until a later call loads it
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
                cudaGetLastError();
                return false;
            }
            if (cs != cudaStreamCaptureStatusNone) return false;
        }
        l = loaded_on(en, dev);
        if (l == nullptr) return false;
    }
    const uint64_t full = (uint64_t)l->per_sm[half] * sm_count() * (uint64_t)(waves > 0 ? waves : 1);
    const uint64_t need = ((uint64_t)work_items + block - 1) / block;
    const int grid = (int)std::max<uint64_t>(1, std::min(full, need));
    void* args[] = {const_cast<SweepArgs*>(&a)};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;   // as launch_pdl
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    *err = cudaLaunchKernelExC(&cfg, reinterpret_cast<const void*>(l->k[half]), args);
    return true;
#endif
}

// Queues (wait: and waits for) the compile of the specialised form of a
// sweep variant for one threshold table, without launching anything.
int jit_prepare(int layout, int variant, const uint32_t T[6], bool wait, std::string* why) {
#ifdef SHK_DEBUG_BOUNDS
    (void)layout, (void)variant, (void)T, (void)wait;
    *why = "the bounds-checked build never specialises";
    return SHK_ESTATE;
#else
    const char* e0 = nullptr;
    const char* e1 = nullptr;
    int block = 0;
    if (!sweep_variant_jit(layout, variant, &e0, &e1, &block)) {
        *why = "no such variant";
        return SHK_EINVAL;
    }
    if (e0 == nullptr) {
        *why = "this variant has no specialised form";
        return SHK_EINVAL;
    }
    if (g_jit_mode.load() == 0) {
        *why = "specialisation is off";
        return SHK_ESTATE;
    }
    const uint32_t U[3] = {T[3], T[4], T[5]};
    std::unique_lock<std::mutex> lock(g_mu);
    JitEntry* en = find_or_queue(e0, e1, block, U, true);
    if (en == nullptr) {
        *why = g_last_log.empty() ? std::string("no more entries can be compiled") : g_last_log;
        return SHK_ESTATE;
    }
    if (!wait) return SHK_OK;
    if (!g_cv.wait_for(lock, kWaitLimit, [en] { return en->state != JitEntry::kQueued || g_stop; })) {
        *why = "the compile did not finish within the wait limit";
        return SHK_ETIMEOUT;
    }
    if (en->state != JitEntry::kCompiled) {
        *why = g_last_log.empty() ? std::string("the compile did not finish") : g_last_log;
        return SHK_ESTATE;
    }
    return SHK_OK;
#endif
}

}  // namespace shk

extern "C" {

int shk_set_specialize(int mode) {
    if (mode < 0 || mode > 2) return SHK_EINVAL;
    shk::g_jit_mode.store(mode);
    return SHK_OK;
}

int shk_get_specialize(void) { return shk::g_jit_mode.load(); }

int shk_specialize_status(int* compiled, int* failed, int* queued, double* compile_seconds, char* log,
                          size_t log_bytes) {
    std::lock_guard<std::mutex> lock(shk::g_mu);
    int c = 0, f = 0, qd = 0;
    for (const auto& kv : shk::g_cache) {
        const shk::JitEntry* en = kv.second;
        bool load_failed = false;
        for (const auto& d : en->dev) load_failed |= !d.second.ok;
        if (en->state == shk::JitEntry::kFailed || load_failed) ++f;
        else if (en->state == shk::JitEntry::kQueued) ++qd;
        else ++c;
    }
    if (compiled) *compiled = c;
    if (failed) *failed = f;
    if (queued) *queued = qd;
    if (compile_seconds) *compile_seconds = shk::g_compile_s;
    if (log && log_bytes > 0) {
        const size_t n = std::min(log_bytes - 1, shk::g_last_log.size());
        std::memcpy(log, shk::g_last_log.data(), n);
        log[n] = '\0';
    }
    return SHK_OK;
}

int shk_specialize_shutdown(void) {
    shk::stop_worker();
    return SHK_OK;
}

int shk_specialize_prepare(int layout, int variant, double q, double J, int wait) {
    uint32_t T[6];
    if (shk::host_thresholds(q, J, T) != SHK_OK) {
        shk::set_thread_error("shk_specialize_prepare: q and J must be finite");
        return SHK_EINVAL;
    }
    std::string why;
    const int rc = shk::jit_prepare(layout, variant, T, wait != 0, &why);
    if (rc != SHK_OK) shk::set_thread_error(("shk_specialize_prepare: " + why).c_str());
    return rc;
}

}  // extern "C"
