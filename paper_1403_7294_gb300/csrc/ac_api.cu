// ac_api.cu - the C-ABI entry points of libac.so (see include/ac.h).
//
// Memory: the dfa's tables live in plain device allocations owned by the
// ac_dfa. Per-call scratch (the per-state hit counters, the occurrence
// counter, staging for host texts/results, the packed copy of an ASCII text)
// comes from the device's stream-ordered pool (cudaMallocAsync on the
// caller's stream, released with cudaFreeAsync), so concurrent scans of one
// dfa never share scratch.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <unordered_map>
#include <vector>

#include "ac_internal.h"
#include "ac_trace.h"

namespace {

int cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return AC_OK;
    if (e == cudaErrorMemoryAllocation) return AC_ERR_OOM;
    return AC_ERR_CUDA;
}

// ---- host-side fault injection (ac_fault_inject, or AC_FAULT at the first
// allocation): "oom@k" makes the k-th device allocation after the plan was
// set fail as if the device were full; "cuda_err@k" makes the k-th kernel
// launch report a launch failure without launching anything. Both are
// counted from the moment the plan is set; nothing reaches the GPU.
std::mutex g_fault_mu;
bool g_fault_env_read = false;
long g_alloc_count = 0, g_launch_count = 0;
long g_fault_oom_at = -1, g_fault_launch_at = -1;

bool parse_fault_plan(const char* spec, long* oom_at, long* launch_at) {
    *oom_at = *launch_at = -1;
    if (!spec || !*spec) return true;
    const char* p = spec;
    while (*p) {
        long* slot = nullptr;
        if (std::strncmp(p, "oom@", 4) == 0) {
            slot = oom_at;
            p += 4;
        } else if (std::strncmp(p, "cuda_err@", 9) == 0) {
            slot = launch_at;
            p += 9;
        } else {
            return false;
        }
        char* end = nullptr;
        const long k = std::strtol(p, &end, 10);
        if (end == p || k < 1) return false;
        *slot = k;
        p = end;
        if (*p == ',') {
            if (!*++p) return false;  // a list does not end in a comma
        } else if (*p) {
            return false;
        }
    }
    return true;
}

void read_fault_env_locked() {
    if (g_fault_env_read) return;
    g_fault_env_read = true;
    long a = -1, b = -1;
    if (parse_fault_plan(std::getenv("AC_FAULT"), &a, &b)) {
        g_fault_oom_at = a;
        g_fault_launch_at = b;
    }
}

bool inject_oom() {
    std::lock_guard<std::mutex> lk(g_fault_mu);
    read_fault_env_locked();
    ++g_alloc_count;
    return g_fault_oom_at > 0 && g_alloc_count == g_fault_oom_at;
}

// Device bytes held by the library's own synchronous allocations (machines,
// streams, batch plans, tuner buffers), for ac_mem_usage.
std::mutex g_live_mu;
std::unordered_map<void*, size_t> g_live;
uint64_t g_live_bytes = 0;

}  // namespace

bool ac_fault_launch() {
    std::lock_guard<std::mutex> lk(g_fault_mu);
    read_fault_env_locked();
    ++g_launch_count;
    return g_fault_launch_at > 0 && g_launch_count == g_fault_launch_at;
}

cudaError_t ac_dev_alloc_async(void** p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    if (bytes == 0) return cudaSuccess;
    if (inject_oom()) return cudaErrorMemoryAllocation;
    return cudaMallocAsync(p, bytes, st);
}

cudaError_t ac_dev_alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) return cudaSuccess;
    if (inject_oom()) return cudaErrorMemoryAllocation;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) {
        std::lock_guard<std::mutex> lk(g_live_mu);
        g_live[*p] = bytes;
        g_live_bytes += bytes;
    }
    return e;
}

void ac_dev_free(void* p) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lk(g_live_mu);
        auto it = g_live.find(p);
        if (it != g_live.end()) {
            g_live_bytes -= it->second;
            g_live.erase(it);
        }
    }
    cudaFree(p);
}

extern "C" int ac_fault_inject(const char* spec) {
    long a = -1, b = -1;
    if (!parse_fault_plan(spec, &a, &b)) return AC_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lk(g_fault_mu);
    g_fault_env_read = true;  // an explicit plan replaces AC_FAULT
    g_fault_oom_at = a;
    g_fault_launch_at = b;
    g_alloc_count = g_launch_count = 0;
    return AC_OK;
}

extern "C" int ac_mem_usage(ac_mem_usage_t* out) {
    if (!out) return AC_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof *out);
    {
        std::lock_guard<std::mutex> lk(g_live_mu);
        out->live_bytes = g_live_bytes;
        out->live_allocations = (uint64_t)g_live.size();
    }
    int dev = 0;
    cudaMemPool_t pool;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess)
        return AC_ERR_CUDA;
    uint64_t v = 0;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &v) != cudaSuccess) return AC_ERR_CUDA;
    out->pool_used_bytes = v;
    if (cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &v) != cudaSuccess) return AC_ERR_CUDA;
    out->pool_reserved_bytes = v;
    {
        std::lock_guard<std::mutex> lk(g_fault_mu);
        out->allocations_seen = (uint64_t)g_alloc_count;
        out->launches_seen = (uint64_t)g_launch_count;
    }
    return AC_OK;
}

namespace {

cudaError_t dev_alloc_async(void** p, size_t bytes, cudaStream_t st) { return ac_dev_alloc_async(p, bytes, st); }
cudaError_t dev_alloc(void** p, size_t bytes) { return ac_dev_alloc(p, bytes); }

void keep_pool_memory() {
    static std::once_flag once[64];
    int dev = 0;
    cudaGetDevice(&dev);
    std::call_once(once[dev & 63], [dev] {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;  // this process's pool keeps freed blocks for reuse
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    });
}

// A list of stream-ordered allocations released together at the end of a call.
struct Scratch {
    cudaStream_t st;
    std::vector<void*> ptrs;
    explicit Scratch(cudaStream_t s) : st(s) {}
    cudaError_t get(void** p, size_t bytes) {
        cudaError_t e = dev_alloc_async(p, bytes, st);
        if (e == cudaSuccess && *p) ptrs.push_back(*p);
        return e;
    }
    ~Scratch() {
        for (void* p : ptrs) cudaFreeAsync(p, st);
    }
};

// pinned 32-byte landing pad per host thread for the small D2H reads
unsigned long long* pinned_pad() {
    static thread_local unsigned long long* pad = nullptr;
    if (!pad) {
        if (cudaMallocHost(&pad, 4 * sizeof(unsigned long long)) != cudaSuccess) pad = nullptr;
    }
    return pad;
}

// Sets a 4-word counter block to {0, 0, ~0, ~0} (occurrences, cursor, bad
// offset, pad) with one copy from a constant pinned block.
cudaError_t init_counters(unsigned long long* d_ctr, cudaStream_t st) {
    static unsigned long long* init = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* p = nullptr;
        if (cudaMallocHost(&p, 4 * sizeof(unsigned long long)) == cudaSuccess) {
            unsigned long long* v = static_cast<unsigned long long*>(p);
            v[0] = v[1] = 0;
            v[2] = v[3] = ~0ull;
            init = v;
        }
    });
    if (!init) {  // no pinned memory: two memsets
        cudaError_t e = cudaMemsetAsync(d_ctr, 0, 2 * sizeof(unsigned long long), st);
        return e != cudaSuccess ? e : cudaMemsetAsync(d_ctr + 2, 0xff, 2 * sizeof(unsigned long long), st);
    }
    return cudaMemcpyAsync(d_ctr, init, 4 * sizeof(unsigned long long), cudaMemcpyHostToDevice, st);
}

struct Events {
    bool on = false;
    cudaEvent_t ev[8] = {};
    cudaStream_t st = nullptr;
    Events(bool enable, cudaStream_t s) : on(enable), st(s) {
        if (on)
            for (auto& e : ev) cudaEventCreate(&e);
    }
    void rec(int i) {
        if (on) cudaEventRecord(ev[i], st);
    }
    float ms(int a, int b) {
        float v = 0.f;
        if (on) cudaEventElapsedTime(&v, ev[a], ev[b]);
        return v;
    }
    ~Events() {
        if (on)
            for (auto& e : ev) cudaEventDestroy(e);
    }
};

uint64_t round_up(uint64_t x, uint64_t m) { return (x + m - 1) / m * m; }

}  // namespace

// ------------------------------------------------------------------ status

extern "C" const char* ac_status_str(int s) {
    switch (s) {
        case AC_OK: return "ok";
        case AC_ERR_INVALID_ARG: return "invalid argument";
        case AC_ERR_ALPHABET: return "byte outside {A,C,G,T}";
        case AC_ERR_EMPTY_PATTERN: return "empty keyword";
        case AC_ERR_TOO_LARGE: return "too large";
        case AC_ERR_OOM: return "out of memory";
        case AC_ERR_OVERFLOW: return "occurrence buffer too small (counts exact)";
        case AC_ERR_CUDA: return "CUDA error";
        case AC_ERR_TIMEOUT: return "timed out";
        case AC_ERR_BUSY: return "busy (admission refused)";
        case AC_ERR_NOT_FOUND: return "not found";
        case AC_ERR_NO_DEVICE: return "object has no device tables";
        default: return "unknown status";
    }
}

// ------------------------------------------------------------------- build

extern "C" int ac_build(const char* const* patterns, const uint32_t* lens, uint32_t n_patterns,
                        const ac_build_opts* opts, ac_dfa** out) {
    AcRange trace_("ac_build");
    if (!out || !patterns || !lens || n_patterns == 0) return AC_ERR_INVALID_ARG;
    const auto t0 = std::chrono::steady_clock::now();
    const uint32_t flags = opts ? opts->flags : 0u;
    ac_dfa* d = new (std::nothrow) ac_dfa();
    if (!d) return AC_ERR_OOM;
    static std::atomic<uint64_t> next_serial{1};
    d->serial = next_serial++;
    int rc = ac_build_host(patterns, lens, n_patterns, (flags & AC_BUILD_FOLD_CASE) != 0,
                           (flags & AC_BUILD_NO_STRIDE2) == 0, opts ? opts->stride2_states : 0u,
                           (flags & AC_BUILD_NO_STRIDE3) == 0, opts ? opts->stride3_states : 0u,
                           (flags & AC_BUILD_FAILURELESS) != 0, &d->host, nullptr);
    if (rc != AC_OK) {
        delete d;
        return rc;
    }
    if (!(flags & AC_BUILD_HOST_ONLY)) {
        const HostTables& h = d->host;
        cudaGetDevice(&d->device);
        struct Up {
            uint32_t** dst;
            const std::vector<uint32_t>* src;
        } ups[] = {{&d->d_delta, &h.delta},   {&d->d_out_off, &h.out_off}, {&d->d_out_ent, &h.out_ent},
                   {&d->d_delta2, &h.delta2}, {&d->d_gotos, &h.gotos},     {&d->d_own_off, &h.own_off},
                   {&d->d_own_ent, &h.own_ent}, {&d->d_delta3, &h.delta3}};
        cudaError_t e = cudaSuccess;
        for (auto& u : ups) {
            const bool optional =
                u.dst == &d->d_delta2 || u.dst == &d->d_gotos || u.dst == &d->d_own_off || u.dst == &d->d_own_ent ||
                u.dst == &d->d_delta3;
            if (optional && u.src->empty()) continue;  // two-base / failure-less tables not built
            const size_t bytes = std::max<size_t>(u.src->size(), 1) * sizeof(uint32_t);
            e = dev_alloc((void**)u.dst, bytes);
            if (e != cudaSuccess) break;
            d->device_bytes += bytes;
            if (!u.src->empty()) e = cudaMemcpy(*u.dst, u.src->data(), u.src->size() * 4, cudaMemcpyHostToDevice);
            if (e != cudaSuccess) break;
        }
        if (e != cudaSuccess) {
            ac_free(d);
            return cuda_status(e);
        }
        d->on_device = true;
    }
    d->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    *out = d;
    return AC_OK;
}

extern "C" void ac_free(ac_dfa* d) {
    if (!d) return;
    if (d->d_delta || d->d_delta2 || d->d_out_off || d->d_out_ent) {
        int cur = 0;
        cudaGetDevice(&cur);
        if (d->device >= 0) cudaSetDevice(d->device);
        cudaDeviceSynchronize();
        ac_dev_free(d->d_delta);
        ac_dev_free(d->d_delta2);
        ac_dev_free(d->d_delta3);
        ac_dev_free(d->d_out_off);
        ac_dev_free(d->d_out_ent);
        ac_dev_free(d->d_gotos);
        ac_dev_free(d->d_own_off);
        ac_dev_free(d->d_own_ent);
        cudaSetDevice(cur);
    }
    delete d;
}

extern "C" int ac_dfa_info(const ac_dfa* d, ac_dfa_info_t* o) {
    if (!d || !o) return AC_ERR_INVALID_ARG;
    const HostTables& h = d->host;
    o->n_states = h.n_states;
    o->n_patterns = h.n_patterns;
    o->max_len = h.max_len;
    o->min_len = h.min_len;
    o->max_depth = h.max_depth;
    o->on_device = d->on_device ? 1u : 0u;
    o->table_bytes = (uint64_t)h.n_states * 16;
    o->out_entries = h.out_pid.size();
    o->device_bytes = d->device_bytes;
    o->build_ms = d->build_ms;
    o->table2_bytes = (uint64_t)h.s2_rows * 64;
    o->table3_bytes = (uint64_t)h.s3_rows * 256;
    return AC_OK;
}

extern "C" int ac_dfa_tables(const ac_dfa* d, ac_dfa_tables_t* o) {
    if (!d || !o) return AC_ERR_INVALID_ARG;
    const HostTables& h = d->host;
    o->delta = h.delta.data();
    o->out_off = h.out_off.data();
    o->out_pid = h.out_pid.data();
    o->pat_len = h.pat_len.data();
    o->pat_state = h.pat_state.data();
    o->depth = h.depth.data();
    o->fail = h.fail.data();
    o->delta2 = h.delta2.empty() ? nullptr : h.delta2.data();
    o->delta3 = h.delta3.empty() ? nullptr : h.delta3.data();
    o->gotos = h.gotos.empty() ? nullptr : h.gotos.data();
    o->own_off = h.own_off.empty() ? nullptr : h.own_off.data();
    o->own_pid = h.own_pid.empty() ? nullptr : h.own_pid.data();
    return AC_OK;
}

// -------------------------------------------------------------------- pack

extern "C" int ac_pack(const uint8_t* ascii, uint64_t n, uint32_t* packed, uint32_t flags, uint64_t* bad_offset,
                       void* stream) {
    AcRange trace_("ac_pack");
    if (bad_offset) *bad_offset = ~0ull;
    if (n == 0) return AC_OK;
    if (!ascii || !packed || (reinterpret_cast<uintptr_t>(packed) & 15)) return AC_ERR_INVALID_ARG;
    keep_pool_memory();
    cudaStream_t st = (cudaStream_t)stream;
    unsigned long long* d_bad = nullptr;
    Scratch sc(st);
    cudaError_t e = sc.get((void**)&d_bad, sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_status(e);
    e = cudaMemsetAsync(d_bad, 0xff, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return cuda_status(e);
    int rc = ac_launch_pack(ascii, n, packed, (flags & AC_SCAN_FOLD_CASE) != 0, d_bad, stream);
    if (rc) return cuda_status((cudaError_t)rc);
    unsigned long long* pad = pinned_pad();
    if (!pad) return AC_ERR_OOM;
    e = cudaMemcpyAsync(pad, d_bad, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    if (bad_offset) *bad_offset = pad[0];
    return pad[0] == ~0ull ? AC_OK : AC_ERR_ALPHABET;
}

// ----------------------------------------------------------------- shapes

uint32_t ac_chunk_for(uint64_t owned, uint64_t lanes, uint32_t cpl, uint32_t halo) {
    const uint64_t per = std::max<uint64_t>(lanes, 1) * std::max<uint32_t>(cpl, 1);
    uint64_t c = (owned + per - 1) / per;
    // short texts: at least 64 owned bases per chunk (walk latency, not halo
    // re-reads, is what a short text costs)
    c = std::max<uint64_t>(c, std::max<uint64_t>(64, round_up(halo, 64)));
    return (uint32_t)std::min<uint64_t>(c, 1u << 30);
}

ScanShape ac_default_shape(const ac_dfa* dfa, uint64_t owned, const ac_scan_opts* o) {
    const DeviceProps& p = ac_device_props();
    const HostTables& h = dfa->host;
    ScanShape sh;
    bool tuned_hot_set = false;  // a tuned shape may ask for 0 states in shared memory
    if (!(o && o->chunk && o->threads && o->interleave && o->hot_states >= 0)) {
        ScanShape tuned;
        if (ac_tuned_lookup(dfa, owned, &tuned)) {
            sh = tuned;
            tuned_hot_set = true;
        }
    }
    if (o && o->threads) sh.threads = o->threads;
    if (o && o->interleave) sh.interleave = o->interleave;
    if (o && o->stride) sh.stride = o->stride;
    if (o && o->hot_states >= 0) sh.hot = (uint32_t)o->hot_states;
    if (o && o->chunks_per_lane) sh.cpl = o->chunks_per_lane;
    if (o && o->chunk) sh.chunk = o->chunk;
    // built-in default (measured best on the benchmark workloads when untuned):
    // one chain per thread, 1024 threads, half of the shared memory for states
    if (!sh.interleave) sh.interleave = 1;
    if (sh.stride == 3 && !dfa->d_delta3) sh.stride = 2;
    if (!sh.stride || (sh.stride == 2 && !dfa->d_delta2)) sh.stride = 1;
    if (sh.stride == 2 && sh.interleave > 4) sh.interleave = 4;
    if (sh.stride == 3 && sh.interleave > 2) sh.interleave = 2;
    if (!sh.threads) sh.threads = ac_max_threads(sh.interleave, sh.stride);
    sh.threads = std::min(sh.threads, ac_max_threads(sh.interleave, sh.stride));
    const uint32_t max_hot = ac_max_hot_states(sh.threads, sh.stride);
    if (!(o && o->hot_states >= 0) && !sh.hot && !tuned_hot_set) sh.hot = std::min(h.n_states, max_hot / 2);
    sh.hot = std::min(std::min(sh.hot, h.n_states), max_hot);
    if (sh.stride == 2) sh.hot = std::min(sh.hot, h.s2_rows);  // staged from the two-base rows
    if (sh.stride == 3) sh.hot = std::min(sh.hot, h.s3_rows);  // staged from the three-base rows
    sh.blocks_per_sm = std::max(1u, ac_blocks_per_sm(sh, h.s3_rows >= h.n_states));
    const uint64_t lanes = (uint64_t)p.sms * sh.blocks_per_sm * sh.threads * sh.interleave;
    if (!sh.chunk) {
        if (!sh.cpl) sh.cpl = 1;  // one chunk per lane unless tuned or asked otherwise
        sh.chunk = ac_chunk_for(owned, lanes, sh.cpl, h.max_len ? h.max_len - 1 : 0);
    } else if (o && o->chunk) {
        sh.cpl = 0;  // the caller's chunk
    }
    const uint64_t n_chunks = (owned + sh.chunk - 1) / sh.chunk;
    const uint64_t per_block = (uint64_t)sh.threads * sh.interleave;
    const uint64_t want = std::max<uint64_t>(1, (n_chunks + per_block - 1) / per_block);
    sh.grid = (uint32_t)std::min<uint64_t>(want, (uint64_t)p.sms * sh.blocks_per_sm);
    return sh;
}

bool ac_valid_shape_opts(const ac_scan_opts* o) {
    if (!o) return true;
    if (o->threads && (o->threads < 32 || o->threads > 1024 || o->threads % 32)) return false;
    if (o->interleave && o->interleave != 1 && o->interleave != 2 && o->interleave != 4 && o->interleave != 8)
        return false;
    if (o->threads && o->threads > ac_max_threads(o->interleave ? o->interleave : 1)) return false;
    if (o->stride > 3 || (o->stride == 2 && o->interleave == 8) || (o->stride == 3 && o->interleave > 2)) return false;
    if (o->chunks_per_lane && o->chunks_per_lane != 1 && o->chunks_per_lane != 2 && o->chunks_per_lane != 4 &&
        o->chunks_per_lane != 8)
        return false;
    return true;
}

bool ac_stride_tables_present(const ac_dfa* dfa, const ac_scan_opts* o) {
    return !(o && ((o->stride == 2 && !dfa->d_delta2) || (o->stride == 3 && !dfa->d_delta3)));
}

namespace {

bool valid_shape_opts(const ac_scan_opts* o) { return ac_valid_shape_opts(o); }

size_t text_bytes(const ac_text& t) {
    return t.encoding == AC_TEXT_ASCII ? (size_t)t.n_bases : (size_t)((t.n_bases + 15) / 16) * 4;
}

// Finishes a scan: reads n_matches and the bad offset, copies host results.
int finish(cudaStream_t st, const unsigned long long* d_counter, const unsigned long long* d_bad,
           ac_result* r, const ac_match* d_matches, const unsigned long long* d_counts, uint32_t n_pat) {
    unsigned long long* pad = pinned_pad();
    if (!pad) return AC_ERR_OOM;
    cudaError_t e;
    uint64_t nm = 0, bad = ~0ull;
    if (d_bad == d_counter + 2) {  // counter and bad offset of one block: one read
        e = cudaMemcpyAsync(pad, d_counter, 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_status(e);
        nm = pad[0];
        bad = pad[2];
    } else {
        e = cudaMemcpyAsync(pad, d_counter, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && d_bad)
            e = cudaMemcpyAsync(pad + 1, d_bad, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_status(e);
        nm = pad[0];
        bad = d_bad ? pad[1] : ~0ull;
    }
    r->n_matches = nm;
    r->bad_offset = bad;
    if (bad != ~0ull) return AC_ERR_ALPHABET;
    if (!r->on_device) {
        const uint64_t k = std::min<uint64_t>(nm, r->capacity);
        if (k) e = cudaMemcpyAsync(r->matches, d_matches, k * sizeof(ac_match), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess && r->counts)
            e = cudaMemcpyAsync(r->counts, d_counts, (size_t)n_pat * 8, cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return cuda_status(e);
    }
    return nm > r->capacity ? AC_ERR_OVERFLOW : AC_OK;
}

// The scan over device-resident packed words, the count kernel and the final
// read of the occurrence count (events 3..6 of `ev`; 0..2 are the caller's).
int scan_core(const ac_dfa* dfa, const uint32_t* words, uint64_t n, uint64_t own_begin, uint64_t own_end,
              uint64_t pos_offset, ac_result* r, const ac_scan_opts* opts, cudaStream_t st, Scratch& sc,
              unsigned long long* d_ctr, unsigned long long* d_hits, bool check_alphabet, Events& ev,
              ac_scan_stats* stats, bool failureless = false) {
    const HostTables& h = dfa->host;
    cudaError_t e;
    // ---- outputs
    ac_match* d_matches = r->matches;
    unsigned long long* d_counts = (unsigned long long*)r->counts;
    if (!r->on_device) {
        if ((e = sc.get((void**)&d_matches, r->capacity * sizeof(ac_match))) != cudaSuccess) return cuda_status(e);
        if (r->counts && (e = sc.get((void**)&d_counts, (size_t)h.n_patterns * 8)) != cudaSuccess)
            return cuda_status(e);
    }
    if (failureless) {  // one lane per start position over the trie edges
        const uint32_t hot = std::min(h.n_states, ac_max_hot_states(1024, 1));
        FlArgs f;
        f.gotos = dfa->d_gotos;
        f.own_off = dfa->d_own_off;
        f.own_ent = reinterpret_cast<const uint2*>(dfa->d_own_ent);
        f.text = words;
        f.n = n;
        f.own_begin = own_begin;
        f.own_end = own_end;
        f.halo = h.max_len - 1;
        f.text_id = opts ? opts->text_id : 0u;
        f.matches = d_matches;
        f.capacity = r->capacity;
        f.counter = d_ctr;
        f.hits = d_hits;
        ev.rec(3);
        int rc = ac_launch_failureless(f, hot, st);
        if (rc) return cuda_status((cudaError_t)rc);
        ev.rec(4);
        if (d_counts) {
            if ((e = cudaMemsetAsync(d_counts, 0, (size_t)h.n_patterns * 8, st)) != cudaSuccess) return cuda_status(e);
            rc = ac_launch_counts(dfa->d_own_off, reinterpret_cast<const uint2*>(dfa->d_own_ent), h.n_states, d_hits, d_counts, st);
            if (rc) return cuda_status((cudaError_t)rc);
        }
        ev.rec(5);
        const int status =
            finish(st, d_ctr, check_alphabet ? d_ctr + 2 : nullptr, r, d_matches, d_counts, h.n_patterns);
        ev.rec(6);
        if (stats) {
            cudaEventSynchronize(ev.ev[6]);
            stats->total_ms = ev.ms(0, 6);
            stats->pack_ms = ev.ms(1, 2);
            stats->scan_ms = ev.ms(3, 4);
            stats->counts_ms = ev.ms(4, 5);
            stats->chunk = 1;
            stats->threads = 1024;
            stats->interleave = 1;
            stats->hot_states = hot;
            stats->grid = 0;
            stats->blocks_per_sm = 0;
            stats->stride = 1;
            stats->chunks_per_lane = 0;
            stats->bases_walked = own_end - own_begin;
        }
        return status;
    }
    // ---- the scan
    const ScanShape sh = ac_default_shape(dfa, own_end - own_begin, opts);
    ScanArgs a;
    a.delta = dfa->d_delta;
    a.delta2 = dfa->d_delta2;
    a.s2_rows = h.s2_rows;
    a.delta3 = dfa->d_delta3;
    a.s3_rows = h.s3_rows;
    a.out_off = dfa->d_out_off;
    a.out_ent = reinterpret_cast<const uint2*>(dfa->d_out_ent);
    a.n_states = h.n_states;
    a.text = words;
    a.n = n;
    a.own_begin = own_begin;
    a.own_end = own_end;
    a.halo = h.max_len - 1;
    a.text_id = opts ? opts->text_id : 0u;
    a.matches = d_matches;
    a.capacity = r->capacity;
    a.counter = d_ctr;
    a.hits = d_hits;
    a.pos_offset = pos_offset;
    ev.rec(3);
    int rc = ac_launch_scan(a, sh, st);
    if (rc) return cuda_status((cudaError_t)rc);
    ev.rec(4);
    if (d_counts) {
        if ((e = cudaMemsetAsync(d_counts, 0, (size_t)h.n_patterns * 8, st)) != cudaSuccess) return cuda_status(e);
        rc = ac_launch_counts(dfa->d_out_off, reinterpret_cast<const uint2*>(dfa->d_out_ent), h.n_states, d_hits, d_counts, st);
        if (rc) return cuda_status((cudaError_t)rc);
    }
    ev.rec(5);
    const int status = finish(st, d_ctr, check_alphabet ? d_ctr + 2 : nullptr, r, d_matches, d_counts, h.n_patterns);
    ev.rec(6);
    if (stats) {
        cudaEventSynchronize(ev.ev[6]);
        stats->total_ms = ev.ms(0, 6);
        stats->pack_ms = ev.ms(1, 2);
        stats->scan_ms = ev.ms(3, 4);
        stats->counts_ms = ev.ms(4, 5);
        stats->chunk = sh.chunk;
        stats->threads = sh.threads;
        stats->interleave = sh.interleave;
        stats->hot_states = sh.hot;
        stats->grid = sh.grid;
        stats->blocks_per_sm = sh.blocks_per_sm;
        stats->stride = sh.stride;
        stats->chunks_per_lane = sh.cpl;
        const uint64_t owned = own_end - own_begin;
        const uint64_t n_chunks = owned ? (owned + sh.chunk - 1) / sh.chunk : 0;
        stats->bases_walked = owned + n_chunks * (uint64_t)(h.max_len - 1);
    }
    return status;
}

// Brings a text onto the device as packed words (staging host data through
// scratch, packing ASCII with the alphabet check into bad).
int stage_packed(const ac_text* text, uint32_t fold, cudaStream_t st, Scratch& sc, unsigned long long* bad,
                 const uint32_t** words) {
    cudaError_t e;
    const uint64_t n = text->n_bases;
    const void* src = text->data;
    *words = nullptr;
    if (!n) return AC_OK;
    if (!text->on_device) {
        void* d_src = nullptr;
        if ((e = sc.get(&d_src, round_up(text_bytes(*text), 16))) != cudaSuccess) return cuda_status(e);
        if ((e = cudaMemcpyAsync(d_src, text->data, text_bytes(*text), cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_status(e);
        src = d_src;
    }
    if (text->encoding == AC_TEXT_ASCII) {
        uint32_t* d_packed = nullptr;
        if ((e = sc.get((void**)&d_packed, round_up((n + 15) / 16 * 4, 16))) != cudaSuccess) return cuda_status(e);
        const int rc = ac_launch_pack((const uint8_t*)src, n, d_packed, fold != 0, bad, st);
        if (rc) return cuda_status((cudaError_t)rc);
        *words = d_packed;
    } else {
        *words = (const uint32_t*)src;
    }
    return AC_OK;
}

constexpr uint64_t kPipePiece = 256ull << 20;  // owned bases per piece of a host-buffer scan
int scan_pipelined(const ac_dfa* dfa, const ac_text* text, ac_result* r, const ac_scan_opts* opts, cudaStream_t st,
                   uint64_t own_begin, uint64_t own_end);

}  // namespace

// -------------------------------------------------------------------- scan

extern "C" int ac_scan(const ac_dfa* dfa, const ac_text* text, ac_result* r, const ac_scan_opts* opts, void* stream,
                       ac_scan_stats* stats) {
    AcRange trace_("ac_scan");
    if (!dfa || !text || !r) return AC_ERR_INVALID_ARG;
    r->bad_offset = ~0ull;
    if (!dfa->on_device) return AC_ERR_NO_DEVICE;
    if (text->encoding != AC_TEXT_ASCII && text->encoding != AC_TEXT_PACKED2) return AC_ERR_INVALID_ARG;
    if (text->n_bases && !text->data) return AC_ERR_INVALID_ARG;
    if (text->n_bases >= AC_MAX_BASES) return AC_ERR_TOO_LARGE;
    if (r->capacity && !r->matches) return AC_ERR_INVALID_ARG;
    if (r->on_device && (reinterpret_cast<uintptr_t>(r->matches) & 15)) return AC_ERR_INVALID_ARG;  // 16-byte records
    if (!valid_shape_opts(opts)) return AC_ERR_INVALID_ARG;
    if (opts && ((opts->stride == 2 && !dfa->d_delta2) || (opts->stride == 3 && !dfa->d_delta3)))
        return AC_ERR_INVALID_ARG;
    const uint64_t n = text->n_bases;
    const uint64_t own_begin = opts ? opts->range_begin : 0;
    const uint64_t own_end = (opts && opts->range_end) ? opts->range_end : n;
    if (own_begin > own_end || own_end > n) return AC_ERR_INVALID_ARG;
    if (text->on_device && text->encoding == AC_TEXT_PACKED2 && (reinterpret_cast<uintptr_t>(text->data) & 15))
        return AC_ERR_INVALID_ARG;
    const HostTables& h = dfa->host;
    const uint32_t fold = opts ? (opts->flags & AC_SCAN_FOLD_CASE) : 0u;
    keep_pool_memory();
    cudaStream_t st = (cudaStream_t)stream;
    if (!text->on_device && !r->on_device && !stats && own_end - own_begin >= 2 * kPipePiece)
        return scan_pipelined(dfa, text, r, opts, st, own_begin, own_end);  // overlap copies with the scan
    Events ev(stats != nullptr, st);
    Scratch sc(st);
    cudaError_t e;
    ev.rec(0);

    // ---- text onto the device, packed
    const uint32_t* words = nullptr;
    const void* src = text->data;
    if (!text->on_device && n) {
        void* d_src = nullptr;
        if ((e = sc.get(&d_src, round_up(text_bytes(*text), 16))) != cudaSuccess) return cuda_status(e);
        if ((e = cudaMemcpyAsync(d_src, text->data, text_bytes(*text), cudaMemcpyHostToDevice, st)) != cudaSuccess)
            return cuda_status(e);
        src = d_src;
    }
    unsigned long long* d_ctr = nullptr;  // [0] occurrences [1] cursor [2] bad offset [3] pad
    unsigned long long* d_hits = nullptr;
    if ((e = sc.get((void**)&d_ctr, 4 * sizeof(unsigned long long))) != cudaSuccess) return cuda_status(e);
    if ((e = sc.get((void**)&d_hits, (size_t)h.n_states * 8)) != cudaSuccess) return cuda_status(e);
    if ((e = init_counters(d_ctr, st)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaMemsetAsync(d_hits, 0, (size_t)h.n_states * 8, st)) != cudaSuccess) return cuda_status(e);
    ev.rec(1);
    if (text->encoding == AC_TEXT_ASCII && n) {
        uint32_t* d_packed = nullptr;
        if ((e = sc.get((void**)&d_packed, round_up((n + 15) / 16 * 4, 16))) != cudaSuccess) return cuda_status(e);
        int rc = ac_launch_pack((const uint8_t*)src, n, d_packed, fold != 0, d_ctr + 2, stream);
        if (rc) return cuda_status((cudaError_t)rc);
        words = d_packed;
    } else {
        words = (const uint32_t*)src;
    }
    ev.rec(2);
    return scan_core(dfa, words, n, own_begin, own_end, 0, r, opts, st, sc, d_ctr, d_hits,
                     text->encoding == AC_TEXT_ASCII, ev, stats);
}

// ------------------------------------------- host buffers: overlapped pieces
// When the text and the results are both in host memory and the owned range
// is long, the range is cut into pieces (64-base boundaries). Piece i's bases
// are copied in on one stream, scanned on the caller's stream, and its
// occurrences - which the occurrence counter places right after piece i-1's -
// are copied out on a third stream while piece i+1 is being scanned. Same
// results as the one-shot path.

namespace {

constexpr int kPipeMaxPieces = 64;
// The first piece is short, so that its occurrences, and with them the copy-out
// that bounds the whole call, start after a short copy-in and scan.
constexpr uint64_t kPipeFirstPiece = 8ull << 20;

struct CopyStreams {
    cudaStream_t in = nullptr, out = nullptr;
};

const CopyStreams& copy_streams() {
    static CopyStreams cs[64];
    static std::once_flag once[64];
    int dev = 0;
    cudaGetDevice(&dev);
    dev &= 63;
    std::call_once(once[dev], [dev] {
        cudaStreamCreateWithFlags(&cs[dev].in, cudaStreamNonBlocking);
        cudaStreamCreateWithFlags(&cs[dev].out, cudaStreamNonBlocking);
    });
    return cs[dev];
}

unsigned long long* pinned_counts() {  // one pinned slot per piece, per host thread
    static thread_local unsigned long long* pad = nullptr;
    if (!pad && cudaMallocHost(&pad, (kPipeMaxPieces + 2) * sizeof(unsigned long long)) != cudaSuccess) pad = nullptr;
    return pad;
}

int scan_pipelined(const ac_dfa* dfa, const ac_text* text, ac_result* r, const ac_scan_opts* opts, cudaStream_t st,
                   uint64_t own_begin, uint64_t own_end) {
    const HostTables& h = dfa->host;
    const uint64_t n = text->n_bases;
    const bool ascii = text->encoding == AC_TEXT_ASCII;
    const uint32_t fold = opts ? (opts->flags & AC_SCAN_FOLD_CASE) : 0u;
    const uint64_t halo = h.max_len - 1;
    const uint64_t owned = own_end - own_begin;
    const uint64_t piece = std::max<uint64_t>(kPipePiece, round_up((owned + kPipeMaxPieces - 1) / kPipeMaxPieces, 64));
    const CopyStreams& cs = copy_streams();
    unsigned long long* pad = pinned_counts();
    if (!pad || !cs.in || !cs.out) return AC_ERR_CUDA;
    Scratch sc(st);
    cudaError_t e;
    void* d_src = nullptr;  // the text as given (ASCII bytes or packed words)
    uint32_t* d_words = nullptr;
    unsigned long long *d_ctr = nullptr, *d_hits = nullptr, *d_counts = nullptr;
    ac_match* d_m = nullptr;
    if ((e = sc.get(&d_src, round_up(text_bytes(*text), 16))) != cudaSuccess) return cuda_status(e);
    if (ascii && (e = sc.get((void**)&d_words, round_up((n + 15) / 16 * 4, 16))) != cudaSuccess)
        return cuda_status(e);
    if (!ascii) d_words = (uint32_t*)d_src;
    if ((e = sc.get((void**)&d_ctr, 4 * 8)) != cudaSuccess) return cuda_status(e);
    if ((e = sc.get((void**)&d_hits, (size_t)h.n_states * 8)) != cudaSuccess) return cuda_status(e);
    if ((e = sc.get((void**)&d_m, r->capacity * sizeof(ac_match))) != cudaSuccess) return cuda_status(e);
    if (r->counts && (e = sc.get((void**)&d_counts, (size_t)h.n_patterns * 8)) != cudaSuccess) return cuda_status(e);
    if ((e = init_counters(d_ctr, st)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaMemsetAsync(d_hits, 0, (size_t)h.n_states * 8, st)) != cudaSuccess) return cuda_status(e);
    cudaEvent_t ready, in_done[kPipeMaxPieces], cnt_done[kPipeMaxPieces], out_done;
    cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&out_done, cudaEventDisableTiming);
    for (int i = 0; i < kPipeMaxPieces; ++i) {
        cudaEventCreateWithFlags(&in_done[i], cudaEventDisableTiming);
        cudaEventCreateWithFlags(&cnt_done[i], cudaEventDisableTiming);
    }
    cudaEventRecord(ready, st);  // scratch allocated and cleared
    cudaStreamWaitEvent(cs.in, ready, 0);
    const ScanShape full = ac_default_shape(dfa, owned, opts);
    const DeviceProps& p = ac_device_props();
    const uint64_t lanes = (uint64_t)p.sms * full.blocks_per_sm * full.threads * full.interleave;
    int status = AC_OK;
    uint64_t copied = (own_begin > halo ? own_begin - halo : 0) & ~63ull;  // bases on the device so far
    uint64_t out_from = 0;                                                 // occurrences already copied out
    int k = 0;
    for (uint64_t a = own_begin, b = 0; a < own_end && status == AC_OK; a = b, ++k) {
        // piece boundaries on absolute 64-base multiples (word-aligned packing); the last takes the rest
        const uint64_t step = k == 0 ? std::min<uint64_t>(piece, kPipeFirstPiece) : piece;
        b = (k == kPipeMaxPieces - 1) ? own_end : std::min<uint64_t>(own_end, (a + step) & ~63ull);
        const uint64_t upto = (b == own_end) ? n : b;  // bases the piece needs
        // ---- copy in [copied, upto)
        if (upto > copied) {
            if (ascii) {
                e = cudaMemcpyAsync((uint8_t*)d_src + copied, (const uint8_t*)text->data + copied, upto - copied,
                                    cudaMemcpyHostToDevice, cs.in);
            } else {
                const uint64_t w0 = copied / 16, w1 = (upto + 15) / 16;
                e = cudaMemcpyAsync((uint32_t*)d_src + w0, (const uint32_t*)text->data + w0, (w1 - w0) * 4,
                                    cudaMemcpyHostToDevice, cs.in);
            }
            if (e != cudaSuccess) {
                status = cuda_status(e);
                break;
            }
        }
        cudaEventRecord(in_done[k], cs.in);
        cudaStreamWaitEvent(st, in_done[k], 0);
        if (ascii && upto > copied) {  // copied is a multiple of 64 bases, so packing stays word-aligned
            // d_ctr[3] records that some piece had a bad byte (offset relative to the piece)
            const int rc = ac_launch_pack((const uint8_t*)d_src + copied, upto - copied, d_words + copied / 16,
                                          fold != 0, d_ctr + 3, st);
            if (rc) {
                status = cuda_status((cudaError_t)rc);
                break;
            }
        }
        copied = std::max(copied, upto);
        // ---- scan the owned piece
        ScanShape sh = full;  // shape of the whole range; chunks re-sized to the piece unless given
        const uint64_t len = b - a;
        if (!(opts && opts->chunk)) sh.chunk = ac_chunk_for(len, lanes, full.cpl, (uint32_t)halo);
        const uint64_t nch = (len + sh.chunk - 1) / sh.chunk;
        sh.grid = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(1, (nch + (uint64_t)sh.threads * sh.interleave - 1) /
                                                                      ((uint64_t)sh.threads * sh.interleave)),
                                               (uint64_t)p.sms * sh.blocks_per_sm);
        ScanArgs sa;
        sa.delta = dfa->d_delta;
        sa.delta2 = dfa->d_delta2;
        sa.s2_rows = h.s2_rows;
        sa.delta3 = dfa->d_delta3;
        sa.s3_rows = h.s3_rows;
        sa.out_off = dfa->d_out_off;
        sa.out_ent = reinterpret_cast<const uint2*>(dfa->d_out_ent);
        sa.n_states = h.n_states;
        sa.text = d_words;
        sa.n = n;
        sa.own_begin = a;
        sa.own_end = b;
        sa.halo = (uint32_t)halo;
        sa.text_id = opts ? opts->text_id : 0u;
        sa.matches = d_m;
        sa.capacity = r->capacity;
        sa.counter = d_ctr;
        sa.hits = d_hits;
        sa.pos_offset = 0;
        int rc = ac_launch_scan(sa, sh, st);
        if (rc) {
            status = cuda_status((cudaError_t)rc);
            break;
        }
        cudaMemcpyAsync(pad + k, d_ctr, 8, cudaMemcpyDeviceToHost, st);
        cudaEventRecord(cnt_done[k], st);
        // ---- while piece k runs: copy out piece k-1's occurrences
        if (k > 0) {
            cudaEventSynchronize(cnt_done[k - 1]);
            const uint64_t to = std::min<uint64_t>(pad[k - 1], r->capacity);
            if (to > out_from) {
                cudaStreamWaitEvent(cs.out, cnt_done[k - 1], 0);
                cudaMemcpyAsync(r->matches + out_from, d_m + out_from, (to - out_from) * sizeof(ac_match),
                                cudaMemcpyDeviceToHost, cs.out);
                out_from = to;
            }
        }
    }
    if (status == AC_OK && d_counts) {
        if ((e = cudaMemsetAsync(d_counts, 0, (size_t)h.n_patterns * 8, st)) != cudaSuccess) status = cuda_status(e);
        const int rc = ac_launch_counts(dfa->d_out_off, reinterpret_cast<const uint2*>(dfa->d_out_ent), h.n_states, d_hits, d_counts, st);
        if (status == AC_OK && rc) status = cuda_status((cudaError_t)rc);
    }
    if (status == AC_OK) {
        cudaMemcpyAsync(pad + kPipeMaxPieces, d_ctr, 8, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(pad + kPipeMaxPieces + 1, d_ctr + 3, 8, cudaMemcpyDeviceToHost, st);
        if ((e = cudaStreamSynchronize(st)) != cudaSuccess) status = cuda_status(e);
    }
    if (status == AC_OK && ascii && pad[kPipeMaxPieces + 1] != ~0ull) {
        // a bad byte somewhere: pack the whole text once more for its absolute offset
        const int rc = ac_launch_pack((const uint8_t*)d_src, n, d_words, fold != 0, d_ctr + 2, st);
        cudaMemcpyAsync(pad + kPipeMaxPieces + 1, d_ctr + 2, 8, cudaMemcpyDeviceToHost, st);
        if (rc || (e = cudaStreamSynchronize(st)) != cudaSuccess) status = AC_ERR_CUDA;
    }
    if (status == AC_OK) {
        const uint64_t nm = pad[kPipeMaxPieces];
        const uint64_t bad = ascii ? pad[kPipeMaxPieces + 1] : ~0ull;
        r->n_matches = nm;
        r->bad_offset = bad;
        const uint64_t to = std::min<uint64_t>(nm, r->capacity);
        if (to > out_from)
            cudaMemcpyAsync(r->matches + out_from, d_m + out_from, (to - out_from) * sizeof(ac_match),
                            cudaMemcpyDeviceToHost, cs.out);
        if (r->counts) cudaMemcpyAsync(r->counts, d_counts, (size_t)h.n_patterns * 8, cudaMemcpyDeviceToHost, cs.out);
        if ((e = cudaStreamSynchronize(cs.out)) != cudaSuccess) status = cuda_status(e);
        if (status == AC_OK) status = bad != ~0ull ? AC_ERR_ALPHABET : (nm > r->capacity ? AC_ERR_OVERFLOW : AC_OK);
    }
    // the scratch is released on `st`; make it wait for the copy streams first
    cudaEventRecord(out_done, cs.out);
    cudaStreamWaitEvent(st, out_done, 0);
    cudaEventRecord(ready, cs.in);
    cudaStreamWaitEvent(st, ready, 0);
    cudaStreamSynchronize(cs.in);
    cudaStreamSynchronize(cs.out);
    cudaEventDestroy(ready);
    cudaEventDestroy(out_done);
    for (int i = 0; i < kPipeMaxPieces; ++i) {
        cudaEventDestroy(in_done[i]);
        cudaEventDestroy(cnt_done[i]);
    }
    return status;
}

}  // namespace

// ------------------------------------------------------ failure-less scan

extern "C" int ac_scan_failureless(const ac_dfa* dfa, const ac_text* text, ac_result* r, const ac_scan_opts* opts,
                                   void* stream, ac_scan_stats* stats) {
    AcRange trace_("ac_scan_failureless");
    if (!dfa || !text || !r) return AC_ERR_INVALID_ARG;
    r->bad_offset = ~0ull;
    if (!dfa->on_device) return AC_ERR_NO_DEVICE;
    if (!dfa->d_gotos) return AC_ERR_INVALID_ARG;  // built without AC_BUILD_FAILURELESS
    if (text->encoding != AC_TEXT_ASCII && text->encoding != AC_TEXT_PACKED2) return AC_ERR_INVALID_ARG;
    if (text->n_bases && !text->data) return AC_ERR_INVALID_ARG;
    if (text->n_bases >= AC_MAX_BASES) return AC_ERR_TOO_LARGE;
    if (r->capacity && !r->matches) return AC_ERR_INVALID_ARG;
    if (r->on_device && (reinterpret_cast<uintptr_t>(r->matches) & 15)) return AC_ERR_INVALID_ARG;  // 16-byte records
    if (text->on_device && text->encoding == AC_TEXT_PACKED2 && (reinterpret_cast<uintptr_t>(text->data) & 15))
        return AC_ERR_INVALID_ARG;
    const uint64_t n = text->n_bases;
    const uint64_t own_begin = opts ? opts->range_begin : 0;
    const uint64_t own_end = (opts && opts->range_end) ? opts->range_end : n;
    if (own_begin > own_end || own_end > n) return AC_ERR_INVALID_ARG;
    const HostTables& h = dfa->host;
    const uint32_t fold = opts ? (opts->flags & AC_SCAN_FOLD_CASE) : 0u;
    keep_pool_memory();
    cudaStream_t st = (cudaStream_t)stream;
    Events ev(stats != nullptr, st);
    Scratch sc(st);
    cudaError_t e;
    ev.rec(0);
    unsigned long long* d_ctr = nullptr;
    unsigned long long* d_hits = nullptr;
    if ((e = sc.get((void**)&d_ctr, 4 * sizeof(unsigned long long))) != cudaSuccess) return cuda_status(e);
    if ((e = sc.get((void**)&d_hits, (size_t)h.n_states * 8)) != cudaSuccess) return cuda_status(e);
    if ((e = init_counters(d_ctr, st)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaMemsetAsync(d_hits, 0, (size_t)h.n_states * 8, st)) != cudaSuccess) return cuda_status(e);
    ev.rec(1);
    const uint32_t* words = nullptr;
    const int rc = stage_packed(text, fold, st, sc, d_ctr + 2, &words);
    if (rc != AC_OK) return rc;
    ev.rec(2);
    return scan_core(dfa, words, n, own_begin, own_end, 0, r, opts, st, sc, d_ctr, d_hits,
                     text->encoding == AC_TEXT_ASCII, ev, stats, true);
}

// --------------------------------------------------------------- streaming
// A text delivered in consecutive pieces. The stream keeps the last L_max - 1
// bases seen (the longest state string any position can depend on); each
// piece is spliced behind them and scanned owning only the piece's own end
// positions, so occurrences spanning a piece boundary are reported once, with
// global start positions.

struct ac_stream {
    const ac_dfa* dfa = nullptr;
    int device = 0;
    uint32_t* d_carry = nullptr;  // packed, carry_cap bases
    uint64_t carry_cap = 0;
    uint64_t carry_n = 0;         // bases held (<= L_max - 1)
    uint64_t consumed = 0;        // bases of the text before the next piece
};

extern "C" int ac_stream_create(const ac_dfa* dfa, ac_stream** out) {
    if (!dfa || !out) return AC_ERR_INVALID_ARG;
    if (!dfa->on_device) return AC_ERR_NO_DEVICE;
    ac_stream* s = new (std::nothrow) ac_stream();
    if (!s) return AC_ERR_OOM;
    s->dfa = dfa;
    cudaGetDevice(&s->device);
    s->carry_cap = round_up(std::max<uint64_t>(dfa->host.max_len, 16), 16);
    const cudaError_t e = dev_alloc((void**)&s->d_carry, s->carry_cap / 4 + 16);
    if (e != cudaSuccess) {
        delete s;
        return cuda_status(e);
    }
    *out = s;
    return AC_OK;
}

extern "C" int ac_stream_reset(ac_stream* s) {
    if (!s) return AC_ERR_INVALID_ARG;
    s->carry_n = 0;
    s->consumed = 0;
    return AC_OK;
}

extern "C" void ac_stream_free(ac_stream* s) {
    if (!s) return;
    cudaDeviceSynchronize();
    ac_dev_free(s->d_carry);
    delete s;
}

extern "C" int ac_stream_scan(ac_stream* s, const ac_text* piece, ac_result* r, const ac_scan_opts* opts, void* stream,
                              ac_scan_stats* stats) {
    AcRange trace_("ac_stream_scan");
    if (!s || !piece || !r) return AC_ERR_INVALID_ARG;
    r->bad_offset = ~0ull;
    const ac_dfa* dfa = s->dfa;
    if (piece->encoding != AC_TEXT_ASCII && piece->encoding != AC_TEXT_PACKED2) return AC_ERR_INVALID_ARG;
    if (piece->n_bases && !piece->data) return AC_ERR_INVALID_ARG;
    if (piece->n_bases >= AC_MAX_BASES) return AC_ERR_TOO_LARGE;
    if (r->capacity && !r->matches) return AC_ERR_INVALID_ARG;
    if (r->on_device && (reinterpret_cast<uintptr_t>(r->matches) & 15)) return AC_ERR_INVALID_ARG;  // 16-byte records
    if (!valid_shape_opts(opts)) return AC_ERR_INVALID_ARG;
    if (opts && ((opts->stride == 2 && !dfa->d_delta2) || (opts->stride == 3 && !dfa->d_delta3)))
        return AC_ERR_INVALID_ARG;
    if (piece->on_device && piece->encoding == AC_TEXT_PACKED2 && (reinterpret_cast<uintptr_t>(piece->data) & 15))
        return AC_ERR_INVALID_ARG;
    const HostTables& h = dfa->host;
    const uint64_t n = piece->n_bases;
    const uint64_t total = s->carry_n + n;
    const uint32_t fold = opts ? (opts->flags & AC_SCAN_FOLD_CASE) : 0u;
    keep_pool_memory();
    cudaStream_t st = (cudaStream_t)stream;
    Events ev(stats != nullptr, st);
    Scratch sc(st);
    cudaError_t e;
    ev.rec(0);
    unsigned long long* d_ctr = nullptr;  // [0] occurrences [1] cursor [2] bad offset [3] pad
    unsigned long long* d_hits = nullptr;
    if ((e = sc.get((void**)&d_ctr, 4 * sizeof(unsigned long long))) != cudaSuccess) return cuda_status(e);
    if ((e = sc.get((void**)&d_hits, (size_t)h.n_states * 8)) != cudaSuccess) return cuda_status(e);
    if ((e = init_counters(d_ctr, st)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaMemsetAsync(d_hits, 0, (size_t)h.n_states * 8, st)) != cudaSuccess) return cuda_status(e);
    ev.rec(1);
    const uint32_t* pw = nullptr;
    int rc = stage_packed(piece, fold, st, sc, d_ctr + 2, &pw);
    if (rc != AC_OK) return rc;
    // carry ++ piece, bit-exact at any base offset
    uint32_t* comb = nullptr;
    if ((e = sc.get((void**)&comb, round_up((total + 15) / 16 * 4, 16) + 16)) != cudaSuccess) return cuda_status(e);
    if ((rc = ac_launch_splice(comb, 0, s->d_carry, 0, s->carry_n, st)) != 0) return cuda_status((cudaError_t)rc);
    if ((rc = ac_launch_splice(comb, s->carry_n, pw, 0, n, st)) != 0) return cuda_status((cudaError_t)rc);
    ev.rec(2);
    const int status = scan_core(dfa, comb, total, s->carry_n, total, s->consumed - s->carry_n, r, opts, st, sc, d_ctr,
                                 d_hits, piece->encoding == AC_TEXT_ASCII, ev, stats);
    // on any error (overflow included) the stream is unchanged and the piece can
    // be sent again (an alphabet error's bad_offset is relative to the piece)
    if (status != AC_OK) return status;
    // the last L_max - 1 bases become the carry of the next piece (keep <= carry_cap)
    const uint64_t keep = std::min<uint64_t>(total, h.max_len ? h.max_len - 1 : 0);
    if ((rc = ac_launch_splice(s->d_carry, 0, comb, total - keep, keep, st)) != 0) return cuda_status((cudaError_t)rc);
    s->carry_n = keep;
    s->consumed += n;
    return status;
}

// ------------------------------------------------- partitioned keyword sets

namespace {
// 2-bit code of a base in either case (other bytes map to 0 here; ac_build rejects them)
inline int sym2(uint8_t c) { return ((c >> 1) ^ (c >> 2)) & 3; }
}  // namespace

struct ac_part_set {
    std::vector<ac_dfa*> parts;
    std::vector<uint32_t> first_pid;  // first keyword id of each chunk
    uint32_t n_patterns = 0;
    uint32_t max_states = 0;
    uint32_t halo = 0;
    uint64_t total_states = 0;
};

extern "C" void ac_part_set_free(ac_part_set* s) {
    if (!s) return;
    for (ac_dfa* d : s->parts) ac_free(d);
    delete s;
}

extern "C" int ac_build_partitioned(const char* const* patterns, const uint32_t* lens, uint32_t n, uint32_t max_states,
                                    const ac_build_opts* opts, ac_part_set** out) {
    AcRange trace_("ac_build_partitioned");
    if (!patterns || !lens || n == 0 || !out) return AC_ERR_INVALID_ARG;
    const uint32_t cap = max_states ? max_states : ac_max_hot_states(ac_max_threads(1), 1);
    if (cap < 2) return AC_ERR_INVALID_ARG;
    // Chunk boundaries: insert keywords into a trie, counting its states, and
    // close the chunk before a keyword that would take it past `cap`.
    std::vector<uint32_t> bounds{0};
    try {
        std::vector<int32_t> child(4, -1);
        uint32_t nodes = 1;
        for (uint32_t p = 0; p < n; ++p) {
            if (!patterns[p] || lens[p] == 0) return lens[p] == 0 ? AC_ERR_EMPTY_PATTERN : AC_ERR_INVALID_ARG;
            if ((uint64_t)lens[p] + 1 > cap) return AC_ERR_TOO_LARGE;
            for (int pass = 0; pass < 2; ++pass) {
                // new states this keyword adds (bytes outside ACGT are left to ac_build to reject)
                uint32_t s = 0, j = 0;
                for (; j < lens[p]; ++j) {
                    const int c = sym2((uint8_t)patterns[p][j]);
                    const int32_t t = child[(size_t)s * 4 + c];
                    if (t < 0) break;
                    s = (uint32_t)t;
                }
                if (nodes + (lens[p] - j) <= cap) {
                    for (; j < lens[p]; ++j) {
                        const int c = sym2((uint8_t)patterns[p][j]);
                        child[(size_t)s * 4 + c] = (int32_t)nodes;
                        child.insert(child.end(), {-1, -1, -1, -1});
                        s = nodes++;
                    }
                    break;
                }
                // close the chunk and start a new trie with this keyword
                bounds.push_back(p);
                child.assign(4, -1);
                nodes = 1;
            }
        }
        bounds.push_back(n);
    } catch (const std::bad_alloc&) {
        return AC_ERR_OOM;
    }
    ac_part_set* s = new (std::nothrow) ac_part_set();
    if (!s) return AC_ERR_OOM;
    s->n_patterns = n;
    ac_build_opts o{};
    o.flags = (opts ? opts->flags : 0u) | AC_BUILD_NO_STRIDE2 | AC_BUILD_NO_STRIDE3;
    for (size_t i = 0; i + 1 < bounds.size(); ++i) {
        const uint32_t a = bounds[i], b = bounds[i + 1];
        if (a == b) continue;
        ac_dfa* d = nullptr;
        const int rc = ac_build(patterns + a, lens + a, b - a, &o, &d);
        if (rc != AC_OK) {
            ac_part_set_free(s);
            return rc;
        }
        if (d->host.n_states > cap) {  // cannot happen with the trie count above; keep the invariant checked
            ac_free(d);
            ac_part_set_free(s);
            return AC_ERR_TOO_LARGE;
        }
        s->parts.push_back(d);
        s->first_pid.push_back(a);
        s->max_states = std::max(s->max_states, d->host.n_states);
        s->halo = std::max(s->halo, d->host.max_len - 1);
        s->total_states += d->host.n_states;
    }
    *out = s;
    return AC_OK;
}

extern "C" int ac_part_set_info(const ac_part_set* s, uint32_t* n_parts, uint32_t* max_states) {
    if (!s) return AC_ERR_INVALID_ARG;
    if (n_parts) *n_parts = (uint32_t)s->parts.size();
    if (max_states) *max_states = s->max_states;
    return AC_OK;
}

extern "C" int ac_scan_partitioned(const ac_part_set* set, const ac_text* text, ac_result* r,
                                   const ac_scan_opts* opts, void* stream, ac_scan_stats* stats) {
    AcRange trace_("ac_scan_partitioned");
    if (!set || !text || !r) return AC_ERR_INVALID_ARG;
    r->bad_offset = ~0ull;
    if (text->encoding != AC_TEXT_ASCII && text->encoding != AC_TEXT_PACKED2) return AC_ERR_INVALID_ARG;
    if (text->n_bases && !text->data) return AC_ERR_INVALID_ARG;
    if (text->n_bases >= AC_MAX_BASES) return AC_ERR_TOO_LARGE;
    if (r->capacity && !r->matches) return AC_ERR_INVALID_ARG;
    if (r->on_device && (reinterpret_cast<uintptr_t>(r->matches) & 15)) return AC_ERR_INVALID_ARG;  // 16-byte records
    if (text->on_device && text->encoding == AC_TEXT_PACKED2 && (reinterpret_cast<uintptr_t>(text->data) & 15))
        return AC_ERR_INVALID_ARG;
    const uint64_t n = text->n_bases;
    const uint64_t own_begin = opts ? opts->range_begin : 0;
    const uint64_t own_end = (opts && opts->range_end) ? opts->range_end : n;
    if (own_begin > own_end || own_end > n) return AC_ERR_INVALID_ARG;
    const uint32_t k = (uint32_t)set->parts.size();
    const uint32_t fold = opts ? (opts->flags & AC_SCAN_FOLD_CASE) : 0u;
    keep_pool_memory();
    cudaStream_t st = (cudaStream_t)stream;
    Events ev(stats != nullptr, st);
    Scratch sc(st);
    cudaError_t e;
    ev.rec(0);
    unsigned long long* d_ctr = nullptr;
    unsigned long long* d_hits = nullptr;
    PartDesc* d_parts = nullptr;
    if ((e = sc.get((void**)&d_ctr, 4 * sizeof(unsigned long long))) != cudaSuccess) return cuda_status(e);
    if ((e = sc.get((void**)&d_hits, std::max<uint64_t>(set->total_states, 1) * 8)) != cudaSuccess)
        return cuda_status(e);
    if ((e = sc.get((void**)&d_parts, std::max<size_t>(k, 1) * sizeof(PartDesc))) != cudaSuccess)
        return cuda_status(e);
    if ((e = init_counters(d_ctr, st)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaMemsetAsync(d_hits, 0, set->total_states * 8, st)) != cudaSuccess) return cuda_status(e);
    std::vector<PartDesc> pd(k);
    uint64_t off = 0;
    for (uint32_t i = 0; i < k; ++i) {
        const ac_dfa* d = set->parts[i];
        pd[i] = PartDesc{d->d_delta, d->d_out_off, reinterpret_cast<const uint2*>(d->d_out_ent), d_hits + off, d->host.n_states,
                         set->first_pid[i]};
        off += d->host.n_states;
    }
    if (k && (e = cudaMemcpyAsync(d_parts, pd.data(), k * sizeof(PartDesc), cudaMemcpyHostToDevice, st)) !=
                 cudaSuccess)
        return cuda_status(e);
    ev.rec(1);
    const uint32_t* words = nullptr;
    int rc = stage_packed(text, fold, st, sc, d_ctr + 2, &words);
    if (rc != AC_OK) return rc;
    ev.rec(2);
    ac_match* d_matches = r->matches;
    unsigned long long* d_counts = (unsigned long long*)r->counts;
    if (!r->on_device) {
        if ((e = sc.get((void**)&d_matches, r->capacity * sizeof(ac_match))) != cudaSuccess) return cuda_status(e);
        if (r->counts && (e = sc.get((void**)&d_counts, (size_t)set->n_patterns * 8)) != cudaSuccess)
            return cuda_status(e);
    }
    // one grid row per machine; the rows share the SMs
    const DeviceProps& p = ac_device_props();
    const uint32_t threads = ac_max_threads(1);
    const uint32_t gx = std::max<uint32_t>(1, (uint32_t)p.sms / std::max<uint32_t>(k, 1));
    const uint64_t owned = own_end - own_begin;
    const uint32_t chunk = (uint32_t)std::min<uint64_t>(
        std::max<uint64_t>((owned + (uint64_t)gx * threads - 1) / ((uint64_t)gx * threads),
                           std::max<uint64_t>(64, round_up(set->halo, 64))),
        1u << 30);
    PartArgs a;
    a.parts = d_parts;
    a.text = words;
    a.n = n;
    a.own_begin = own_begin;
    a.own_end = own_end;
    a.halo = set->halo;
    a.max_states = set->max_states;
    a.matches = d_matches;
    a.capacity = r->capacity;
    a.counter = d_ctr;
    ev.rec(3);
    rc = ac_launch_part_scan(a, k, gx, threads, chunk, st);
    if (rc) return cuda_status((cudaError_t)rc);
    ev.rec(4);
    if (d_counts) {
        if ((e = cudaMemsetAsync(d_counts, 0, (size_t)set->n_patterns * 8, st)) != cudaSuccess) return cuda_status(e);
        for (uint32_t i = 0; i < k; ++i) {
            const ac_dfa* d = set->parts[i];
            rc = ac_launch_counts(d->d_out_off, reinterpret_cast<const uint2*>(d->d_out_ent), d->host.n_states, pd[i].hits, d_counts + set->first_pid[i],
                                  st);
            if (rc) return cuda_status((cudaError_t)rc);
        }
    }
    ev.rec(5);
    const int status =
        finish(st, d_ctr, text->encoding == AC_TEXT_ASCII ? d_ctr + 2 : nullptr, r, d_matches, d_counts, set->n_patterns);
    ev.rec(6);
    if (stats) {
        cudaEventSynchronize(ev.ev[6]);
        stats->total_ms = ev.ms(0, 6);
        stats->pack_ms = ev.ms(1, 2);
        stats->scan_ms = ev.ms(3, 4);
        stats->counts_ms = ev.ms(4, 5);
        stats->chunk = chunk;
        stats->threads = threads;
        stats->interleave = 1;
        stats->hot_states = set->max_states;
        stats->grid = gx * k;
        stats->blocks_per_sm = 1;
        stats->stride = 1;
        stats->chunks_per_lane = 0;
        const uint64_t n_chunks = owned ? (owned + chunk - 1) / chunk : 0;
        stats->bases_walked = (uint64_t)k * (owned + n_chunks * set->halo);
    }
    return status;
}

// ------------------------------------------------------------------- batch

namespace {

struct BatchLayout {
    std::vector<BatchText> texts;             // device pointers
    std::vector<unsigned long long> prefix;   // [T+1]
};

// Shape for the persistent batched kernel: one wave of resident blocks.
ScanShape batch_shape(const ac_dfa* dfa, uint64_t total, const ac_scan_opts* opts, uint32_t n_texts) {
    ScanShape sh = ac_default_shape(dfa, total, opts);
    const DeviceProps& p = ac_device_props();
    sh.cpl = 0;
    uint32_t tuned = 0;
    if (!(opts && opts->chunk) && ac_tuned_batch_chunk(dfa, total, &tuned)) {
        sh.chunk = tuned;
    } else if (!(opts && opts->chunk)) {
        // built-in default: enough chunks for every lane of the wave, at least 256 bases each
        const uint64_t lanes = (uint64_t)p.sms * sh.blocks_per_sm * sh.threads * sh.interleave;
        const uint64_t halo = dfa->host.max_len ? dfa->host.max_len - 1 : 0;
        uint64_t c = round_up(std::max<uint64_t>(1, total / std::max<uint64_t>(lanes, 1)), 64);
        c = std::max<uint64_t>(c, std::max<uint64_t>(256, round_up(4 * halo, 64)));
        sh.chunk = (uint32_t)std::min<uint64_t>(c, 1u << 20);
    }
    (void)n_texts;
    sh.grid = (uint32_t)p.sms * sh.blocks_per_sm;
    return sh;
}

int make_prefix(const std::vector<uint64_t>& lens, uint32_t chunk, std::vector<unsigned long long>* prefix) {
    prefix->assign(lens.size() + 1, 0);
    for (size_t i = 0; i < lens.size(); ++i) (*prefix)[i + 1] = (*prefix)[i] + (lens[i] + chunk - 1) / chunk;
    return AC_OK;
}

}  // namespace

extern "C" int ac_scan_batch(const ac_dfa* dfa, const ac_text* texts, uint32_t n_texts, ac_result* r,
                             const ac_scan_opts* opts, void* stream, ac_scan_stats* stats) {
    AcRange trace_("ac_scan_batch");
    if (!dfa || !r || (n_texts && !texts)) return AC_ERR_INVALID_ARG;
    r->bad_offset = ~0ull;
    if (!dfa->on_device) return AC_ERR_NO_DEVICE;
    if (r->capacity && !r->matches) return AC_ERR_INVALID_ARG;
    if (r->on_device && (reinterpret_cast<uintptr_t>(r->matches) & 15)) return AC_ERR_INVALID_ARG;  // 16-byte records
    if (!valid_shape_opts(opts)) return AC_ERR_INVALID_ARG;
    if (opts && ((opts->stride == 2 && !dfa->d_delta2) || (opts->stride == 3 && !dfa->d_delta3)))
        return AC_ERR_INVALID_ARG;
    const HostTables& h = dfa->host;
    const int enc = n_texts ? texts[0].encoding : AC_TEXT_PACKED2;
    const int on_dev = n_texts ? texts[0].on_device : 1;
    uint64_t total = 0;
    for (uint32_t i = 0; i < n_texts; ++i) {
        const ac_text& t = texts[i];
        if (t.encoding != enc || t.on_device != on_dev) return AC_ERR_INVALID_ARG;
        if (t.encoding != AC_TEXT_ASCII && t.encoding != AC_TEXT_PACKED2) return AC_ERR_INVALID_ARG;
        if (t.n_bases && !t.data) return AC_ERR_INVALID_ARG;
        if (t.n_bases >= AC_MAX_BASES) return AC_ERR_TOO_LARGE;
        if (t.on_device && t.encoding == AC_TEXT_PACKED2 && (reinterpret_cast<uintptr_t>(t.data) & 15))
            return AC_ERR_INVALID_ARG;
        total += t.n_bases;
    }
    const uint32_t fold = opts ? (opts->flags & AC_SCAN_FOLD_CASE) : 0u;
    keep_pool_memory();
    cudaStream_t st = (cudaStream_t)stream;
    Events ev(stats != nullptr, st);
    Scratch sc(st);
    cudaError_t e;
    ev.rec(0);

    unsigned long long* d_ctr = nullptr;
    unsigned long long* d_hits = nullptr;
    if ((e = sc.get((void**)&d_ctr, 4 * sizeof(unsigned long long))) != cudaSuccess) return cuda_status(e);
    if ((e = sc.get((void**)&d_hits, (size_t)h.n_states * 8)) != cudaSuccess) return cuda_status(e);
    if ((e = init_counters(d_ctr, st)) != cudaSuccess) return cuda_status(e);
    if ((e = cudaMemsetAsync(d_hits, 0, (size_t)h.n_states * 8, st)) != cudaSuccess) return cuda_status(e);

    // ---- every text onto the device, packed, each starting on a 64-base boundary
    std::vector<BatchText> bt(n_texts);
    std::vector<uint64_t> lens(n_texts);
    for (uint32_t i = 0; i < n_texts; ++i) lens[i] = texts[i].n_bases;
    ev.rec(1);
    if (enc == AC_TEXT_PACKED2 && on_dev) {
        for (uint32_t i = 0; i < n_texts; ++i) bt[i] = BatchText{(const uint32_t*)texts[i].data, lens[i]};
    } else {
        // staging: each text at a 64-base aligned slot in one buffer
        std::vector<uint64_t> slot(n_texts + 1, 0);  // in bases
        for (uint32_t i = 0; i < n_texts; ++i) slot[i + 1] = slot[i] + round_up(lens[i], 64);
        const uint64_t all = slot[n_texts];
        uint32_t* d_words = nullptr;
        if ((e = sc.get((void**)&d_words, std::max<uint64_t>(all / 16 * 4, 16))) != cudaSuccess)
            return cuda_status(e);
        if (enc == AC_TEXT_PACKED2) {  // host packed texts: copy word ranges
            for (uint32_t i = 0; i < n_texts; ++i)
                if (lens[i] &&
                    (e = cudaMemcpyAsync(d_words + slot[i] / 16, texts[i].data, (lens[i] + 15) / 16 * 4,
                                         cudaMemcpyHostToDevice, st)) != cudaSuccess)
                    return cuda_status(e);
        } else {  // ASCII: gather into one ASCII buffer padded with 'A', then one pack
            uint8_t* d_ascii = nullptr;
            if ((e = sc.get((void**)&d_ascii, std::max<uint64_t>(all, 16))) != cudaSuccess) return cuda_status(e);
            if (all && (e = cudaMemsetAsync(d_ascii, 'A', all, st)) != cudaSuccess) return cuda_status(e);
            for (uint32_t i = 0; i < n_texts; ++i)
                if (lens[i] &&
                    (e = cudaMemcpyAsync(d_ascii + slot[i], texts[i].data, lens[i],
                                         on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st)) !=
                        cudaSuccess)
                    return cuda_status(e);
            int rc = ac_launch_pack(d_ascii, all, d_words, fold != 0, d_ctr + 2, stream);
            if (rc) return cuda_status((cudaError_t)rc);
        }
        for (uint32_t i = 0; i < n_texts; ++i) bt[i] = BatchText{d_words + slot[i] / 16, lens[i]};
    }
    ev.rec(2);

    // ---- work items and the text table
    ScanShape sh = batch_shape(dfa, total, opts, n_texts);
    std::vector<unsigned long long> prefix;
    make_prefix(lens, sh.chunk, &prefix);
    BatchText* d_bt = nullptr;
    unsigned long long* d_prefix = nullptr;
    if ((e = sc.get((void**)&d_bt, std::max<size_t>(n_texts, 1) * sizeof(BatchText))) != cudaSuccess)
        return cuda_status(e);
    if ((e = sc.get((void**)&d_prefix, prefix.size() * 8)) != cudaSuccess) return cuda_status(e);
    if (n_texts &&
        (e = cudaMemcpyAsync(d_bt, bt.data(), n_texts * sizeof(BatchText), cudaMemcpyHostToDevice, st)) !=
            cudaSuccess)
        return cuda_status(e);
    if ((e = cudaMemcpyAsync(d_prefix, prefix.data(), prefix.size() * 8, cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
        return cuda_status(e);
    // the host vectors must outlive the async copies from pageable memory:
    // pageable cudaMemcpyAsync returns after the source has been staged.

    ac_match* d_matches = r->matches;
    unsigned long long* d_counts = (unsigned long long*)r->counts;
    if (!r->on_device) {
        if ((e = sc.get((void**)&d_matches, r->capacity * sizeof(ac_match))) != cudaSuccess) return cuda_status(e);
        if (r->counts && (e = sc.get((void**)&d_counts, (size_t)h.n_patterns * 8)) != cudaSuccess)
            return cuda_status(e);
    }
    BatchArgs a;
    a.delta = dfa->d_delta;
    a.delta2 = dfa->d_delta2;
    a.s2_rows = h.s2_rows;
    a.delta3 = dfa->d_delta3;
    a.s3_rows = h.s3_rows;
    a.out_off = dfa->d_out_off;
    a.out_ent = reinterpret_cast<const uint2*>(dfa->d_out_ent);
    a.n_states = h.n_states;
    a.texts = d_bt;
    a.item_prefix = d_prefix;
    a.n_texts = n_texts;
    a.n_items = prefix.back();
    a.chunk = sh.chunk;
    a.halo = h.max_len - 1;
    a.matches = d_matches;
    a.capacity = r->capacity;
    a.counter = d_ctr;
    a.hits = d_hits;
    ev.rec(3);
    int rc = ac_launch_batch(a, sh, stream);
    if (rc) return cuda_status((cudaError_t)rc);
    ev.rec(4);
    if (d_counts) {
        if ((e = cudaMemsetAsync(d_counts, 0, (size_t)h.n_patterns * 8, st)) != cudaSuccess) return cuda_status(e);
        rc = ac_launch_counts(dfa->d_out_off, reinterpret_cast<const uint2*>(dfa->d_out_ent), h.n_states, d_hits, d_counts, stream);
        if (rc) return cuda_status((cudaError_t)rc);
    }
    ev.rec(5);
    int status = finish(st, d_ctr, enc == AC_TEXT_ASCII ? d_ctr + 2 : nullptr, r, d_matches, d_counts, h.n_patterns);
    ev.rec(6);
    if (stats) {
        cudaEventSynchronize(ev.ev[6]);
        stats->total_ms = ev.ms(0, 6);
        stats->pack_ms = ev.ms(1, 2);
        stats->scan_ms = ev.ms(3, 4);
        stats->counts_ms = ev.ms(4, 5);
        stats->chunk = sh.chunk;
        stats->threads = sh.threads;
        stats->interleave = sh.interleave;
        stats->hot_states = sh.hot;
        stats->grid = sh.grid;
        stats->blocks_per_sm = sh.blocks_per_sm;
        stats->stride = sh.stride;
        stats->chunks_per_lane = 0;
        stats->bases_walked = total + prefix.back() * (uint64_t)(h.max_len - 1);
    }
    return status;
}

// ------------------------------------------------------------ batch plans

struct ac_batch_plan {
    const ac_dfa* dfa = nullptr;
    int device = 0;
    uint32_t n_patterns = 0;
    uint64_t capacity = 0;
    BatchText* d_bt = nullptr;
    unsigned long long* d_prefix = nullptr;
    unsigned long long* d_ctr = nullptr;
    unsigned long long* d_hits = nullptr;
    unsigned long long* h_pad = nullptr;  // pinned: [0] n_matches
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

extern "C" void ac_batch_plan_free(ac_batch_plan* p) {
    if (!p) return;
    cudaDeviceSynchronize();
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    ac_dev_free(p->d_bt);
    ac_dev_free(p->d_prefix);
    ac_dev_free(p->d_ctr);
    ac_dev_free(p->d_hits);
    if (p->h_pad) cudaFreeHost(p->h_pad);
    delete p;
}

extern "C" int ac_batch_plan_create(const ac_dfa* dfa, const ac_text* texts, uint32_t n_texts, ac_result* r,
                                    const ac_scan_opts* opts, void* stream, ac_batch_plan** out) {
    AcRange trace_("ac_batch_plan_create");
    if (!dfa || !r || !out || (n_texts && !texts)) return AC_ERR_INVALID_ARG;
    if (!dfa->on_device) return AC_ERR_NO_DEVICE;
    if (!r->on_device || (r->capacity && !r->matches)) return AC_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(r->matches) & 15) return AC_ERR_INVALID_ARG;  // 16-byte records
    if (!valid_shape_opts(opts)) return AC_ERR_INVALID_ARG;
    if (opts && ((opts->stride == 2 && !dfa->d_delta2) || (opts->stride == 3 && !dfa->d_delta3)))
        return AC_ERR_INVALID_ARG;
    const HostTables& h = dfa->host;
    std::vector<BatchText> bt(n_texts);
    std::vector<uint64_t> lens(n_texts);
    uint64_t total = 0;
    for (uint32_t i = 0; i < n_texts; ++i) {
        const ac_text& t = texts[i];
        if (t.encoding != AC_TEXT_PACKED2 || !t.on_device) return AC_ERR_INVALID_ARG;
        if ((t.n_bases && !t.data) || (reinterpret_cast<uintptr_t>(t.data) & 15)) return AC_ERR_INVALID_ARG;
        if (t.n_bases >= AC_MAX_BASES) return AC_ERR_TOO_LARGE;
        bt[i] = BatchText{(const uint32_t*)t.data, t.n_bases};
        lens[i] = t.n_bases;
        total += t.n_bases;
    }
    ac_batch_plan* p = new (std::nothrow) ac_batch_plan();
    if (!p) return AC_ERR_OOM;
    p->dfa = dfa;
    p->n_patterns = h.n_patterns;
    p->capacity = r->capacity;
    cudaGetDevice(&p->device);
    ScanShape sh = batch_shape(dfa, total, opts, n_texts);
    std::vector<unsigned long long> prefix;
    make_prefix(lens, sh.chunk, &prefix);
    cudaError_t e = cudaSuccess;
    (void)stream;  // capture happens on a private stream; runs go to the caller's
    auto fail = [&](cudaError_t err) {
        ac_batch_plan_free(p);
        return cuda_status(err);
    };
    if ((e = dev_alloc((void**)&p->d_bt, std::max<size_t>(n_texts, 1) * sizeof(BatchText))) != cudaSuccess)
        return fail(e);
    if ((e = dev_alloc((void**)&p->d_prefix, prefix.size() * 8)) != cudaSuccess) return fail(e);
    if ((e = dev_alloc((void**)&p->d_ctr, 4 * 8)) != cudaSuccess) return fail(e);
    if ((e = dev_alloc((void**)&p->d_hits, (size_t)h.n_states * 8)) != cudaSuccess) return fail(e);
    if ((e = cudaMallocHost(&p->h_pad, 4 * 8)) != cudaSuccess) return fail(e);
    if (n_texts && (e = cudaMemcpy(p->d_bt, bt.data(), n_texts * sizeof(BatchText), cudaMemcpyHostToDevice)) !=
                       cudaSuccess)
        return fail(e);
    if ((e = cudaMemcpy(p->d_prefix, prefix.data(), prefix.size() * 8, cudaMemcpyHostToDevice)) != cudaSuccess)
        return fail(e);

    BatchArgs a;
    a.delta = dfa->d_delta;
    a.delta2 = dfa->d_delta2;
    a.s2_rows = h.s2_rows;
    a.delta3 = dfa->d_delta3;
    a.s3_rows = h.s3_rows;
    a.out_off = dfa->d_out_off;
    a.out_ent = reinterpret_cast<const uint2*>(dfa->d_out_ent);
    a.n_states = h.n_states;
    a.texts = p->d_bt;
    a.item_prefix = p->d_prefix;
    a.n_texts = n_texts;
    a.n_items = prefix.back();
    a.chunk = sh.chunk;
    a.halo = h.max_len - 1;
    a.matches = r->matches;
    a.capacity = r->capacity;
    a.counter = p->d_ctr;
    a.hits = p->d_hits;
    unsigned long long* d_counts = (unsigned long long*)r->counts;

    // capture on a private stream, then replay on any stream
    if ((e = (cudaError_t)ac_prepare_batch(sh)) != cudaSuccess) return fail(e);
    cudaStream_t cap = nullptr;
    if ((e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) return fail(e);
    int rc = AC_OK;
    // with counts, the count kernel sets the per-state hit counters back to 0
    // as it reads them, so replays start from zeroed counters without a memset
    if (d_counts && ((e = cudaMemsetAsync(p->d_hits, 0, (size_t)h.n_states * 8, cap)) != cudaSuccess ||
                     (e = cudaStreamSynchronize(cap)) != cudaSuccess)) {
        cudaStreamDestroy(cap);
        return fail(e);
    }
    e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        cudaMemsetAsync(p->d_ctr, 0, 4 * 8, cap);
        if (!d_counts) cudaMemsetAsync(p->d_hits, 0, (size_t)h.n_states * 8, cap);
        rc = ac_launch_batch(a, sh, cap);
        if (d_counts) {
            cudaMemsetAsync(d_counts, 0, (size_t)h.n_patterns * 8, cap);
            if (!rc)
                rc = ac_launch_counts(dfa->d_out_off, reinterpret_cast<const uint2*>(dfa->d_out_ent), h.n_states,
                                      p->d_hits, d_counts, cap, true);
        }
        cudaMemcpyAsync(p->h_pad, p->d_ctr, 8, cudaMemcpyDeviceToHost, cap);
        cudaError_t e2 = cudaStreamEndCapture(cap, &p->graph);
        if (e2 != cudaSuccess) e = e2;
    }
    cudaStreamDestroy(cap);
    if (e == cudaSuccess && rc) e = (cudaError_t)rc;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&p->exec, p->graph, 0);
    if (e != cudaSuccess) return fail(e);
    *out = p;
    return AC_OK;
}

extern "C" int ac_batch_plan_run(ac_batch_plan* p, void* stream, int sync, ac_result* r) {
    AcRange trace_("ac_batch_plan_run");
    if (!p) return AC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaGraphLaunch(p->exec, st);
    if (e != cudaSuccess) return cuda_status(e);
    if (!sync) return AC_OK;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return cuda_status(e);
    const uint64_t nm = p->h_pad[0];
    if (r) {
        r->n_matches = nm;
        r->bad_offset = ~0ull;
    }
    return nm > p->capacity ? AC_ERR_OVERFLOW : AC_OK;
}
