// ac_tune.cpp - launch-shape autotuner for the scan kernels.
//
// A shape is (bases per lookup, threads per block, chunks walked per thread,
// states staged in shared memory, chunks per resident lane); the chunk
// length follows from the shape and the text length (the owned range cut
// into chunks-per-lane chunks for every resident lane). ac_autotune times
// the candidates with CUDA events on a sample text - first every (stride,
// threads, interleave, shared-memory states) at one chunk per lane, then 2,
// 4 and 8 chunks per lane for the fastest of those - and keeps the fastest
// per (device, machine size class, text size class), where a size class is
// ceil(log2(x)). Later scans whose classes match use the tuned shape unless
// the caller fixes one. ac_autotune_batch tunes the work-item chunk of
// batched scans the same way, per (device, machine size class, total-length
// class).
//
// Environment:
//   AC_TUNE=off          skip the trials; return the built-in default shape
//   AC_TUNE_CACHE=path   load tuned shapes from / append them to a JSON file
//   AC_TUNE_VERBOSE=1    print every candidate's time to stderr
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "ac_internal.h"
#include "ac_trace.h"

namespace {

using Key = std::tuple<std::string, uint32_t, uint32_t>;  // device name+sms, log2 S, log2 n

struct Entry {
    uint32_t threads, interleave, hot, stride, cpl;
    float ms;
};

struct BatchEntry {
    uint32_t chunk;
    float ms;
};

std::mutex g_mu;
std::map<Key, Entry> g_cache;
std::map<Key, BatchEntry> g_batch;  // tuned work-item chunk of batched scans
std::map<uint64_t, Entry> g_by_dfa;  // last shape tuned (or looked up) by ac_autotune per dfa serial
bool g_loaded = false;

uint32_t size_class(uint64_t x) { return x <= 1 ? 0u : (uint32_t)std::ceil(std::log2((double)x)); }

// "<device name>_sm<count>", looked up once per device.
const std::string& device_tag() {
    static std::string tags[64];
    static std::mutex mu;
    int dev = 0;
    cudaGetDevice(&dev);
    dev &= 63;
    std::lock_guard<std::mutex> lk(mu);
    if (tags[dev].empty()) {
        cudaDeviceProp p;
        if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) {
            tags[dev] = "unknown";
        } else {
            std::string s = p.name;
            for (char& c : s)
                if (c == ' ' || c == '"') c = '_';
            tags[dev] = s + "_sm" + std::to_string(p.multiProcessorCount);
        }
    }
    return tags[dev];
}

// Cache file: one JSON object per line, either a scan shape
// {"device": "...", "s_class": N, "n_class": N, "threads": N, "interleave": N, "hot": N, "stride": N,
//  "chunks_per_lane": N, "ms": F}
// (lines without "chunks_per_lane" are read as one chunk per lane) or a batch chunk
// {"device": "...", "s_class": N, "n_class": N, "batch_chunk": N, "ms": F}.
void load_file_locked() {
    if (g_loaded) return;
    g_loaded = true;
    const char* path = std::getenv("AC_TUNE_CACHE");
    if (!path) return;
    FILE* f = std::fopen(path, "r");
    if (!f) return;
    char line[512], dev[256];
    while (std::fgets(line, sizeof line, f)) {
        unsigned sc, nc, th, il, hot, stride, cpl = 1, chunk;
        float ms;
        if (std::sscanf(line, " {\"device\": \"%255[^\"]\", \"s_class\": %u, \"n_class\": %u, \"batch_chunk\": %u, "
                              "\"ms\": %f}",
                        dev, &sc, &nc, &chunk, &ms) == 5) {
            if (chunk) g_batch[Key{dev, sc, nc}] = BatchEntry{chunk, ms};
            continue;
        }
        const int got = std::sscanf(line,
                                    " {\"device\": \"%255[^\"]\", \"s_class\": %u, \"n_class\": %u, \"threads\": %u, "
                                    "\"interleave\": %u, \"hot\": %u, \"stride\": %u, \"chunks_per_lane\": %u, "
                                    "\"ms\": %f}",
                                    dev, &sc, &nc, &th, &il, &hot, &stride, &cpl, &ms);
        if (got == 9) {
            g_cache[Key{dev, sc, nc}] = Entry{th, il, hot, stride, cpl ? cpl : 1u, ms};
        } else if (std::sscanf(line,
                               " {\"device\": \"%255[^\"]\", \"s_class\": %u, \"n_class\": %u, \"threads\": %u, "
                               "\"interleave\": %u, \"hot\": %u, \"stride\": %u, \"ms\": %f}",
                               dev, &sc, &nc, &th, &il, &hot, &stride, &ms) == 8) {
            g_cache[Key{dev, sc, nc}] = Entry{th, il, hot, stride, 1u, ms};
        }
    }
    std::fclose(f);
}

void append_file(const Key& k, const Entry& e) {
    const char* path = std::getenv("AC_TUNE_CACHE");
    if (!path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f,
                 "{\"device\": \"%s\", \"s_class\": %u, \"n_class\": %u, \"threads\": %u, \"interleave\": %u, "
                 "\"hot\": %u, \"stride\": %u, \"chunks_per_lane\": %u, \"ms\": %.6f}\n",
                 std::get<0>(k).c_str(), std::get<1>(k), std::get<2>(k), e.threads, e.interleave, e.hot, e.stride,
                 e.cpl, e.ms);
    std::fclose(f);
}

void append_batch_file(const Key& k, const BatchEntry& e) {
    const char* path = std::getenv("AC_TUNE_CACHE");
    if (!path) return;
    FILE* f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "{\"device\": \"%s\", \"s_class\": %u, \"n_class\": %u, \"batch_chunk\": %u, \"ms\": %.6f}\n",
                 std::get<0>(k).c_str(), std::get<1>(k), std::get<2>(k), e.chunk, e.ms);
    std::fclose(f);
}

void fill_opts(const Entry& e, ac_scan_opts* o) {
    o->threads = e.threads;
    o->interleave = e.interleave;
    o->hot_states = (int32_t)e.hot;
    o->stride = e.stride;
    o->chunks_per_lane = e.cpl;
}

bool tuning_off() {
    const char* v = std::getenv("AC_TUNE");
    return v && (std::strcmp(v, "off") == 0 || std::strcmp(v, "0") == 0);
}

}  // namespace

bool ac_tuned_lookup(const ac_dfa* dfa, uint64_t n, ScanShape* out) {
    std::lock_guard<std::mutex> lk(g_mu);
    load_file_locked();
    const Entry* e = nullptr;
    auto it = g_cache.find(Key{device_tag(), size_class(dfa->host.n_states), size_class(n)});
    if (it != g_cache.end()) {
        e = &it->second;
    } else {
        // no shape tuned for this machine size and text size: the shape last
        // tuned for this very machine (on another text size) if there is one
        auto jt = g_by_dfa.find(dfa->serial);
        if (jt != g_by_dfa.end()) e = &jt->second;
    }
    if (!e) return false;
    out->threads = e->threads;
    out->interleave = e->interleave;
    out->hot = e->hot;
    out->stride = e->stride;
    out->cpl = e->cpl;
    out->chunk = 0;
    return true;
}

bool ac_tuned_batch_chunk(const ac_dfa* dfa, uint64_t total, uint32_t* chunk) {
    std::lock_guard<std::mutex> lk(g_mu);
    load_file_locked();
    auto it = g_batch.find(Key{device_tag(), size_class(dfa->host.n_states), size_class(total)});
    if (it == g_batch.end()) return false;
    *chunk = it->second.chunk;
    return true;
}

namespace {

// Timed repetitions of a candidate after one untimed run: two, or eight when
// the run is short (below 0.5 ms launch noise decides between close shapes).
int timed_reps(float first_ms) { return first_ms < 0.5f ? 8 : 2; }

// Time of one candidate: the fastest of its timed scans after one untimed.
int time_scan(const ac_dfa* dfa, const ac_text* sample, const ac_scan_opts& o, ac_match* d_m, uint64_t cap,
              void* stream, float* ms, uint32_t* chunk) {
    float t_best = 1e30f;
    int reps = 3;
    for (int rep = 0; rep < reps; ++rep) {
        ac_result r;
        std::memset(&r, 0, sizeof r);
        r.matches = d_m;
        r.capacity = cap;
        r.on_device = 1;
        ac_scan_stats stt;
        const int s = ac_scan(dfa, sample, &r, &o, stream, &stt);
        if (s != AC_OK && s != AC_ERR_OVERFLOW) return s;
        if (rep == 0) reps = 1 + timed_reps(stt.scan_ms);
        if (rep > 0) t_best = std::min(t_best, stt.scan_ms);
        if (chunk) *chunk = stt.chunk;
    }
    *ms = t_best;
    return AC_OK;
}

// Room for every occurrence of a sample (one counting pass), at most half of the free device memory.
int size_output(const ac_dfa* dfa, const ac_text* texts, uint32_t n_texts, bool batch, void* stream, uint64_t* cap) {
    ac_result r0;
    std::memset(&r0, 0, sizeof r0);
    r0.on_device = 1;
    const int s0 = batch ? ac_scan_batch(dfa, texts, n_texts, &r0, nullptr, stream, nullptr)
                         : ac_scan(dfa, texts, &r0, nullptr, stream, nullptr);
    if (s0 != AC_OK && s0 != AC_ERR_OVERFLOW) return s0;
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    *cap = std::min<uint64_t>(r0.n_matches + 1024, free_b / 2 / sizeof(ac_match));
    return AC_OK;
}

}  // namespace

extern "C" int ac_autotune(const ac_dfa* dfa, const ac_text* sample, ac_scan_opts* best, void* stream) {
    AcRange trace_("ac_autotune");
    if (!dfa || !sample || !best) return AC_ERR_INVALID_ARG;
    if (!dfa->on_device) return AC_ERR_NO_DEVICE;
    if (!sample->on_device || sample->encoding != AC_TEXT_PACKED2) return AC_ERR_INVALID_ARG;
    const uint64_t n = sample->n_bases;
    std::memset(best, 0, sizeof *best);
    best->hot_states = -1;
    const Key key{device_tag(), size_class(dfa->host.n_states), size_class(n)};
    auto report_chunk = [&] {  // the chunk length the shape gives for this text
        best->chunk = ac_default_shape(dfa, n, best).chunk;
    };
    {
        std::unique_lock<std::mutex> lk(g_mu);
        load_file_locked();
        auto it = g_cache.find(key);
        if (it != g_cache.end()) {
            g_by_dfa[dfa->serial] = it->second;
            fill_opts(it->second, best);
            lk.unlock();
            report_chunk();
            return AC_OK;
        }
    }
    const uint32_t S = dfa->host.n_states;
    if (tuning_off() || n == 0) {  // the built-in default shape
        ScanShape sh = ac_default_shape(dfa, n, nullptr);
        best->interleave = sh.interleave;
        best->threads = sh.threads;
        best->hot_states = (int32_t)sh.hot;
        best->stride = sh.stride;
        best->chunks_per_lane = sh.cpl;
        best->chunk = sh.chunk;
        return AC_OK;
    }
    // size the occurrence buffer with one counting pass, so every trial writes
    // all of its occurrences (emission costs what it costs in real use)
    uint64_t cap = 0;
    int rc = size_output(dfa, sample, 1, false, stream, &cap);
    if (rc != AC_OK) return rc;
    ac_match* d_m = nullptr;
    if (ac_dev_alloc((void**)&d_m, std::max<uint64_t>(cap, 1) * sizeof(ac_match)) != cudaSuccess) return AC_ERR_OOM;

    const uint32_t threads_c[] = {256, 512, 0, 768, 1024};  // 0: the two-blocks-per-SM build's size, if any
    const uint32_t inter_c[] = {1, 2, 4, 8};
    const uint32_t frac_c[] = {0, 1, 2, 4};  // shared-memory states: none, 1/4, 1/2, all that fit
    const uint32_t cpl_c[] = {2, 4, 8};      // chunks per lane tried on the fastest shape
    Entry top{0, 0, 0, 0, 1, 1e30f};
    const char* vb = std::getenv("AC_TUNE_VERBOSE");
    const bool verbose = vb && vb[0] == '1';
    for (uint32_t sd = 1; sd <= 3 && rc == AC_OK; ++sd)
        for (uint32_t fr : frac_c)
            for (uint32_t th0 : threads_c)
                for (uint32_t il : inter_c) {
                    if (rc != AC_OK) break;
                    if ((sd == 2 && !dfa->d_delta2) || (sd == 3 && !dfa->d_delta3)) continue;  // table not built
                    const uint32_t th = th0 ? th0 : ac_wide_threads(il, sd);
                    if (th == 0) continue;
                    if (th > ac_max_threads(il, sd) || !ac_shape_compiled(il, sd)) continue;
                    const uint32_t hot = std::min(S, ac_max_hot_states(th, sd) * fr / 4);
                    if (fr && fr < 4 && hot >= S) continue;  // same as "all" for small machines
                    ScanShape probe;
                    probe.threads = th;
                    probe.interleave = il;
                    probe.hot = hot;
                    probe.stride = sd;
                    if (ac_blocks_per_sm(probe, dfa->host.s3_rows >= S) == 0) continue;  // does not fit
                    const Entry e{th, il, hot, sd, 1u, 0.f};
                    ac_scan_opts o;
                    std::memset(&o, 0, sizeof o);
                    fill_opts(e, &o);
                    float ms = 0.f;
                    rc = time_scan(dfa, sample, o, d_m, cap, stream, &ms, nullptr);
                    if (rc != AC_OK) break;
                    if (verbose)
                        std::fprintf(stderr, "[ac_autotune] stride=%u threads=%u interleave=%u hot=%u: %.4f ms\n", sd,
                                     th, il, hot, ms);
                    if (ms < top.ms) top = Entry{th, il, hot, sd, 1u, ms};
                }
    if (rc == AC_OK && top.threads) {  // the chunk length: more, shorter chunks per lane on the fastest shape
        const Entry base = top;
        for (uint32_t cpl : cpl_c) {
            Entry e = base;
            e.cpl = cpl;
            ac_scan_opts o;
            std::memset(&o, 0, sizeof o);
            fill_opts(e, &o);
            float ms = 0.f;
            uint32_t chunk = 0;
            rc = time_scan(dfa, sample, o, d_m, cap, stream, &ms, &chunk);
            if (rc != AC_OK) break;
            if (verbose)
                std::fprintf(stderr, "[ac_autotune] chunks per lane %u (chunk %u): %.4f ms\n", cpl, chunk, ms);
            if (ms < top.ms) {
                e.ms = ms;
                top = e;
            }
        }
    }
    ac_dev_free(d_m);
    if (rc != AC_OK) return rc;
    if (top.threads == 0) return AC_ERR_CUDA;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_cache[key] = top;
        g_by_dfa[dfa->serial] = top;
        append_file(key, top);
    }
    fill_opts(top, best);
    report_chunk();
    return AC_OK;
}

extern "C" int ac_autotune_batch(const ac_dfa* dfa, const ac_text* texts, uint32_t n_texts, ac_scan_opts* best,
                                 void* stream) {
    AcRange trace_("ac_autotune_batch");
    if (!dfa || !best || (n_texts && !texts)) return AC_ERR_INVALID_ARG;
    if (!dfa->on_device) return AC_ERR_NO_DEVICE;
    uint64_t total = 0;
    for (uint32_t i = 0; i < n_texts; ++i) {
        if (!texts[i].on_device || texts[i].encoding != AC_TEXT_PACKED2) return AC_ERR_INVALID_ARG;
        total += texts[i].n_bases;
    }
    std::memset(best, 0, sizeof *best);
    best->hot_states = -1;
    const Key key{device_tag(), size_class(dfa->host.n_states), size_class(total)};
    {
        std::lock_guard<std::mutex> lk(g_mu);
        load_file_locked();
        auto it = g_batch.find(key);
        if (it != g_batch.end()) {
            best->chunk = it->second.chunk;
            return AC_OK;
        }
    }
    if (tuning_off() || total == 0) return AC_OK;  // chunk 0: the built-in default
    uint64_t cap = 0;
    int rc = size_output(dfa, texts, n_texts, true, stream, &cap);
    if (rc != AC_OK) return rc;
    ac_match* d_m = nullptr;
    if (ac_dev_alloc((void**)&d_m, std::max<uint64_t>(cap, 1) * sizeof(ac_match)) != cudaSuccess) return AC_ERR_OOM;
    const uint32_t halo = dfa->host.max_len ? dfa->host.max_len - 1 : 0;
    const uint32_t unit = std::max<uint32_t>(64, (halo + 63) / 64 * 64);
    std::vector<uint32_t> cands = {0};  // 0: the built-in default
    for (uint32_t m = 1; m <= 32; m *= 2) cands.push_back(unit * m);
    BatchEntry top{0, 1e30f};
    const char* vb = std::getenv("AC_TUNE_VERBOSE");
    const bool verbose = vb && vb[0] == '1';
    for (uint32_t c : cands) {
        ac_scan_opts o;
        std::memset(&o, 0, sizeof o);
        o.hot_states = -1;
        o.chunk = c;
        float t_best = 1e30f;
        uint32_t used = c;
        int reps = 3;
        for (int rep = 0; rep < reps && rc == AC_OK; ++rep) {
            ac_result r;
            std::memset(&r, 0, sizeof r);
            r.matches = d_m;
            r.capacity = cap;
            r.on_device = 1;
            ac_scan_stats stt;
            const int s = ac_scan_batch(dfa, texts, n_texts, &r, &o, stream, &stt);
            if (s != AC_OK && s != AC_ERR_OVERFLOW) rc = s;
            if (rep == 0) reps = 1 + timed_reps(stt.scan_ms);
            if (rep > 0) t_best = std::min(t_best, stt.scan_ms);
            used = stt.chunk;
        }
        if (rc != AC_OK) break;
        if (verbose) std::fprintf(stderr, "[ac_autotune_batch] chunk %u: %.4f ms\n", used, t_best);
        if (t_best < top.ms) top = BatchEntry{used, t_best};
    }
    ac_dev_free(d_m);
    if (rc != AC_OK) return rc;
    {
        std::lock_guard<std::mutex> lk(g_mu);
        g_batch[key] = top;
        append_batch_file(key, top);
    }
    best->chunk = top.chunk;
    return AC_OK;
}
