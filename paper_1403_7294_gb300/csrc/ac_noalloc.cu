// ac_noalloc.cu - ac_scan_noalloc: a scan that allocates no device memory.
//
// ac_scan takes its scratch (one 64-bit hit counter per machine state and a
// small counter block) from the device's stream-ordered pool on every call.
// Some callers cannot allocate at the moment they scan: for example a process
// whose device memory has been handed in full to another allocator (a
// framework's caching pool that reserved the GPU up front), or a
// latency-critical loop that must not enter the allocator at all. For them
// this entry point uses one fixed scratch array compiled into the library
// instead. The array lives in device memory of every GPU that loads the
// library, from load until the process exits, whether or not it is used.
//
// The caller still passes the text and the result buffers (both in device
// memory). Scratch holds AC_NOALLOC_MAX_STATES hit counters plus a 4-word
// counter block, so machines with more states than that are refused.
#include <cuda_runtime.h>

#include <mutex>

#include "ac_internal.h"

namespace {
constexpr uint32_t kMaxStates = AC_NOALLOC_MAX_STATES;
constexpr uint32_t kCounterWords = 4;  // [0] occurrences [1] work cursor [2] bad offset [3] pad
}  // namespace

// The fixed scratch: counter block first, then one hit counter per state
// (16 MiB + 32 B).
static __device__ __align__(256) unsigned long long g_scratch[kCounterWords + kMaxStates];

namespace {

// Device address of g_scratch for each device, looked up once per device.
// In host code the symbol g_scratch is only a host-side stand-in for the
// device array; passing it to a kernel would fault or touch the wrong memory.
std::mutex g_mu;
unsigned long long* g_addr[64] = {};

int scratch_address(unsigned long long** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return AC_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) return AC_ERR_CUDA;
        g_addr[dev] = static_cast<unsigned long long*>(p);
    }
    *out = g_addr[dev];
    return AC_OK;
}

}  // namespace

extern "C" int ac_scan_noalloc(const ac_dfa* dfa, const ac_text* text, ac_result* r, const ac_scan_opts* opts,
                               void* stream) {
    if (!dfa || !text || !r) return AC_ERR_INVALID_ARG;
    r->bad_offset = ~0ull;
    if (!dfa->on_device) return AC_ERR_NO_DEVICE;
    if (text->encoding != AC_TEXT_PACKED2 || !text->on_device || !r->on_device) return AC_ERR_INVALID_ARG;
    if (text->n_bases && (!text->data || (reinterpret_cast<uintptr_t>(text->data) & 15))) return AC_ERR_INVALID_ARG;
    if (text->n_bases >= AC_MAX_BASES) return AC_ERR_TOO_LARGE;
    if (r->capacity && !r->matches) return AC_ERR_INVALID_ARG;
    if (r->on_device && (reinterpret_cast<uintptr_t>(r->matches) & 15)) return AC_ERR_INVALID_ARG;  // 16-byte records
    // the launch-shape options ac_scan accepts, and the table a requested stride reads
    if (!ac_valid_shape_opts(opts) || !ac_stride_tables_present(dfa, opts)) return AC_ERR_INVALID_ARG;
    const HostTables& h = dfa->host;
    if (h.n_states > kMaxStates) return AC_ERR_TOO_LARGE;  // the fixed scratch is too small
    const uint64_t n = text->n_bases;
    const uint64_t own_begin = opts ? opts->range_begin : 0;
    const uint64_t own_end = (opts && opts->range_end) ? opts->range_end : n;
    if (own_begin > own_end || own_end > n) return AC_ERR_INVALID_ARG;

    unsigned long long* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc != AC_OK) return rc;
    unsigned long long* ctr = scratch;
    unsigned long long* hits = scratch + kCounterWords;
    cudaStream_t st = (cudaStream_t)stream;
    // the array keeps the previous call's values: clear what this call counts
    if (cudaMemsetAsync(ctr, 0, kCounterWords * sizeof(unsigned long long), st) != cudaSuccess) return AC_ERR_CUDA;
    if (cudaMemsetAsync(hits, 0, (size_t)h.n_states * sizeof(unsigned long long), st) != cudaSuccess)
        return AC_ERR_CUDA;

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
    a.text = (const uint32_t*)text->data;
    a.n = n;
    a.own_begin = own_begin;
    a.own_end = own_end;
    a.halo = h.max_len - 1;
    a.text_id = opts ? opts->text_id : 0u;
    a.matches = r->matches;
    a.capacity = r->capacity;
    a.counter = ctr;
    a.hits = hits;
    a.pos_offset = 0;
    if (ac_launch_scan(a, sh, stream) != 0) return AC_ERR_CUDA;
    if (r->counts) {
        if (cudaMemsetAsync(r->counts, 0, (size_t)h.n_patterns * 8, st) != cudaSuccess) return AC_ERR_CUDA;
        if (ac_launch_counts(dfa->d_out_off, reinterpret_cast<const uint2*>(dfa->d_out_ent), h.n_states, hits,
                             (unsigned long long*)r->counts, stream) != 0)
            return AC_ERR_CUDA;
    }
    unsigned long long nm = 0;  // pageable 8-byte read; the stream is synchronised below
    if (cudaMemcpyAsync(&nm, ctr, sizeof nm, cudaMemcpyDeviceToHost, st) != cudaSuccess) return AC_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return AC_ERR_CUDA;
    r->n_matches = nm;
    return nm > r->capacity ? AC_ERR_OVERFLOW : AC_OK;
}
