// ac_internal.h - shared between the translation units of libac.so only.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "../../include/ac.h"

// Transition entry: low bits next state, bit 31 "next state has output";
// in the two-base table bit 30 is "the state after the first base has output".
static constexpr uint32_t AC_FLAG = 0x80000000u;
static constexpr uint32_t AC_FLAG_MID = 0x40000000u;
static constexpr uint32_t AC_STATE_MASK = 0x3fffffffu;
static constexpr uint32_t AC_MAX_STATES = 1u << 27;          // 16 B rows stay below 2 GiB
static constexpr uint32_t AC_MAX_STATES_STRIDE2 = 1u << 24;  // 64 B rows stay below 1 GiB
// Two-base rows for every state by default: a lockstep warp then never waits
// for a lane's second dependent lookup (64 B per state).
static constexpr uint32_t AC_DEFAULT_STRIDE2_ROWS = 1u << 24;
// Three-base table: bit 29 "the state after the first base has output", bit
// 30 "after the second", bit 31 "after the third"; the state in bits 0-28.
static constexpr uint32_t AC_FLAG_MID1 = 0x20000000u;
static constexpr uint32_t AC_STATE_MASK3 = 0x1fffffffu;
// Three-base rows for every state of machines up to 2M states (512 MiB at most):
// with all states covered the three-base walk runs its lanes in lockstep.
static constexpr uint32_t AC_DEFAULT_STRIDE3_ROWS = 1u << 21;
static constexpr uint32_t AC_MAX_STATES_STRIDE3 = 1u << 22;    // 256 B rows stay at 1 GiB
// Texts are shorter than 2^56 bases: a queued hit keeps its end position in
// 56 bits and a tag in the top byte.
static constexpr uint64_t AC_MAX_BASES = 1ull << 56;

struct HostTables {
    uint32_t n_states = 0, n_patterns = 0, max_len = 0, min_len = 0, max_depth = 0;
    std::vector<uint32_t> delta;      // [S*4]
    std::vector<uint32_t> delta2;     // [s2_rows*16] two bases per lookup (empty if not built)
    uint32_t s2_rows = 0;             // states [0, s2_rows) have two-base rows
    std::vector<uint32_t> delta3;     // [s3_rows*64] three bases per lookup (empty if not built)
    uint32_t s3_rows = 0;             // states [0, s3_rows) have three-base rows
    std::vector<uint32_t> out_off;    // [S+1]
    std::vector<uint32_t> out_pid;    // [E]
    std::vector<uint32_t> pat_len;    // [P]
    std::vector<uint32_t> out_ent;    // [2E] {out_pid[k], pat_len[out_pid[k]]}: the device's output entries
    std::vector<uint32_t> pat_state;  // [P]
    std::vector<uint32_t> depth;      // [S]
    std::vector<uint32_t> fail;       // [S]
    // failure-less form (built on request): trie edges and the keywords ending at each state
    std::vector<uint32_t> gotos;      // [S*4] child | AC_FLAG (child has own keywords), or AC_NO_EDGE
    std::vector<uint32_t> own_off;    // [S+1]
    std::vector<uint32_t> own_pid;    // [P]
    std::vector<uint32_t> own_ent;    // [2P] {own_pid[j], pat_len[own_pid[j]]}
};
static constexpr uint32_t AC_NO_EDGE = 0x7fffffffu;

// Builds the flattened machine on the host. Returns an ac_status.
int ac_build_host(const char* const* patterns, const uint32_t* lens, uint32_t n, bool fold_case,
                  bool with_stride2, uint32_t stride2_states, bool with_stride3, uint32_t stride3_states,
                  bool with_failureless, HostTables* t, uint32_t* bad_pattern);

struct ac_dfa {
    HostTables host;
    bool on_device = false;
    int device = -1;
    // device tables
    uint32_t* d_delta = nullptr;
    uint32_t* d_delta2 = nullptr;  // null when the two-base table was not built
    uint32_t* d_delta3 = nullptr;  // null when the three-base table was not built
    uint32_t* d_out_off = nullptr;
    uint32_t* d_out_ent = nullptr;  // [2E] {keyword id, keyword length} per output entry
    uint32_t* d_gotos = nullptr;    // failure-less form (null unless built)
    uint32_t* d_own_off = nullptr;
    uint32_t* d_own_ent = nullptr;  // [2P] {keyword id, keyword length} per own entry
    uint64_t device_bytes = 0;
    double build_ms = 0.0;
    uint64_t serial = 0;  // unique per built dfa in this process (tuned-shape reuse)
};

// ------------------------------------------------------------ launch shapes

struct ScanShape {
    uint32_t stride = 0;      // bases per lookup: 1, 2 or 3
    uint32_t chunk = 0;       // owned bases per chunk
    uint32_t threads = 0;     // per block
    uint32_t interleave = 0;  // chunks per thread
    uint32_t hot = 0;         // states in shared memory
    uint32_t grid = 0;        // blocks
    uint32_t blocks_per_sm = 0;
    uint32_t cpl = 0;         // chunks per resident lane the chunk came from (0: given or fixed)
};

struct DeviceProps {
    int device = 0;
    int sms = 0;
    size_t smem_optin = 0;
    size_t l2 = 0;
};

const DeviceProps& ac_device_props();

// Kernel launchers (ac_kernels.cu). All return cudaError_t as int.
struct ScanArgs {
    const uint32_t* delta;
    const uint32_t* delta2;  // two-base table (stride 2 and 3)
    uint32_t s2_rows;        // states with a two-base row
    const uint32_t* delta3;  // three-base table (stride 3 only)
    uint32_t s3_rows;        // states with a three-base row
    const uint32_t* out_off;
    const uint2* out_ent;   // {keyword id, keyword length} per output entry
    uint32_t n_states;
    const uint32_t* text;   // packed words (16-byte aligned)
    uint64_t n;             // bases in the text
    uint64_t own_begin;     // owned end positions [own_begin, own_end)
    uint64_t own_end;
    uint32_t halo;          // L_max - 1
    uint32_t text_id;
    ac_match* matches;
    uint64_t capacity;
    unsigned long long* counter;  // [0] = occurrences
    unsigned long long* hits;     // [S] flagged steps per state
    uint64_t pos_offset;          // added to every reported start position
};

int ac_launch_pack(const uint8_t* ascii, uint64_t n, uint32_t* packed, bool fold,
                   unsigned long long* bad, void* stream);
int ac_launch_scan(const ScanArgs& a, const ScanShape& sh, void* stream);
// clear_hits: set every counter read back to 0 (hits must then be writable).
int ac_launch_counts(const uint32_t* out_off, const uint2* out_ent, uint32_t n_states,
                     const unsigned long long* hits, unsigned long long* counts, void* stream,
                     bool clear_hits = false);
// Copies n packed bases from base src_off of src to base dst_off of dst.
int ac_launch_splice(uint32_t* dst, uint64_t dst_off, const uint32_t* src, uint64_t src_off, uint64_t n,
                     void* stream);
// Largest block size the kernels are compiled for at a given interleave and
// stride (0 counts as 1).
uint32_t ac_max_threads(uint32_t interleave, uint32_t stride = 1);
// Whether kernels exist for an (interleave, stride) pair.
bool ac_shape_compiled(uint32_t interleave, uint32_t stride);
// Block size at or below which a shape runs the build with two blocks per SM
// and 48 registers a thread (three bases per lookup, interleave 1); 0 where
// there is no such build.
uint32_t ac_wide_threads(uint32_t interleave, uint32_t stride);
// Largest number of states a scan block of `threads` threads can stage in
// shared memory (next to its per-warp event queues); rows are 16 B at
// stride 1 and 64 B at stride 2.
uint32_t ac_max_hot_states(uint32_t threads, uint32_t stride);
// Dynamic shared memory of a scan block: hot rows plus event queues.
size_t ac_scan_smem_bytes(uint32_t hot, uint32_t threads, uint32_t stride);
// Resident blocks per SM for a shape (occupancy query of the kernel variant
// the launch runs: all_rows3 when every state has a three-base row); 0 on error.
uint32_t ac_blocks_per_sm(const ScanShape& sh, bool all_rows3);

// Batched scan (ac_kernels.cu)
struct BatchText {
    const uint32_t* words;  // packed, 16-byte aligned
    uint64_t n;             // bases
};
struct BatchArgs {
    const uint32_t* delta;
    const uint32_t* delta2;
    uint32_t s2_rows;
    const uint32_t* delta3;
    uint32_t s3_rows;
    const uint32_t* out_off;
    const uint2* out_ent;   // {keyword id, keyword length} per output entry
    uint32_t n_states;
    const BatchText* texts;         // [T] device
    const unsigned long long* item_prefix;  // [T+1] device: first work item of each text
    uint32_t n_texts;
    unsigned long long n_items;     // total chunks
    uint32_t chunk;
    uint32_t halo;
    ac_match* matches;
    uint64_t capacity;
    unsigned long long* counter;    // [0] occurrences, [1] work cursor
    unsigned long long* hits;
};
int ac_launch_batch(const BatchArgs& a, const ScanShape& sh, void* stream);

// Partitioned keyword sets (ac_kernels.cu): one machine per chunk of keywords.
struct PartDesc {
    const uint32_t* delta;     // [S*4], all rows staged in shared memory
    const uint32_t* out_off;
    const uint2* out_ent;      // {local keyword id, keyword length}
    unsigned long long* hits;  // [S] slice of the shared hit buffer
    uint32_t n_states;
    uint32_t pid_offset;       // first keyword id of the chunk
};
struct PartArgs {
    const PartDesc* parts;     // [n_parts] device
    const uint32_t* text;
    uint64_t n;
    uint64_t own_begin, own_end;
    uint32_t halo;             // longest keyword of all chunks - 1
    uint32_t max_states;       // largest machine (shared-memory rows)
    ac_match* matches;
    uint64_t capacity;
    unsigned long long* counter;
};
// Launches grid (grid_x, n_parts) x threads, interleave 1.
int ac_launch_part_scan(const PartArgs& a, uint32_t n_parts, uint32_t grid_x, uint32_t threads, uint32_t chunk,
                        void* stream);
// Failure-less matching (ac_kernels.cu): one lane per start position.
static constexpr uint32_t AC_STATE_MASK31 = 0x7fffffffu;
struct FlArgs {
    const uint32_t* gotos;    // [S*4] trie edges (AC_NO_EDGE where none), bit 31 = child has own keywords
    const uint32_t* own_off;  // [S+1]
    const uint2* own_ent;     // [P] {keyword id, keyword length}
    const uint32_t* text;
    uint64_t n;
    uint64_t own_begin, own_end;
    uint32_t halo;            // L_max - 1
    uint32_t text_id;
    ac_match* matches;
    uint64_t capacity;
    unsigned long long* counter;
    unsigned long long* hits;  // [S] own-keyword hits per state
};
int ac_launch_failureless(const FlArgs& a, uint32_t hot, void* stream);
// Serving (ac_kernels.cu): splits the nm occurrences of a batch of n_req
// requests (text_id = request index) per request on the device. n_per,
// cursor [n_req] and req_counts [n_req * n_patterns] must be zero on entry.
// Fills offs[0..n_req] (exclusive offsets of each request's range of out),
// out (text_id 0) and req_counts (each request's per-keyword counts).
int ac_launch_serve_split(const ac_match* in, uint64_t nm, uint32_t n_req, uint32_t n_patterns, ac_match* out,
                          unsigned long long* req_counts, unsigned long long* n_per, unsigned long long* offs,
                          unsigned long long* cursor, void* stream);
// Sets the batch kernel's shared-memory limit for a shape (call before graph capture).
int ac_prepare_batch(const ScanShape& sh);

// Device allocations of the library (ac_api.cu): every one goes through these
// so that host-side fault injection (ac_fault_inject) reaches it and
// ac_mem_usage can account for what the library holds. ac_dev_alloc /
// ac_dev_free are synchronous (cudaMalloc / cudaFree); ac_dev_alloc_async
// takes stream-ordered pool memory (release it with cudaFreeAsync).
cudaError_t ac_dev_alloc(void** p, size_t bytes);
void ac_dev_free(void* p);
cudaError_t ac_dev_alloc_async(void** p, size_t bytes, cudaStream_t st);
// True when the fault plan says this kernel launch is to fail (the caller
// then returns cudaErrorLaunchFailure without launching).
bool ac_fault_launch();

// Launch-shape options a scan accepts (threads, interleave, stride and their
// compiled combinations), and whether the dfa has the table a requested
// stride reads (ac_api.cu).
bool ac_valid_shape_opts(const ac_scan_opts* o);
bool ac_stride_tables_present(const ac_dfa* dfa, const ac_scan_opts* o);

// Default / tuned shape selection (ac_api.cu / ac_tune.cpp)
ScanShape ac_default_shape(const ac_dfa* dfa, uint64_t owned_bases, const ac_scan_opts* opts);
bool ac_tuned_lookup(const ac_dfa* dfa, uint64_t n, ScanShape* out);
// The chunk tuned for batches of this dfa size and total length, if any.
bool ac_tuned_batch_chunk(const ac_dfa* dfa, uint64_t total, uint32_t* chunk);
// Chunk length for `owned` bases cut into `cpl` chunks per lane over `lanes`
// lanes: at least 64 bases and at least the halo rounded up to 64.
uint32_t ac_chunk_for(uint64_t owned, uint64_t lanes, uint32_t cpl, uint32_t halo);
