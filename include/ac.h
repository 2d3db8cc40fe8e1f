/*
 * ac.h - C-ABI of the GB300 Aho-Corasick DNA scan (libac.so).
 *
 * The problem statement follows the paper (Sec. IV.B, the matching module it
 * builds on): given an array of keyword strings and a text, report every
 * keyword occurrence and its position; Aho-Corasick does this in a single
 * pass over the text (Sec. I, Sec. III.A). The machine is built in two
 * stages (Sec. III.A): the goto/failure/output machine from the keywords,
 * then one pass over the text. This library flattens the machine into a full
 * deterministic transition table over {A,C,G,T} (the failure transitions are
 * folded in at build time, so the scan takes exactly one table lookup per
 * base) and runs the pass on the GPU.
 *
 * Conventions (the paper leaves them open):
 *   - an occurrence is (start, pattern_id, text_id); start is the 0-based
 *     offset of the keyword's first base; pattern_id is the 0-based index in
 *     the caller's keyword array; duplicate keywords are separate ids and are
 *     all reported; overlapping occurrences are all reported (Fig. 2);
 *   - the alphabet is exactly A, C, G, T (lower case only with
 *     AC_BUILD_FOLD_CASE / AC_SCAN_FOLD_CASE); any other byte is an error;
 *   - occurrences come out in no particular order; (text_id, start,
 *     pattern_id) is unique, so a sort on that key gives the canonical form.
 *
 * General rules for every call:
 *   - every call returns an ac_status (0 = AC_OK, negative = error) and never
 *     throws across the ABI; ac_status_str() names the code;
 *   - "device pointer" means memory of the current CUDA device; "host
 *     pointer" means ordinary (pageable or pinned) host memory;
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream); work is enqueued on it; calls that must return a count
 *     synchronise that stream only;
 *   - the library owns ac_dfa and ac_server objects; the caller owns every
 *     text and result buffer it passes in and keeps it alive for the call;
 *   - an ac_dfa is immutable after ac_build, so concurrent scans of one
 *     ac_dfa from several host threads / streams are safe;
 *   - a text (or a streamed piece, or one text of a batch) has fewer than
 *     2^56 bases; a longer one is refused with AC_ERR_TOO_LARGE.
 */
#ifndef AC_H
#define AC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------ status */

enum ac_status_code {
    AC_OK = 0,
    AC_ERR_INVALID_ARG = -1,   /* NULL pointer, bad size, misaligned buffer, bad option      */
    AC_ERR_ALPHABET = -2,      /* a byte outside {A,C,G,T}; ac_result.bad_offset says where  */
    AC_ERR_EMPTY_PATTERN = -3, /* a keyword of length 0                                      */
    AC_ERR_TOO_LARGE = -4,     /* machine or text beyond the documented limits               */
    AC_ERR_OOM = -5,           /* host or device allocation failed (nothing leaked)          */
    AC_ERR_OVERFLOW = -6,      /* more occurrences than ac_result.capacity; n_matches and
                                  counts are still exact, matches[0..capacity) valid          */
    AC_ERR_CUDA = -7,          /* a CUDA runtime call failed                                 */
    AC_ERR_TIMEOUT = -8,       /* a bounded wait ran out (serving)                           */
    AC_ERR_BUSY = -9,          /* serving admission refused (over the device budget)         */
    AC_ERR_NOT_FOUND = -10,    /* unknown ticket / slot                                      */
    AC_ERR_NO_DEVICE = -11     /* the object lives on the host only (AC_BUILD_HOST_ONLY)     */
};

const char* ac_status_str(int status);

/* ------------------------------------------------------------------ machine */

typedef struct ac_dfa ac_dfa;

enum ac_build_flags {
    AC_BUILD_FOLD_CASE = 1u, /* accept a,c,g,t in keywords as A,C,G,T                          */
    AC_BUILD_HOST_ONLY = 2u, /* build the tables on the host only (no GPU needed); such a dfa
                                can be inspected with ac_dfa_tables but not scanned          */
    AC_BUILD_NO_STRIDE2 = 4u, /* skip the two-bases-per-lookup table (saves 64 B per state of
                                device memory; scans then always read one base per lookup)   */
    AC_BUILD_FAILURELESS = 8u, /* also keep the trie edges and per-state own keywords, for
                                ac_scan_failureless (16 B per state + 8 B per keyword)        */
    AC_BUILD_NO_STRIDE3 = 16u /* skip the three-bases-per-lookup table (256 B per row)          */
};

typedef struct {
    uint32_t flags;          /* ac_build_flags                                           */
    uint32_t stride2_states; /* rows of the two-base table: the first (breadth-first, i.e.
                                shallowest) this many states; 0 = every state, up to 2^24.
                                Steps from deeper states take two one-base lookups.       */
    uint32_t stride3_states; /* rows of the three-base table, likewise; 0 = min(S, 2^21)
                                (every state of machines up to 2^21 states); at most 2^22.
                                Three-base steps from deeper states take a two-base or a
                                one-base lookup instead.                                  */
} ac_build_opts;

/*
 * ac_build - stage 1 of Sec. III.A: build the pattern matching machine.
 *
 * patterns[i] points to lens[i] bytes (not NUL-terminated) of keyword i, for
 * i < n_patterns. All host memory, read only during the call.
 * Builds goto (a trie), failure (breadth first) and output (own keywords
 * plus the output of the failure state), then the full transition table
 * delta[s][c], c in {A=0,C=1,G=2,T=3}, with states renumbered breadth first
 * (so shallow, frequently visited states have small ids). Unless
 * AC_BUILD_NO_STRIDE2 is set it also builds delta2[s][x | y<<2] =
 * delta[delta[s][x]][y] for the shallowest opts->stride2_states states, which
 * lets a scan read two bases per lookup, and unless AC_BUILD_NO_STRIDE3 is set
 * delta3[s][x | y<<2 | z<<4] (three bases) for the shallowest
 * opts->stride3_states states. Unless AC_BUILD_HOST_ONLY is set the
 * tables are copied to the current device (synchronously) and the dfa is
 * ready to scan.
 * Errors: AC_ERR_INVALID_ARG (NULL pointers, n_patterns == 0),
 * AC_ERR_EMPTY_PATTERN, AC_ERR_ALPHABET (*out untouched), AC_ERR_TOO_LARGE
 * (more than 2^27 states), AC_ERR_OOM, AC_ERR_CUDA.
 */
int ac_build(const char* const* patterns, const uint32_t* lens, uint32_t n_patterns,
             const ac_build_opts* opts /* nullable */, ac_dfa** out);

/* Frees the dfa and its device tables (synchronises the device first). NULL is a no-op. */
void ac_free(ac_dfa* dfa);

typedef struct {
    uint32_t n_states;     /* S                                                   */
    uint32_t n_patterns;   /* P                                                   */
    uint32_t max_len;      /* L_max: longest keyword                              */
    uint32_t min_len;      /* shortest keyword                                    */
    uint32_t max_depth;    /* deepest state (= max_len)                           */
    uint32_t on_device;    /* 1 when the tables are on the device                 */
    uint64_t table_bytes;  /* 16 * S: the transition table                        */
    uint64_t out_entries;  /* total size of all output sets                       */
    uint64_t device_bytes; /* all device memory held by the dfa                   */
    double build_ms;       /* host time of the build (construction + upload)      */
    uint64_t table2_bytes; /* 64 * rows of the two-base table, 0 if not built     */
    uint64_t table3_bytes; /* 256 * rows of the three-base table, 0 if not built  */
} ac_dfa_info_t;

int ac_dfa_info(const ac_dfa* dfa, ac_dfa_info_t* out);

/* Read-only views of the host copies of the tables (valid until ac_free).
 *   delta[4*s + c]: bits 0-30 the next state, bit 31 set when the next state
 *                   has a non-empty output set;
 *   out_off[S+1], out_pid[out_entries]: output set of s is
 *                   out_pid[out_off[s] .. out_off[s+1]);
 *   pat_len[P], pat_state[P]: keyword length and the state where it ends;
 *   depth[S]: distance of each state from the root;
 *   fail[S]: failure state of each state (breadth-first ids);
 *   delta2[16*s + (x | y<<2)] for s < table2_bytes/64 (NULL if not built):
 *                   bits 0-29 the state after bases x then y, bit 31 set when
 *                   that state has output, bit 30 set when the state after x
 *                   alone has output;
 *   delta3[64*s + (x | y<<2 | z<<4)] for s < table3_bytes/256 (NULL if not
 *                   built): bits 0-28 the state after bases x, y, z; bits 31,
 *                   30 and 29 set when the states after z, after y and after x
 *                   have output. */
typedef struct {
    const uint32_t* delta;
    const uint32_t* out_off;
    const uint32_t* out_pid;
    const uint32_t* pat_len;
    const uint32_t* pat_state;
    const uint32_t* depth;
    const uint32_t* fail;
    const uint32_t* delta2;
    /* failure-less form (NULL unless built with AC_BUILD_FAILURELESS):
     * gotos[4*s + c] = trie child (bit 31 set when keywords end there) or
     * 0x7fffffff where s has no c edge; own_off[S+1], own_pid[P]: the keywords
     * ending exactly at each state */
    const uint32_t* gotos;
    const uint32_t* own_off;
    const uint32_t* own_pid;
    const uint32_t* delta3;
} ac_dfa_tables_t;

int ac_dfa_tables(const ac_dfa* dfa, ac_dfa_tables_t* out);

/* ------------------------------------------------------------------- texts */

enum ac_encoding {
    AC_TEXT_ASCII = 0,  /* one byte per base, n_bases bytes                              */
    AC_TEXT_PACKED2 = 1 /* 2 bits per base, A=0 C=1 G=2 T=3, 16 bases per little-endian
                           uint32 word, base j in bits 2*(j%16).. of word j/16;
                           ceil(n_bases/16) words; the pointer must be 16-byte aligned   */
};

typedef struct {
    const void* data;  /* the bases, see ac_encoding (may be NULL when n_bases == 0)    */
    uint64_t n_bases;  /* number of bases                                                */
    int32_t encoding;  /* ac_encoding                                                    */
    int32_t on_device; /* 1: data is a device pointer, 0: host pointer                   */
} ac_text;

/* ------------------------------------------------------------------ results */

typedef struct {
    uint64_t pos;        /* 0-based start of the occurrence in its text             */
    uint32_t pattern_id; /* index into the keyword array given to ac_build          */
    uint32_t text_id;    /* ac_scan_opts.text_id, or the text's index in a batch    */
} ac_match;              /* 16 bytes */

typedef struct {
    ac_match* matches;   /* capacity entries, or NULL with capacity 0 (counts only);
                            in device memory it must be 16-byte aligned (else
                            AC_ERR_INVALID_ARG): occurrences are written as whole
                            16-byte records                                         */
    uint64_t capacity;   /* entries available at matches                            */
    uint64_t n_matches;  /* out: exact number of occurrences (also on overflow)      */
    uint64_t* counts;    /* [n_patterns] out: occurrences per keyword, or NULL       */
    int32_t on_device;   /* 1: matches/counts are device pointers, 0: host pointers  */
    int32_t reserved;
    uint64_t bad_offset; /* out: first invalid base on AC_ERR_ALPHABET, else ~0      */
} ac_result;

/* ------------------------------------------------------------------- scans */

enum ac_scan_flags {
    AC_SCAN_FOLD_CASE = 1u /* ASCII text: accept a,c,g,t as A,C,G,T */
};

typedef struct {
    uint64_t range_begin; /* owned end positions [range_begin, range_end): only
                             occurrences ending there are reported; the scan
                             reads max(0, range_begin - (L_max - 1)) onwards.   */
    uint64_t range_end;   /* 0 = n_bases                                        */
    uint32_t chunk;       /* bases owned per GPU chunk; 0 = tuned                */
    uint32_t threads;     /* threads per block (64..1024, multiple of 32); 0 = tuned */
    uint32_t interleave;  /* chunks walked per thread: 1, 2, 4 or 8; 0 = tuned  */
    int32_t hot_states;   /* states staged in shared memory: -1 = tuned,
                             0..S = exactly that many (breadth-first prefix)    */
    uint32_t flags;       /* ac_scan_flags                                      */
    uint32_t text_id;     /* copied into every ac_match.text_id (ac_scan only)  */
    uint32_t stride;      /* bases per table lookup: 1, 2 (needs the two-base
                             table), 3 (needs the three-base table), or 0 = tuned */
    uint32_t chunks_per_lane; /* when chunk is 0: the owned range is cut into
                             this many chunks per resident lane (1, 2, 4 or 8);
                             0 = tuned (1 when untuned)                         */
} ac_scan_opts;

/* Timing and launch shape of the last scan, filled when requested. */
typedef struct {
    float total_ms;      /* device time of the whole call (events on the stream)   */
    float scan_ms;       /* device time of the scan kernel                         */
    float pack_ms;       /* device time of the ASCII pack kernel (0 if packed)     */
    float counts_ms;     /* device time of the count kernel                        */
    uint32_t chunk, threads, interleave, hot_states, grid, blocks_per_sm;
    uint32_t stride;       /* bases per lookup used                                */
    uint32_t chunks_per_lane; /* chunks per resident lane the chunk length came from
                                 (0 when the chunk was given or fixed by a batch)  */
    uint64_t bases_walked; /* owned bases plus halo re-reads                       */
} ac_scan_stats;

/*
 * ac_pack - ASCII bases to the 2-bit packed encoding on the device (the
 * encoding step in front of the scan). ascii: device pointer to n bytes;
 * packed: device pointer to ceil(n/16) words, 16-byte aligned. Lower case is
 * accepted only with AC_SCAN_FOLD_CASE in flags. Synchronises the stream.
 * On a byte outside the alphabet returns AC_ERR_ALPHABET with *bad_offset =
 * the first such offset (else *bad_offset = ~0).
 */
int ac_pack(const uint8_t* ascii, uint64_t n, uint32_t* packed, uint32_t flags, uint64_t* bad_offset,
            void* stream);

/*
 * ac_scan - stage 2 of Sec. III.A over one text: one pass, every occurrence
 * whose end lies in the owned range (see ac_scan_opts) and per-keyword counts.
 *
 * Writes min(n_matches, capacity) occurrences to result->matches (any order)
 * and, if result->counts != NULL, the exact per-keyword counts. Texts and
 * results may be on the host or the device (flags in ac_text / ac_result);
 * host data is staged through stream-ordered device memory. When the text
 * and the results are both on the host, stats is NULL and the owned range
 * has at least 512 Mbase, the range is scanned in 256 Mbase pieces whose
 * host-to-device and device-to-host copies (on two library-owned streams,
 * ordered against `stream` by events) overlap the scans of neighbouring
 * pieces; the results are the same.
 * Synchronises `stream` once (to learn n_matches).
 * Errors: AC_ERR_INVALID_ARG, AC_ERR_NO_DEVICE, AC_ERR_ALPHABET (with
 * bad_offset), AC_ERR_OVERFLOW (n_matches and counts exact; retry with
 * capacity >= n_matches), AC_ERR_TOO_LARGE (2^56 bases or more), AC_ERR_OOM,
 * AC_ERR_CUDA.
 * stats (nullable) receives the launch shape and device times.
 */
int ac_scan(const ac_dfa* dfa, const ac_text* text, ac_result* result, const ac_scan_opts* opts /* nullable */,
            void* stream, ac_scan_stats* stats /* nullable */);

/*
 * ac_scan_batch - many independent texts in one persistent launch.
 *
 * texts[0..n_texts): each text is scanned on its own (no occurrence spans two
 * texts); ac_match.text_id is the text's index. Work is split into chunks of
 * every text and handed out to warps through a device work counter (work
 * stealing), so uneven lengths do not leave the GPU idle. counts are summed
 * over all texts. All texts must share one encoding and one location (host
 * or device). opts->range_* and opts->text_id are ignored.
 * Synchronises `stream` once. Errors as ac_scan.
 */
int ac_scan_batch(const ac_dfa* dfa, const ac_text* texts, uint32_t n_texts, ac_result* result,
                  const ac_scan_opts* opts /* nullable */, void* stream, ac_scan_stats* stats /* nullable */);

/* ------------------------------------------------------- no-allocation scan
 * The paper has no counterpart to this call. It exists for callers that
 * cannot allocate device memory at the moment they scan, for example a
 * process whose device memory is already held in full by another allocator
 * (a framework's caching pool that reserved the GPU up front), or a
 * latency-critical loop that must never enter an allocator. ac_scan takes
 * its scratch from the stream-ordered pool on every call; this call uses a
 * fixed scratch array compiled into the library instead and allocates
 * nothing.
 *
 * The scratch array holds AC_NOALLOC_MAX_STATES per-state hit counters plus
 * a 32-byte counter block (16 MiB + 32 B). It occupies device memory on
 * every GPU that loads the library, until the process exits, whether or not
 * this call is used.
 *
 * Same semantics as ac_scan, restricted to device-resident inputs/outputs:
 * text must be AC_TEXT_PACKED2 with on_device = 1; result->on_device must be
 * 1 (matches and counts in device memory). opts (nullable) as for ac_scan,
 * with the same checks: stride 2 or 3 needs the two- or three-base table.
 * Synchronises `stream` once to learn n_matches.
 *
 * The first call on a device looks up the device address of the scratch
 * array (once per device, with that device current); make that first call
 * before any stream capture. Every call shares the one array and clears the
 * part it uses before the scan, so calls that overlap on the GPU (several
 * streams or host threads at once) race and give undefined results:
 * serialise them.
 *
 * Errors: AC_ERR_TOO_LARGE when the dfa has more than AC_NOALLOC_MAX_STATES
 * states; AC_ERR_INVALID_ARG for host or ASCII texts, host results or bad
 * options; AC_ERR_NO_DEVICE; AC_ERR_OVERFLOW as ac_scan; AC_ERR_CUDA.
 */
#define AC_NOALLOC_MAX_STATES (1u << 21)

int ac_scan_noalloc(const ac_dfa* dfa, const ac_text* text, ac_result* result, const ac_scan_opts* opts /* nullable */,
                    void* stream);

/* ----------------------------------------------------- failure-less matching
 * The failure-less scheme the paper cites among related work (Sec. II, the
 * PFAC algorithm): one GPU thread per start position walks only the trie's
 * goto edges from the root, stops at the first missing edge, and reports the
 * keywords ending at each state it passes. Every occurrence is found by the
 * thread of its own start, so failure transitions are not needed. Same
 * results, buffers and errors as ac_scan (ownership by end position); needs a
 * dfa built with AC_BUILD_FAILURELESS, else AC_ERR_INVALID_ARG. Provided for
 * comparison with the failure-folded walk of ac_scan. */
int ac_scan_failureless(const ac_dfa* dfa, const ac_text* text, ac_result* result,
                        const ac_scan_opts* opts /* nullable */, void* stream, ac_scan_stats* stats /* nullable */);

/* --------------------------------------------------- partitioned keyword sets
 * The paper's own decomposition (Sec. IV.A, approach 2, Fig. 3): the keyword
 * list is cut into consecutive chunks, one machine is built per chunk, and
 * every machine scans the whole text; the union of their occurrences (ids
 * offset by the chunk's first keyword) is the single machine's result. Here
 * each chunk is sized so that its whole transition table fits in one block's
 * shared memory, and one launch runs all machines (one grid row each). */

typedef struct ac_part_set ac_part_set;

/* Arguments as ac_build. max_states: the most states one machine may have;
 * 0 = as many as one block can hold in shared memory on the current device.
 * Chunks are consecutive keyword ranges, closed greedily when the next
 * keyword would push the chunk's trie past max_states. Errors as ac_build;
 * AC_ERR_TOO_LARGE when one keyword alone needs more than max_states states. */
int ac_build_partitioned(const char* const* patterns, const uint32_t* lens, uint32_t n_patterns,
                         uint32_t max_states, const ac_build_opts* opts /* nullable */, ac_part_set** out);
/* Number of machines and the largest machine's state count. */
int ac_part_set_info(const ac_part_set* set, uint32_t* n_parts, uint32_t* max_states);
/* Scans one text with every machine of the set; semantics, buffers and
 * errors as ac_scan (pattern ids in the caller's numbering, counts summed
 * over machines). opts: range_begin/range_end, flags and text_id are used;
 * the launch shape is fixed (one machine per grid row, 1024 threads). */
int ac_scan_partitioned(const ac_part_set* set, const ac_text* text, ac_result* result,
                        const ac_scan_opts* opts /* nullable */, void* stream, ac_scan_stats* stats /* nullable */);
void ac_part_set_free(ac_part_set* set);

/* ---------------------------------------------------------- streaming scans
 * One long text delivered in consecutive pieces (for example read from a
 * file block by block: the paper's module reads both the keywords and the
 * input string from files, Sec. IV.B). Each ac_stream_scan reports the
 * occurrences whose END lies in that piece, with start positions counted
 * from the beginning of the whole text; an occurrence that spans a piece
 * boundary is reported once, by the piece that holds its end. The stream keeps
 * the last L_max - 1 bases on the device (the state at any position depends
 * on no more than that). Pieces may be of any length and encoding, host or
 * device, like ac_scan's text; counts cover the piece's occurrences.
 * Successive calls on one stream must be issued in order (same CUDA stream or
 * synchronised); a call that fails - AC_ERR_OVERFLOW included, which still
 * reports the exact n_matches and counts - leaves the stream unchanged, so the
 * piece can be sent again (with capacity >= n_matches). */

typedef struct ac_stream ac_stream;

int ac_stream_create(const ac_dfa* dfa, ac_stream** out);
/* Scans the next piece; opts->range_* are ignored. Errors as ac_scan; on
 * AC_ERR_ALPHABET bad_offset is relative to the piece. */
int ac_stream_scan(ac_stream* s, const ac_text* piece, ac_result* result, const ac_scan_opts* opts /* nullable */,
                   void* stream, ac_scan_stats* stats /* nullable */);
/* Forgets the carried bases: the next piece starts a new text at position 0. */
int ac_stream_reset(ac_stream* s);
void ac_stream_free(ac_stream* s);

/* -------------------------------------------------------------- batch plans
 * A batch plan fixes a set of device-resident packed texts and a dfa, and
 * captures the whole batched scan (counter reset, persistent scan, counts)
 * into one CUDA graph; ac_batch_plan_run replays it. This removes the
 * per-call host work and launch overhead for repeated batches. */

typedef struct ac_batch_plan ac_batch_plan;

/* texts: device-resident AC_TEXT_PACKED2 descriptors (host array of
 * descriptors, read during the call); result buffers must be device
 * pointers and stay valid while the plan lives. */
int ac_batch_plan_create(const ac_dfa* dfa, const ac_text* texts, uint32_t n_texts, ac_result* result,
                         const ac_scan_opts* opts /* nullable */, void* stream, ac_batch_plan** out);
/* Replays the graph on `stream`; when sync != 0 waits and fills
 * result->n_matches (and returns AC_ERR_OVERFLOW as ac_scan does). */
int ac_batch_plan_run(ac_batch_plan* plan, void* stream, int sync, ac_result* result);
void ac_batch_plan_free(ac_batch_plan* plan);

/* ---------------------------------------------------------------- autotune
 * Times candidate launch shapes (bases per lookup, threads, interleave,
 * shared-memory states, then chunks per lane for the best of those) on a
 * device-resident packed text and returns the fastest in *best (best->chunk
 * = the chunk length it gives for this text). Every trial writes all of its
 * occurrences. Results are cached per (device, dfa size class, text size
 * class), where a size class is ceil(log2(x)), for the life of the process
 * (and in the file AC_TUNE_CACHE names, if set); later scans whose classes
 * match use the tuned shape unless the caller fixes one. AC_TUNE=off skips
 * the trials and returns the built-in defaults. */
int ac_autotune(const ac_dfa* dfa, const ac_text* sample, ac_scan_opts* best, void* stream);

/* Tunes the chunk length of batched scans (ac_scan_batch, batch plans): the
 * work-stealing grain, in bases of one text per work item. Times
 * ac_scan_batch over texts (device-resident AC_TEXT_PACKED2) with candidate
 * chunks from the keyword halo rounded up to 64 bases up to 32 times that,
 * and the built-in default, in the launch shape ac_scan would use for the
 * batch's total length. Cached per (device, dfa size class, class of the
 * total bases); later batches whose classes match use the tuned chunk unless
 * opts->chunk is set. best->chunk is the chosen chunk. Errors as
 * ac_scan_batch. */
int ac_autotune_batch(const ac_dfa* dfa, const ac_text* texts, uint32_t n_texts, ac_scan_opts* best,
                      void* stream);

/* ----------------------------------------------------------------- serving
 * Continuous batching over several resident dfas. Requests (host texts) are
 * admitted while the device budget allows, grouped per dfa, and launched as
 * batched scans on a pool of streams while earlier work is still running;
 * completed requests are returned to their waiters. Every request's result
 * is exactly its stand-alone ac_scan result. */

typedef struct ac_server ac_server;

typedef struct {
    uint64_t device_budget_bytes; /* texts + outputs in flight (dfas not counted); 0 = 40 GB */
    uint32_t n_streams;           /* concurrent batches on the device; 0 = 4               */
    uint32_t max_batch;           /* requests per launched batch; 0 = 256                  */
    uint32_t max_queue;           /* waiting requests before submit returns BUSY; 0 = 1<<16 */
    uint32_t match_capacity_per_base_x1000; /* output reservation per request: n*d + 1024 with d the
                                               larger of x/1000 and twice the densest batch seen
                                               for that dfa (occurrences per base); 0 = 64 */
} ac_serve_opts;

typedef struct {
    uint64_t submitted, completed, rejected, failed;
    uint64_t bases_completed;
    uint64_t batches_launched;
    double p50_ms, p99_ms, mean_ms, max_ms; /* submit -> results on the host   */
    double busy_s;                          /* wall time with work in flight   */
    double gbases_per_s;                    /* bases_completed / busy_s / 1e9  */
    uint64_t overflow_batches;              /* batches that outgrew their output reservation
                                               and ran once more with the exact room        */
    uint64_t cancelled;                     /* requests cancelled before they ran           */
} ac_serve_stats_t;

int ac_serve_create(const ac_serve_opts* opts /* nullable */, ac_server** out);
/* Makes dfa selectable by *slot. The server does not own the dfa: keep it
 * alive until ac_serve_destroy. */
int ac_serve_add_dfa(ac_server* srv, const ac_dfa* dfa, uint32_t* slot);
/* Queues a scan of a HOST text (ASCII or packed) against dfa `slot`; the
 * bases are copied during the call, so the caller may reuse its buffer.
 * Returns AC_ERR_BUSY when the queue is full or the text alone exceeds the
 * device budget, AC_ERR_ALPHABET when an ASCII text holds a byte other than
 * A, C, G, T (checked while it is copied; nothing is queued). */
int ac_serve_submit(ac_server* srv, uint32_t slot, const ac_text* text, uint64_t* ticket);
/* Waits up to timeout_us (<0: forever) for a ticket. On completion copies
 * the occurrences (with text_id 0) and the counts into the HOST buffers of
 * result (on_device must be 0), sets n_matches, and forgets the ticket.
 * Returns AC_ERR_TIMEOUT if not done in time, or AC_ERR_OVERFLOW with
 * n_matches set when capacity is too small - in both cases the ticket stays
 * valid and the call can be repeated - or the request's own error. */
int ac_serve_wait(ac_server* srv, uint64_t ticket, ac_result* result, int64_t timeout_us);
/* A finished request's results, left where the server holds them. */
typedef struct {
    const ac_match* matches;  /* HOST, n_matches occurrences, text_id 0 */
    uint64_t n_matches;
    const uint64_t* counts;   /* HOST, n_counts per-keyword counts           */
    uint64_t n_counts;
    void* handle;             /* pass to ac_serve_release when done with both */
} ac_served;
/* Like ac_serve_wait, but without copying: on completion fills *out with
 * the request's own occurrences and counts, forgets the ticket, and keeps
 * that memory valid until ac_serve_release(out->handle) - also after
 * ac_serve_destroy. Returns AC_ERR_TIMEOUT (ticket kept) or the request's
 * own error (ticket forgotten, nothing to release). */
int ac_serve_take(ac_server* srv, uint64_t ticket, ac_served* out, int64_t timeout_us);
/* Gives back the memory of one ac_serve_take result (null: no-op). */
void ac_serve_release(void* handle);
/* Withdraws a request. One still waiting in the queue is removed and never
 * scanned, and its ticket is forgotten (AC_OK; it counts as cancelled). A
 * finished one that was not yet waited for has its results dropped and its
 * ticket forgotten (AC_OK). One whose batch is running on the device cannot be
 * withdrawn: AC_ERR_BUSY (the ticket stays valid; wait for it or cancel again
 * once it is done). AC_ERR_NOT_FOUND for an unknown ticket. */
int ac_serve_cancel(ac_server* srv, uint64_t ticket);
int ac_serve_stats(ac_server* srv, ac_serve_stats_t* out);
/* Finishes in-flight work, then frees everything. */
void ac_serve_destroy(ac_server* srv);

/* ------------------------------------------ fault injection and accounting
 * The paper has no counterpart to these two calls; they serve failure
 * testing and leak checks. Fault injection stays on the host: no injected
 * failure reaches the GPU.
 *
 * ac_fault_inject sets the process-wide fault plan, replacing any earlier
 * plan (and the AC_FAULT environment variable, which is read once, at the
 * library's first allocation or kernel launch, when no plan was set). spec is a
 * comma-separated list of
 *   "oom@k"       the k-th device allocation (k >= 1) of the library from now
 *                 on fails as if the device were full: the call that made it
 *                 returns AC_ERR_OOM (a serving request, its own error);
 *   "cuda_err@k"  the k-th kernel launch of the library from now on is not
 *                 made and reports a launch failure: the call returns
 *                 AC_ERR_CUDA.
 * NULL or "" clears the plan. Counting restarts at every call. Every call
 * that fails this way releases what it allocated (see ac_mem_usage).
 * Errors: AC_ERR_INVALID_ARG for a spec it cannot parse (the plan is kept).
 */
int ac_fault_inject(const char* spec);

typedef struct {
    uint64_t pool_used_bytes;     /* stream-ordered pool memory in use on the current device
                                     (per-call scratch of the library; also any other user of
                                     the device's default pool)                              */
    uint64_t pool_reserved_bytes; /* memory the device's default pool holds                  */
    uint64_t live_bytes;          /* device bytes held by the library's objects (dfa tables,
                                     streams, batch plans) on all devices                    */
    uint64_t live_allocations;    /* number of those allocations                             */
    uint64_t allocations_seen;    /* device allocations counted since the fault plan was set */
    uint64_t launches_seen;       /* kernel launches counted since the fault plan was set    */
} ac_mem_usage_t;

/* Fills *out (see ac_mem_usage_t). Errors: AC_ERR_INVALID_ARG, AC_ERR_CUDA. */
int ac_mem_usage(ac_mem_usage_t* out);

#ifdef __cplusplus
}
#endif

#endif /* AC_H */
