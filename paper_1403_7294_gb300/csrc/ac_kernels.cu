// ac_kernels.cu - the GPU side of stage 2 of Sec. III.A: one pass of the
// text over the flattened transition table.
//
// Layout in device memory
//   delta    uint32[S][4]   row s = the 4 transitions of state s (16 B);
//                           low bits next state, bit 31 "next state has output"
//   delta2   uint32[R2][16] row s = the 16 two-base transitions (64 B);
//                           bit 31 "final state has output", bit 30 "state
//                           after the first base has output"
//   delta3   uint32[R3][64] row s = the 64 three-base transitions (256 B);
//                           bits 31 / 30 / 29 "the state after the third /
//                           second / first base has output"
//   out_off  uint32[S+1], out_ent uint2[E]: output(s) as CSR, each entry
//                          {keyword id, keyword length} (one 8-byte load gives
//                          an occurrence's id and start position)
//   text     uint32[ceil(n/16)] 2-bit packed, base j in bits 2*(j%16) of word j/16
//
// Work decomposition (the GPU form of the paper's "approach 1", Sec. IV.A):
// the owned range is cut into chunks of `chunk` end positions; a chunk that
// owns [lo, hi) walks from state 0 starting at a position <= lo - (L_max - 1)
// (rounded down to a 64-base boundary, so text loads are aligned uint4s).
// After reading position i the state is the longest suffix of text[..i] that
// is a trie node; its length is at most L_max, so a walk that started at or
// before i - (L_max - 1) is in the same state as a walk from the text start.
// Every keyword ending at i is in output(state at i), and an occurrence has
// one end position, so emitting only for ends in [lo, hi) reports every
// occurrence exactly once.
//
// Each thread walks `I` chunks at once (independent dependency chains: their
// table lookups are in flight together), reading one, two or three bases per
// lookup (walk_any: ST = 1, 2 in lockstep; 3 with lanes on their own
// schedules; 4 three bases in lockstep). States [0, hot) - the breadth-first
// prefix of the machine - can be staged in shared memory; the rest are read
// through L1/L2 with an evict-last policy, while the streamed text uses
// evict-first.
//
// Emission: a step whose entry has a flag set lands on a state with output.
// The warp votes; flagged, owned positions are appended to a per-warp event
// queue in shared memory (ballot + popc); a full queue of 64 events is
// drained: per event the output-set bounds and the per-state hit counts, one
// atomicAdd on the occurrence counter for the whole queue, then one
// occurrence per lane - consecutive lanes read consecutive output entries and
// write consecutive 16-byte occurrences (streaming stores). The per-state hit
// counters feed the exact per-keyword counts (kept exact on overflow).
#include <cuda_runtime.h>

#include <atomic>
#include <cstdint>
#include <map>
#include <mutex>
#include <tuple>

#include "ac_internal.h"

namespace {

constexpr unsigned FULL = 0xffffffffu;

__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

// A table entry, read from L2 under the given policy. With InL1 false the
// entry is not allocated in L1: a long chunk's walk spreads its rows over
// megabytes, so one SM almost never reads a row twice while it is in L1, and
// allocating them would push out the text lines and output entries that are
// read again (plain scans, measured: about 2% faster on the 3 Gbase genome and
// the 256 Mbase chromosome). The batch kernel keeps allocating them: its lanes
// restart from the root every few hundred bases, and without L1 its kernel on
// 4,096 short texts took about 5% longer.
template <bool InL1>
__device__ __forceinline__ uint32_t ld_table(const uint32_t* p, uint64_t pol) {
    uint32_t v;
    if constexpr (InL1)
        asm("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    else
        asm("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}

__device__ __forceinline__ uint4 ld_text4(const uint32_t* p, uint64_t pol) {
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
        : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
        : "l"(p), "l"(pol));
    return v;
}

// One text word through L1 (a lane's following words hit the same line), L2 evict-first.
__device__ __forceinline__ uint32_t ld_text1(const uint32_t* p, uint64_t pol) {
    uint32_t v;
    asm("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(p), "l"(pol));
    return v;
}

// 64 bases starting at word w (w % 4 == 0); words past the end read as 0.
__device__ __forceinline__ uint4 load_block(const uint32_t* text, uint64_t w, uint64_t nwords, uint64_t pol) {
    if (w + 4 <= nwords) return ld_text4(text + w, pol);
    uint4 v = make_uint4(0, 0, 0, 0);
    if (w + 0 < nwords) v.x = text[w + 0];
    if (w + 1 < nwords) v.y = text[w + 1];
    if (w + 2 < nwords) v.z = text[w + 2];
    return v;
}

// What the walk reads at every step.
struct Tables {
    const uint32_t* __restrict__ delta;
    const uint32_t* __restrict__ delta2;
    uint32_t s2_rows;  // states [0, s2_rows) have two-base rows
    const uint32_t* __restrict__ delta3;
    uint32_t s3_rows;   // states [0, s3_rows) have three-base rows
    uint32_t n_states;  // all states have three-base rows when s3_rows == n_states
};

// What drain() reads: one copy per block in shared memory, so the walk keeps
// none of these pointers in registers.
struct Emit {
    const uint32_t* delta;
    const uint32_t* delta2;
    uint32_t s2_rows;
    const uint32_t* out_off;
    const uint2* out_ent;  // {keyword id, keyword length} per output entry
    ac_match* matches;
    uint64_t capacity;
    unsigned long long* counter;
    unsigned long long* hits;
    uint64_t pos_offset;  // added to every reported start (streaming scans)
    uint32_t pid_offset;  // added to every reported keyword id (partitioned keyword sets)
};

// Fills a block's Emit record field by field (one thread; the caller's
// barrier publishes it).
__device__ __forceinline__ void set_emit(Emit& em, const uint32_t* delta, const uint32_t* delta2, uint32_t s2_rows,
                                         const uint32_t* out_off, const uint2* out_ent, ac_match* matches,
                                         uint64_t capacity, unsigned long long* counter, unsigned long long* hits,
                                         uint64_t pos_offset, uint32_t pid_offset) {
    em.delta = delta;
    em.delta2 = delta2;
    em.s2_rows = s2_rows;
    em.out_off = out_off;
    em.out_ent = out_ent;
    em.matches = matches;
    em.capacity = capacity;
    em.counter = counter;
    em.hits = hits;
    em.pos_offset = pos_offset;
    em.pid_offset = pid_offset;
}

// Hits wait in a per-warp queue in shared memory, 16 B per event:
// {end position bits 0-31, end position bits 32-55 | tag << 24, state, text
// id}. The tag gives the bases still to be read after `state` to reach the
// state whose output is reported: none (tag 0), or - for a keyword that
// ends inside a multi-base step - the step's first one or two bases (tag
// bits 0-1 the count, bits 2-3 and 4-5 the bases), queued with the state
// before the step; the drain resolves those with table lookups, so the walk
// never waits for them. Appending costs a ballot and a popc; the queue is
// expanded QCAP events at a time, so the occurrence counter sees one
// atomicAdd per QCAP hits.
constexpr int QCAP = 64;  // events per warp queue (larger queues make ptxas spill the walk)
constexpr int EPL = QCAP / 32;  // events each lane expands in drain()
static_assert(QCAP % 32 == 0, "whole events per lane");
__device__ __forceinline__ uint32_t tag1(uint32_t b0) { return 1u | (b0 << 2); }
__device__ __forceinline__ uint32_t tag2(uint32_t b0, uint32_t b1) { return 2u | (b0 << 2) | (b1 << 4); }

__device__ __forceinline__ uint32_t lanemask_lt() {
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

__device__ __forceinline__ uint32_t warp_inclusive_sum(uint32_t v, uint32_t lane) {
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t u = __shfl_up_sync(FULL, v, d);
        if (lane >= (uint32_t)d) v += u;
    }
    return v;
}

// Expands the n <= QCAP queued hits of this warp; called by all 32 lanes
// together, in two phases.
//   Per event (lane l takes events l, l + 32, ...): the lookups that resolve
//   a hit inside a multi-base step, the output-set bounds, the per-state hit
//   counts (lanes holding the same
//   state combine through __match_any_sync before one atomicAdd per distinct
//   state), a warp prefix sum of the set sizes and one atomicAdd on the
//   occurrence counter for the whole queue.
//   Per occurrence: the queue entries are rewritten as {end position, first
//   output entry, text id}; round r covers occurrence slots [32r, 32r + 32),
//   one per lane. Every queued state has output (its step was flagged), so
//   each event owns at least one slot and the event of a slot is the number
//   of events starting at or before it, less one: a bit per event start,
//   OR-reduced over the warp, and a popcount. Consecutive lanes then read
//   consecutive output entries and write consecutive occurrences.
__device__ __noinline__ void drain(uint4* q, uint32_t n, const Emit* em) {
    __syncwarp();
    const uint32_t lane = threadIdx.x & 31;
    uint4 ev[EPL];
    uint32_t st[EPL], o0[EPL], k[EPL], ex[EPL];
    bool valid[EPL];
#pragma unroll
    for (int h = 0; h < EPL; ++h) {
        const uint32_t i = 32u * h + lane;
        valid[h] = i < n;
        ev[h] = valid[h] ? q[i] : make_uint4(0, 0, 0xffffffffu, 0);
        st[h] = ev[h].z;
    }
#pragma unroll
    for (int h = 0; h < EPL; ++h) {  // hits inside a multi-base step: the state after its first one or two bases
        const uint32_t tag = ev[h].y >> 24;
        if (valid[h] && (tag & 3u)) {
            const uint32_t b0 = (tag >> 2) & 3u, b1 = (tag >> 4) & 3u;
            if ((tag & 3u) == 2u && st[h] < em->s2_rows) {
                st[h] = __ldg(em->delta2 + ((st[h] << 4) | b0 | (b1 << 2))) & AC_STATE_MASK;
            } else {
                st[h] = __ldg(em->delta + ((st[h] << 2) | b0)) & AC_STATE_MASK;
                if ((tag & 3u) == 2u) st[h] = __ldg(em->delta + ((st[h] << 2) | b1)) & AC_STATE_MASK;
            }
        }
    }
    const uint32_t* __restrict__ out_off = em->out_off;
#pragma unroll
    for (int h = 0; h < EPL; ++h) {
        o0[h] = valid[h] ? __ldg(out_off + st[h]) : 0u;
        k[h] = valid[h] ? __ldg(out_off + st[h] + 1) - o0[h] : 0u;
    }
    unsigned long long* hits = em->hits;
#pragma unroll
    for (int h = 0; h < EPL; ++h) {
        const uint32_t peers = __match_any_sync(FULL, st[h]);
        if (valid[h] && lane == (uint32_t)(__ffs(peers) - 1))
            atomicAdd(&hits[st[h]], (unsigned long long)__popc(peers));
    }
    uint32_t total = 0;
#pragma unroll
    for (int h = 0; h < EPL; ++h) {  // exclusive offsets, events in queue order
        const uint32_t in = warp_inclusive_sum(k[h], lane);
        ex[h] = total + in - k[h];
        total += __shfl_sync(FULL, in, 31);
    }
    unsigned long long base = 0;
    if (lane == 31 && total) base = atomicAdd(em->counter, (unsigned long long)total);
    base = __shfl_sync(FULL, base, 31);
#pragma unroll
    for (int h = 0; h < EPL; ++h)
        if (valid[h]) q[32u * h + lane] = make_uint4(ev[h].x, ev[h].y, o0[h], ev[h].w);
    __syncwarp();
    const uint64_t capacity = em->capacity;
    const uint64_t room = capacity > base ? capacity - base : 0ull;
    const uint32_t stored = (uint32_t)min((uint64_t)total, room);
    const uint32_t rounds = (uint32_t)(((uint64_t)stored + 31) >> 5);
    const uint2* __restrict__ out_ent = em->out_ent;
    ac_match* matches = em->matches;
    const uint64_t pos_offset = em->pos_offset;
    const uint32_t pid_offset = em->pid_offset;
    uint32_t started = 0;  // events starting before this round's first slot
    for (uint32_t r = 0; r < rounds; ++r) {
        const uint32_t r0 = r << 5;
        uint32_t bits = 0;
#pragma unroll
        for (int h = 0; h < EPL; ++h)
            if (k[h] && ex[h] >= r0 && ex[h] - r0 < 32u) bits |= 1u << (ex[h] - r0);
        const uint32_t starts = __reduce_or_sync(FULL, bits);
        const uint32_t e = started + __popc(starts & (0xffffffffu >> (31 - lane))) - 1;  // event of this lane's slot
        started += __popc(starts);
        uint32_t ex_e = 0;
#pragma unroll
        for (int h = 0; h < EPL; ++h) {
            const uint32_t v = __shfl_sync(FULL, ex[h], e & 31);
            if ((e >> 5) == (uint32_t)h) ex_e = v;
        }
        const uint32_t slot = r0 + lane;
        if (slot < stored) {
            const uint4 rec = q[e];
            const uint2 ent = __ldg(out_ent + rec.z + (slot - ex_e));
            const uint64_t pos = ((((uint64_t)(rec.y & 0xffffffu)) << 32) | rec.x) + 1 - ent.y + pos_offset;
            // streaming store: occurrences are written once and must not evict table rows from L2
            __stcs(reinterpret_cast<uint4*>(matches + base + slot),
                   make_uint4((uint32_t)pos, (uint32_t)(pos >> 32), ent.x + pid_offset, rec.w));
        }
    }
    __syncwarp();
}

// Appends the hits of one ballot (mask m, this lane's flag h) to the queue.
__device__ __forceinline__ void append(uint4* q, uint32_t& qn, uint32_t m, bool h, uint64_t end_pos, uint32_t tag,
                                       uint32_t st, uint32_t text_id, uint32_t lt, const Emit* em) {
    if (qn + __popc(m) > (uint32_t)QCAP) {
        drain(q, qn, em);
        qn = 0;
    }
    if (h) q[qn + __popc(m & lt)] = make_uint4((uint32_t)end_pos, (uint32_t)(end_pos >> 32) | (tag << 24), st, text_id);
    qn += __popc(m);
}

// One chain of the walk: a text, the first position read (a multiple of
// 64), and the owned end positions [start + lo, start + hi).
struct Chain {
    const uint32_t* text;
    uint64_t nwords;
    uint64_t start;
    uint32_t lo, hi;  // relative to start
    uint32_t text_id;
};

__device__ __forceinline__ void set_chain(Chain& c, const uint32_t* text, uint64_t nwords, uint32_t text_id,
                                          uint64_t lo, uint64_t hi, uint32_t halo) {
    c.text = text;
    c.nwords = nwords;
    c.text_id = text_id;
    c.start = (lo > halo ? lo - halo : 0ull) & ~63ull;
    c.lo = (uint32_t)(lo - c.start);
    c.hi = (uint32_t)(hi - c.start);
}

__device__ __forceinline__ void idle_chain(Chain& c, const uint32_t* text, uint64_t nwords, uint32_t text_id) {
    c.text = text;
    c.nwords = nwords;
    c.text_id = text_id;
    c.start = 0;
    c.lo = c.hi = 0;
}

// Threads per block each (interleave, stride) pair is compiled for (register
// budget).
template <int I, int ST = 1>
struct MaxThreads {  // ST 1-4 as in walk_any
    static constexpr int value = I == 1 ? 1024 : (I <= 4 ? 512 : 256);
};

// Launch bounds of a kernel build. W = 0: one block of up to MaxThreads per
// SM (no minimum asked of the compiler). W = 1, built for three bases per
// lookup with one chain per lane only: at least two blocks of up to
// kWideThreads per SM, so 48 registers a thread instead of 64 and 40 warps
// in flight instead of 32 to cover the L2 misses of the 256-byte rows.
constexpr uint32_t kWideThreads = 640;

template <int I, int ST, int W>
struct Bounds {
    static constexpr int threads = W == 0 ? MaxThreads<I, ST>::value : (int)kWideThreads;
    static constexpr int blocks = W == 0 ? 0 : 2;
};

// The build a launch of `threads` threads per block uses.
template <int I, int ST>
constexpr int wide_build(uint32_t threads) {
    return (I == 1 && ST >= 3 && threads <= kWideThreads) ? 1 : 0;
}

// Walk I chains in lockstep, ST bases per lookup (all 32 lanes of the warp
// call this together). q: this warp's event queue in shared memory.
template <int I, int ST, bool InL1>
__device__ __forceinline__ void walk(const Chain (&ch)[I], const uint32_t* __restrict__ sm, uint32_t hot,
                                     const Tables& tb, const Emit* em, uint4* q, uint64_t pol_tab, uint64_t pol_txt) {
    constexpr uint32_t ROW_SHIFT = ST == 1 ? 2 : 4;  // log2 entries per row
    constexpr uint32_t SYM_MASK = ST == 1 ? 3u : 15u;
    constexpr uint32_t FLAGS = ST == 1 ? AC_FLAG : (AC_FLAG | AC_FLAG_MID);
    const uint32_t* __restrict__ table = ST == 1 ? tb.delta : tb.delta2;
    uint32_t nb = 0;
#pragma unroll
    for (int j = 0; j < I; ++j) {
        const uint32_t b = (ch[j].hi + 63) >> 6;
        nb = b > nb ? b : nb;
    }
    nb = __reduce_max_sync(FULL, nb);
    const uint32_t lt = lanemask_lt();
    uint32_t s[I];
#pragma unroll
    for (int j = 0; j < I; ++j) s[j] = 0;
    uint32_t qn = 0;  // queued events (same value in every lane)

    for (uint32_t b = 0; b < nb; ++b) {
        uint4 buf[I];
        uint32_t fmask[I];
#pragma unroll
        for (int j = 0; j < I; ++j) {
            const bool act = 64u * b < ch[j].hi;
            fmask[j] = act ? FLAGS : 0u;
            buf[j] = act ? load_block(ch[j].text, (ch[j].start >> 4) + 4ull * b, ch[j].nwords, pol_txt)
                         : make_uint4(0, 0, 0, 0);
        }
#pragma unroll 1
        for (uint32_t wq = 0; wq < 4; ++wq) {
            uint32_t wd[I];
#pragma unroll
            for (int j = 0; j < I; ++j) {  // next 16 bases; shift the 64-base buffer down
                wd[j] = buf[j].x;
                buf[j].x = buf[j].y;
                buf[j].y = buf[j].z;
                buf[j].z = buf[j].w;
            }
#pragma unroll
            for (int k = 0; k < 16 / ST; ++k) {
                uint32_t e[I], sp[I];
#pragma unroll
                for (int j = 0; j < I; ++j) {
                    const uint32_t sym = (wd[j] >> (2 * ST * k)) & SYM_MASK;
                    const uint32_t idx = (s[j] << ROW_SHIFT) | sym;
                    if (ST == 1 || s[j] < tb.s2_rows) {
                        e[j] = (s[j] < hot) ? sm[idx] : ld_table<InL1>(table + idx, pol_tab);
                    } else {  // deep state without a two-base row: two one-base lookups
                        const uint32_t e1 = ld_table<InL1>(tb.delta + ((s[j] << 2) | (sym & 3u)), pol_tab);
                        const uint32_t e2 = ld_table<InL1>(tb.delta + (((e1 & AC_STATE_MASK) << 2) | (sym >> 2)), pol_tab);
                        e[j] = e2 | ((e1 & AC_FLAG) >> 1);  // bit 31: final state, bit 30: after the first base
                    }
                }
                uint32_t any = 0;
#pragma unroll
                for (int j = 0; j < I; ++j) {
                    sp[j] = s[j];
                    s[j] = e[j] & AC_STATE_MASK;
                    any |= e[j] & fmask[j];
                }
                if (__any_sync(FULL, any)) {
                    const uint32_t off = 64u * b + 16u * wq + ST * k;  // first base of this step
#pragma unroll
                    for (int j = 0; j < I; ++j) {
                        if (ST == 2) {  // a keyword may end at the first base of the pair
                            const bool hm = (e[j] & fmask[j] & AC_FLAG_MID) && off >= ch[j].lo && off < ch[j].hi;
                            const uint32_t mm = __ballot_sync(FULL, hm);
                            if (mm)
                                append(q, qn, mm, hm, ch[j].start + off, tag1((wd[j] >> (2 * ST * k)) & 3u), sp[j],
                                       ch[j].text_id, lt, em);
                        }
                        const uint32_t oe = off + ST - 1;  // last base of this step
                        const bool h = (e[j] & fmask[j] & AC_FLAG) && oe >= ch[j].lo && oe < ch[j].hi;
                        const uint32_t m = __ballot_sync(FULL, h);
                        if (m) append(q, qn, m, h, ch[j].start + oe, 0u, s[j], ch[j].text_id, lt, em);
                    }
                }
            }
        }
    }
    if (qn) drain(q, qn, em);
}

// Walk I chains three bases per lookup where the tables allow it, every lane
// on its own schedule: each iteration makes exactly one lookup per chain -
// three bases from a three-base row (states [0, s3_rows), from shared memory
// below `hot`), two from a two-base row ([s3_rows, s2_rows)) or one from the
// base table - so a lane in a deep state never holds the others up (steps in
// lockstep would wait for the warp's longest chain of dependent lookups).
// A lookup's entry has one flag per base entered (three-base rows: bits 29,
// 30, 31 after the first, second, third base; two-base rows: bits 30, 31).
// Each lane reads its text through a 64-base block, the next block already
// loading, into a bit buffer of the coming bases.
template <int I, bool InL1>
__device__ __forceinline__ void walk3_free(const Chain (&ch)[I], const uint32_t* __restrict__ sm, uint32_t hot,
                                           const Tables& tb, const Emit* em, uint4* q, uint64_t pol_tab,
                                           uint64_t pol_txt) {
    const uint32_t lt = lanemask_lt();
    uint32_t s[I], pos[I], nb[I], wi[I];
    uint64_t bits[I], nextw[I];
    uint4 cur[I], nxt[I];
#pragma unroll
    for (int j = 0; j < I; ++j) {
        s[j] = 0;
        pos[j] = 0;  // next base to read, relative to ch[j].start
        nb[j] = 0;   // bases in bits[j]
        wi[j] = 0;   // next word of cur[j]
        bits[j] = 0;
        const uint64_t w0 = ch[j].start >> 4;
        const bool live = ch[j].hi > 0;
        cur[j] = live ? load_block(ch[j].text, w0, ch[j].nwords, pol_txt) : make_uint4(0, 0, 0, 0);
        nxt[j] = live ? load_block(ch[j].text, w0 + 4, ch[j].nwords, pol_txt) : make_uint4(0, 0, 0, 0);
        nextw[j] = w0 + 8;
    }
    uint32_t qn = 0;  // queued events (same value in every lane)
    for (;;) {
        bool act[I];
        bool any_act = false;
#pragma unroll
        for (int j = 0; j < I; ++j) {
            act[j] = pos[j] < ch[j].hi;
            any_act |= act[j];
        }
        if (!__any_sync(FULL, any_act)) break;
        uint32_t e[I], k[I], sym[I];
#pragma unroll
        for (int j = 0; j < I; ++j) {
            if (act[j] && nb[j] < 3) {  // 16 more bases into the buffer
                if (wi[j] == 4) {
                    cur[j] = nxt[j];
                    nxt[j] = load_block(ch[j].text, nextw[j], ch[j].nwords, pol_txt);
                    nextw[j] += 4;
                    wi[j] = 0;
                }
                const uint32_t w = wi[j] == 0 ? cur[j].x : (wi[j] == 1 ? cur[j].y : (wi[j] == 2 ? cur[j].z : cur[j].w));
                bits[j] |= (uint64_t)w << (2 * nb[j]);
                nb[j] += 16;
                ++wi[j];
            }
            const uint32_t cs = s[j];
            sym[j] = (uint32_t)bits[j] & 63u;
            const uint32_t* tab;
            uint32_t idx;
            if (cs < tb.s3_rows) {
                k[j] = 3;
                idx = (cs << 6) | sym[j];
                tab = tb.delta3;
            } else if (cs < tb.s2_rows) {
                k[j] = 2;
                idx = (cs << 4) | (sym[j] & 15u);
                tab = tb.delta2;
            } else {
                k[j] = 1;
                idx = (cs << 2) | (sym[j] & 3u);
                tab = tb.delta;
            }
            e[j] = act[j] ? ((cs < hot) ? sm[idx] : ld_table<InL1>(tab + idx, pol_tab)) : 0u;
        }
        uint32_t any = 0, nx[I];
        bool fin[I], m1[I], m2[I];
#pragma unroll
        for (int j = 0; j < I; ++j) {
            const bool k3 = k[j] == 3;
            nx[j] = e[j] & (k3 ? AC_STATE_MASK3 : AC_STATE_MASK);
            fin[j] = (e[j] & AC_FLAG) != 0;
            m1[j] = k3 ? (e[j] & AC_FLAG_MID1) != 0 : (k[j] == 2 && (e[j] & AC_FLAG_MID) != 0);
            m2[j] = k3 && (e[j] & AC_FLAG_MID) != 0;
            any |= (uint32_t)(fin[j] | m1[j] | m2[j]);
        }
        if (__any_sync(FULL, any)) {
#pragma unroll
            for (int j = 0; j < I; ++j) {
                const uint32_t p = pos[j];
                const bool h1 = m1[j] && p >= ch[j].lo && p < ch[j].hi;
                const uint32_t b1 = __ballot_sync(FULL, h1);
                if (b1) append(q, qn, b1, h1, ch[j].start + p, tag1(sym[j] & 3u), s[j], ch[j].text_id, lt, em);
                const bool h2 = m2[j] && p + 1 >= ch[j].lo && p + 1 < ch[j].hi;
                const uint32_t b2 = __ballot_sync(FULL, h2);
                if (b2)
                    append(q, qn, b2, h2, ch[j].start + p + 1, tag2(sym[j] & 3u, (sym[j] >> 2) & 3u), s[j],
                           ch[j].text_id, lt, em);
                const uint32_t pe = p + k[j] - 1;  // last base of this lookup
                const bool hf = fin[j] && pe >= ch[j].lo && pe < ch[j].hi;
                const uint32_t bf = __ballot_sync(FULL, hf);
                if (bf) append(q, qn, bf, hf, ch[j].start + pe, 0u, nx[j], ch[j].text_id, lt, em);
            }
        }
#pragma unroll
        for (int j = 0; j < I; ++j)
            if (act[j]) {
                s[j] = nx[j];
                bits[j] >>= 2 * k[j];
                nb[j] -= k[j];
                pos[j] += k[j];
            }
    }
    if (qn) drain(q, qn, em);
}

// Walk I chains in lockstep three bases per lookup, for machines whose
// three-base table covers every state: each step is one lookup for every
// lane, so no lane waits on another, and the hits of a step are voted on
// together. The text is read 48 bases (three words, sixteen steps) at a time
// through L1: a lane's next groups come from the same cached line. The step
// loop is not unrolled (its three append sites per step made the unrolled
// body large enough to slow the emission-heavy regions).
template <int I, bool InL1>
__device__ __forceinline__ void walk3_lock(const Chain (&ch)[I], const uint32_t* __restrict__ sm, uint32_t hot,
                                           const Tables& tb, const Emit* em, uint4* q, uint64_t pol_tab,
                                           uint64_t pol_txt) {
    constexpr uint32_t FLAGS = AC_FLAG | AC_FLAG_MID | AC_FLAG_MID1;
    uint32_t ng = 0;  // 48-base groups
#pragma unroll
    for (int j = 0; j < I; ++j) {
        const uint32_t g = (ch[j].hi + 47) / 48;
        ng = g > ng ? g : ng;
    }
    ng = __reduce_max_sync(FULL, ng);
    const uint32_t lt = lanemask_lt();
    uint32_t s[I];
#pragma unroll
    for (int j = 0; j < I; ++j) s[j] = 0;
    uint32_t qn = 0;  // queued events (same value in every lane)
    for (uint32_t g = 0; g < ng; ++g) {
        uint32_t w[I][3];
        uint32_t fmask[I];
#pragma unroll
        for (int j = 0; j < I; ++j) {
            const bool act = 48u * g < ch[j].hi;
            fmask[j] = act ? FLAGS : 0u;
            const uint64_t w0 = (ch[j].start >> 4) + 3ull * g;
#pragma unroll
            for (int v = 0; v < 3; ++v)
                w[j][v] = (act && w0 + v < ch[j].nwords) ? ld_text1(ch[j].text + w0 + v, pol_txt) : 0u;
        }
#pragma unroll 1
        for (uint32_t k = 0; k < 16; ++k) {
            uint32_t e[I], sp[I], sy[I];
#pragma unroll
            for (int j = 0; j < I; ++j) {
                sy[j] = w[j][0] & 63u;  // the next three bases
                const uint32_t idx = (s[j] << 6) | sy[j];
                e[j] = (s[j] < hot) ? sm[idx] : ld_table<InL1>(tb.delta3 + idx, pol_tab);
            }
            uint32_t any = 0;
#pragma unroll
            for (int j = 0; j < I; ++j) {
                sp[j] = s[j];
                s[j] = e[j] & AC_STATE_MASK3;
                any |= e[j] & fmask[j];
            }
            if (__any_sync(FULL, any)) {
                const uint32_t off = 48u * g + 3u * k;  // first base of this step
#pragma unroll
                for (int j = 0; j < I; ++j) {
                    const bool h1 = (e[j] & fmask[j] & AC_FLAG_MID1) && off >= ch[j].lo && off < ch[j].hi;
                    const uint32_t m1 = __ballot_sync(FULL, h1);
                    if (m1) append(q, qn, m1, h1, ch[j].start + off, tag1(sy[j] & 3u), sp[j], ch[j].text_id, lt, em);
                    const bool h2 = (e[j] & fmask[j] & AC_FLAG_MID) && off + 1 >= ch[j].lo && off + 1 < ch[j].hi;
                    const uint32_t m2 = __ballot_sync(FULL, h2);
                    if (m2)
                        append(q, qn, m2, h2, ch[j].start + off + 1, tag2(sy[j] & 3u, (sy[j] >> 2) & 3u), sp[j],
                               ch[j].text_id, lt, em);
                    const bool h3 = (e[j] & fmask[j] & AC_FLAG) && off + 2 >= ch[j].lo && off + 2 < ch[j].hi;
                    const uint32_t m3 = __ballot_sync(FULL, h3);
                    if (m3) append(q, qn, m3, h3, ch[j].start + off + 2, 0u, s[j], ch[j].text_id, lt, em);
                }
            }
#pragma unroll
            for (int j = 0; j < I; ++j) {  // move the window 6 bits on
                w[j][0] = __funnelshift_r(w[j][0], w[j][1], 6);
                w[j][1] = __funnelshift_r(w[j][1], w[j][2], 6);
                w[j][2] >>= 6;
            }
        }
    }
    if (qn) drain(q, qn, em);
}

// Kernel variants by ST: 1 and 2 the lockstep walk at one or two bases per
// lookup; 3 the three-base walk with lanes on their own schedules; 4 the
// lockstep three-base walk, used when every state has a three-base row (the
// launchers pick 3 or 4 for a requested stride of 3).
template <int I, int ST, bool InL1>
__device__ __forceinline__ void walk_any(const Chain (&ch)[I], const uint32_t* __restrict__ sm, uint32_t hot,
                                         const Tables& tb, const Emit* em, uint4* q, uint64_t pol_tab,
                                         uint64_t pol_txt) {
    if constexpr (ST == 4)
        walk3_lock<I, InL1>(ch, sm, hot, tb, em, q, pol_tab, pol_txt);
    else if constexpr (ST == 3)
        walk3_free<I, InL1>(ch, sm, hot, tb, em, q, pol_tab, pol_txt);
    else
        walk<I, ST, InL1>(ch, sm, hot, tb, em, q, pol_tab, pol_txt);
}

// Copies `rows16` 16-byte rows (the hot prefix of the table) to shared memory.
__device__ __forceinline__ void stage_hot(uint4* sm_rows, const uint32_t* table, uint32_t rows16) {
    const uint4* g = reinterpret_cast<const uint4*>(table);
    for (uint32_t r = threadIdx.x; r < rows16; r += blockDim.x) sm_rows[r] = __ldg(g + r);
    __syncthreads();
}

template <int I, int ST, int W>
__global__ void __launch_bounds__(Bounds<I, ST, W>::threads, Bounds<I, ST, W>::blocks) scan_kernel(ScanArgs a, uint32_t chunk, uint32_t hot, uint64_t n_chunks) {
    extern __shared__ uint4 sm_rows[];
    __shared__ Emit em;
    if (threadIdx.x == 0)
        set_emit(em, a.delta, a.delta2, a.s2_rows, a.out_off, a.out_ent, a.matches, a.capacity, a.counter, a.hits,
                 a.pos_offset, 0u);
    constexpr uint32_t R16 = ST == 1 ? 1 : (ST == 2 ? 4 : 16);  // 16-byte units per row
    stage_hot(sm_rows, ST == 1 ? a.delta : (ST == 2 ? a.delta2 : a.delta3), hot * R16);  // its barrier also publishes em
    const uint32_t* sm = reinterpret_cast<const uint32_t*>(sm_rows);
    const uint64_t pol_tab = policy_evict_last();
    const uint64_t pol_txt = policy_evict_first();
    const Tables tb{a.delta, a.delta2, a.s2_rows, a.delta3, a.s3_rows, a.n_states};
    uint4* q = sm_rows + hot * R16 + (threadIdx.x >> 5) * QCAP;
    const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nwords = (a.n + 15) >> 4;
    for (uint64_t round = 0; round < n_chunks; round += T * I) {  // uniform over the grid
        Chain ch[I];
#pragma unroll
        for (int j = 0; j < I; ++j) {
            const uint64_t c = round + (uint64_t)j * T + t;
            if (c < n_chunks) {
                const uint64_t lo = a.own_begin + c * chunk;
                set_chain(ch[j], a.text, nwords, a.text_id, lo, min(lo + chunk, a.own_end), a.halo);
            } else {
                idle_chain(ch[j], a.text, nwords, a.text_id);
            }
        }
        walk_any<I, ST, false>(ch, sm, hot, tb, &em, q, pol_tab, pol_txt);
    }
}

// Persistent batched scan: warps take 32*I work items at a time from a
// device cursor; item -> (text, chunk) by binary search over item_prefix.
template <int I, int ST, int W>
__global__ void __launch_bounds__(Bounds<I, ST, W>::threads, Bounds<I, ST, W>::blocks) batch_kernel(BatchArgs a, uint32_t hot) {
    extern __shared__ uint4 sm_rows[];
    __shared__ Emit em;
    if (threadIdx.x == 0)
        set_emit(em, a.delta, a.delta2, a.s2_rows, a.out_off, a.out_ent, a.matches, a.capacity, a.counter, a.hits,
                 0ull, 0u);
    constexpr uint32_t R16 = ST == 1 ? 1 : (ST == 2 ? 4 : 16);
    stage_hot(sm_rows, ST == 1 ? a.delta : (ST == 2 ? a.delta2 : a.delta3), hot * R16);  // its barrier also publishes em
    const uint32_t* sm = reinterpret_cast<const uint32_t*>(sm_rows);
    const uint64_t pol_tab = policy_evict_last();
    const uint64_t pol_txt = policy_evict_first();
    const Tables tb{a.delta, a.delta2, a.s2_rows, a.delta3, a.s3_rows, a.n_states};
    uint4* q = sm_rows + hot * R16 + (threadIdx.x >> 5) * QCAP;
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(&a.counter[1], (unsigned long long)(32 * I));
        base = __shfl_sync(FULL, base, 0);
        if (base >= a.n_items) break;
        Chain ch[I];
#pragma unroll
        for (int j = 0; j < I; ++j) {
            const unsigned long long item = base + (unsigned long long)j * 32 + lane;
            idle_chain(ch[j], nullptr, 0, 0);
            if (item < a.n_items) {
                uint32_t lo_t = 0, hi_t = a.n_texts;  // find t: prefix[t] <= item < prefix[t+1]
                while (hi_t - lo_t > 1) {
                    const uint32_t mid = (lo_t + hi_t) >> 1;
                    if (a.item_prefix[mid] <= item) lo_t = mid; else hi_t = mid;
                }
                const BatchText bt = a.texts[lo_t];
                const uint64_t lo = (item - a.item_prefix[lo_t]) * (uint64_t)a.chunk;
                set_chain(ch[j], bt.words, (bt.n + 15) >> 4, lo_t, lo, min(lo + a.chunk, bt.n), a.halo);
            }
        }
        walk_any<I, ST, true>(ch, sm, hot, tb, &em, q, pol_tab, pol_txt);
    }
}

// The paper's approach 2 (Sec. IV.A, Fig. 3): the keyword list is cut into
// consecutive chunks and each chunk gets its own machine; every machine scans
// the whole text. blockIdx.y selects the machine; each machine is small
// enough to live entirely in shared memory, and its keyword ids are offset
// back into the caller's numbering.
template <int I>
__global__ void __launch_bounds__(MaxThreads<I>::value) part_scan_kernel(PartArgs a, uint32_t chunk, uint64_t n_chunks) {
    extern __shared__ uint4 sm_rows[];
    __shared__ Emit em;
    const PartDesc pd = a.parts[blockIdx.y];
    if (threadIdx.x == 0)
        set_emit(em, pd.delta, nullptr, 0u, pd.out_off, pd.out_ent, a.matches, a.capacity, a.counter, pd.hits, 0ull,
                 pd.pid_offset);
    stage_hot(sm_rows, pd.delta, pd.n_states);  // its barrier also publishes em
    const uint32_t* sm = reinterpret_cast<const uint32_t*>(sm_rows);
    const uint64_t pol_tab = policy_evict_last();
    const uint64_t pol_txt = policy_evict_first();
    const Tables tb{pd.delta, nullptr, 0u, nullptr, 0u, pd.n_states};
    uint4* q = sm_rows + a.max_states + (threadIdx.x >> 5) * QCAP;
    const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nwords = (a.n + 15) >> 4;
    for (uint64_t round = 0; round < n_chunks; round += T * I) {
        Chain ch[I];
#pragma unroll
        for (int j = 0; j < I; ++j) {
            const uint64_t c = round + (uint64_t)j * T + t;
            if (c < n_chunks) {
                const uint64_t lo = a.own_begin + c * chunk;
                set_chain(ch[j], a.text, nwords, 0u, lo, min(lo + chunk, a.own_end), a.halo);
            } else {
                idle_chain(ch[j], a.text, nwords, 0u);
            }
        }
        walk<I, 1, true>(ch, sm, pd.n_states, tb, &em, q, pol_tab, pol_txt);
    }
}

// Failure-less matching (the PFAC scheme the paper cites in Sec. II): one
// lane per start position walks only the trie edges from the root and stops
// at the first missing edge; at every state it passes where keywords end
// (own keywords, not inherited ones) it reports them with its start. Each
// occurrence is found by the lane of its own start, so no failure
// transitions are needed. Lanes run in lockstep over depth so the event
// queue and drain of the main scan serve here too (pointed at the
// own-keyword tables); ownership is by end position, as in the main scan.
__global__ void __launch_bounds__(1024) failureless_kernel(FlArgs a, uint32_t hot) {
    extern __shared__ uint4 sm_rows[];
    __shared__ Emit em;  // no multi-base steps here: the drain needs no transition table
    if (threadIdx.x == 0)
        set_emit(em, nullptr, nullptr, 0u, a.own_off, a.own_ent, a.matches, a.capacity, a.counter, a.hits, 0ull, 0u);
    stage_hot(sm_rows, a.gotos, hot);  // its barrier also publishes em
    const uint32_t* sm = reinterpret_cast<const uint32_t*>(sm_rows);
    const uint64_t pol_tab = policy_evict_last();
    uint4* q = sm_rows + hot + (threadIdx.x >> 5) * QCAP;
    const uint32_t lt = lanemask_lt();
    const uint64_t first = a.own_begin > a.halo ? a.own_begin - a.halo : 0;  // starts whose ends can be owned
    const uint64_t span = a.own_end - first;
    const uint64_t T = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t rounds = (span + T - 1) / T;  // uniform over the grid
    uint32_t qn = 0;
    for (uint64_t r = 0; r < rounds; ++r) {
        const uint64_t i = first + r * T + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
        bool alive = i < a.own_end;
        uint32_t s = 0;
        for (uint32_t k = 0; k <= a.halo && __any_sync(FULL, alive); ++k) {
            const uint64_t p = i + k;
            uint32_t e = AC_NO_EDGE;
            if (alive && p < a.n) {
                const uint32_t c = (__ldg(a.text + (p >> 4)) >> (2 * (p & 15))) & 3u;
                const uint32_t idx = (s << 2) | c;
                e = (s < hot) ? sm[idx] : ld_table<true>(a.gotos + idx, pol_tab);
            }
            alive = alive && (e & AC_STATE_MASK31) != AC_NO_EDGE;
            if (alive) s = e & AC_STATE_MASK31;
            const bool h = alive && (e & AC_FLAG) && p >= a.own_begin && p < a.own_end;
            const uint32_t m = __ballot_sync(FULL, h);
            if (m) append(q, qn, m, h, p, 0u, s, a.text_id, lt, &em);
        }
    }
    if (qn) drain(q, qn, &em);
}

// One word of 16 ASCII bases (the bytes of q.x, q.y, q.z, q.w in order):
// base j's 2-bit code at bits 2j, and in ok whether all 16 bytes are A, C, G
// or T (either case when fold). Four bytes at a time: ((x >> 1) ^ (x >> 2)) & 3
// in every byte is the code (A, C, G, T -> 0, 1, 2, 3 in either case; bits
// shifted across bytes land above bit 1 and are masked off). The letter each
// code stands for is put back with one byte permute of "ACGT" selected by the
// four codes; a byte is a base exactly when it equals that letter (after the
// case fold). The multiply by 0x01041040 moves the code of byte k to bit
// 24 + 2k while every cross product lands below bit 24 in its own two-bit
// field, so the top byte is the four codes in order.
__device__ __forceinline__ uint32_t pack16(const uint4 q, bool fold, bool& ok) {
    const uint32_t by[4] = {q.x, q.y, q.z, q.w};
    uint32_t word = 0, diff = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const uint32_t x = by[k];
        const uint32_t c = ((x >> 1) ^ (x >> 2)) & 0x03030303u;
        const uint32_t t = c | (c >> 4);                            // bytes 0 and 2: two codes a nibble
        const uint32_t sel = (t & 0xffu) | ((t >> 8) & 0xff00u);    // the four codes, one per nibble
        diff |= (fold ? (x & 0xdfdfdfdfu) : x) ^ __byte_perm(0x54474341u, 0u, sel);  // "ACGT"
        word |= ((c * 0x01041040u) >> 24) << (8 * k);
    }
    ok = diff == 0;
    return word;
}

// Index (0-15) of the first byte of q that is not A, C, G or T.
__device__ __noinline__ uint32_t first_bad16(const uint4 q, bool fold) {
    const uint32_t by[4] = {q.x, q.y, q.z, q.w};
    for (uint32_t i = 0; i < 16; ++i) {
        const uint32_t c = (by[i >> 2] >> (8 * (i & 3))) & 0xffu;
        const uint32_t u = fold ? (c & 0xdfu) : c;
        if (!((u == 'A') | (u == 'C') | (u == 'G') | (u == 'T'))) return i;
    }
    return 16;
}

// ASCII bases to 2-bit words (16 bases a word, base j at bits 2j); *bad gets
// the smallest offset of a byte that is not a base (either case when fold).
__global__ void pack_kernel(const uint8_t* __restrict__ ascii, uint64_t n, uint32_t* __restrict__ packed, int fold,
                            unsigned long long* bad) {
    const uint64_t nw = (n + 15) >> 4;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    uint64_t first_bad = ~0ull;
    // a warp takes 128 whole words (2,048 bases) at a time: load j of lane t is
    // word 32j + t, so each load covers 512 contiguous bytes and each store 128
    const uint64_t lane = threadIdx.x & 31;
    const uint64_t warp = t0 >> 5, n_warps = stride >> 5;
    const uint32_t off = (uint32_t)(reinterpret_cast<uintptr_t>(ascii) & 15);
    uint64_t v0 = 0, vn = 0;  // words [v0, v0 + vn) go 128 per warp pass
    if (off == 0) {
        vn = 128 * (n >> 11);
        for (uint64_t g = warp; 128 * g < vn; g += n_warps) {
            const uint4* src = reinterpret_cast<const uint4*>(ascii) + 128 * g + lane;
            uint4 q[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) q[j] = __ldcs(src + 32 * j);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                bool ok;
                const uint64_t w = 128 * g + 32 * j + lane;
                packed[w] = pack16(q[j], fold != 0, ok);
                if (!ok) first_bad = min(first_bad, 16 * w + first_bad16(q[j], fold != 0));
            }
        }
    } else {
        // counted from the aligned address below the text, chunk m holds text bytes
        // [16m - off, 16m - off + 16), so word w is bytes off.. of chunk w and the
        // rest of chunk w + 1. Words from 1 on read no byte before the text, and up
        // to word (n + off - 32) / 16 none after it.
        const uint4* base = reinterpret_cast<const uint4*>(ascii - off);
        const uint64_t last = (n + off >= 32) ? (n + off - 32) >> 4 : 0;
        v0 = 1;
        vn = 128 * (last >> 7);
        const uint32_t r = off >> 2, sh = 8 * (off & 3);
        for (uint64_t g = warp; 128 * g < vn; g += n_warps) {
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const uint64_t w = 1 + 128 * g + 32 * j + lane;
                const uint4 a = __ldcs(base + w), b = __ldcs(base + w + 1);
                uint4 q;  // the 16 bytes from byte off of a:b (r whole words, then sh bits)
                switch (r) {  // the same for every thread
                    case 0: q = make_uint4(__funnelshift_r(a.x, a.y, sh), __funnelshift_r(a.y, a.z, sh),
                                           __funnelshift_r(a.z, a.w, sh), __funnelshift_r(a.w, b.x, sh)); break;
                    case 1: q = make_uint4(__funnelshift_r(a.y, a.z, sh), __funnelshift_r(a.z, a.w, sh),
                                           __funnelshift_r(a.w, b.x, sh), __funnelshift_r(b.x, b.y, sh)); break;
                    case 2: q = make_uint4(__funnelshift_r(a.z, a.w, sh), __funnelshift_r(a.w, b.x, sh),
                                           __funnelshift_r(b.x, b.y, sh), __funnelshift_r(b.y, b.z, sh)); break;
                    default: q = make_uint4(__funnelshift_r(a.w, b.x, sh), __funnelshift_r(b.x, b.y, sh),
                                            __funnelshift_r(b.y, b.z, sh), __funnelshift_r(b.z, b.w, sh)); break;
                }
                bool ok;
                packed[w] = pack16(q, fold != 0, ok);
                if (!ok) first_bad = min(first_bad, 16 * w + first_bad16(q, fold != 0));
            }
        }
    }
    // the rest one word at a time (word 0 of a text that is not 16-byte aligned, and the last bases)
    auto one_word = [&](uint64_t w) {
        const uint64_t b0 = w << 4;
        uint4 q;
        if (b0 + 16 <= n && ((reinterpret_cast<uintptr_t>(ascii + b0) & 15) == 0)) {
            q = __ldcs(reinterpret_cast<const uint4*>(ascii + b0));
        } else {  // past the end: 'A' (code 0, valid)
            uint32_t by[4];
            for (int k = 0; k < 4; ++k) {
                uint32_t x = 0;
                for (int i = 0; i < 4; ++i) {
                    const uint64_t o = b0 + 4 * k + i;
                    x |= (uint32_t)(o < n ? ascii[o] : 'A') << (8 * i);
                }
                by[k] = x;
            }
            q = make_uint4(by[0], by[1], by[2], by[3]);
        }
        bool ok;
        packed[w] = pack16(q, fold != 0, ok);
        if (!ok) first_bad = min(first_bad, b0 + first_bad16(q, fold != 0));
    };
    if (vn && v0 == 1 && t0 == 0) one_word(0);
    for (uint64_t w = (vn ? v0 + vn : 0) + t0; w < nw; w += stride) one_word(w);
    if (first_bad != ~0ull) atomicMin(bad, (unsigned long long)first_bad);
}

// Copies n bases of a packed text from base src_off of src to base dst_off
// of dst (any offsets). One thread per destination word. A word wholly inside
// the range is the 16 source bases starting at its first base: one funnel
// shift of the (at most two) source words that hold them. The (at most two)
// edge words rewrite only the bases of the range, base by base, and keep the
// other bases of the word.
__global__ void splice_kernel(uint32_t* __restrict__ dst, uint64_t dst_off, const uint32_t* __restrict__ src,
                              uint64_t src_off, uint64_t n) {
    const uint64_t w0 = dst_off >> 4, w1 = (dst_off + n + 15) >> 4;
    const uint64_t end = dst_off + n;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t w = w0 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; w < w1; w += stride) {
        const uint64_t p0 = w << 4;
        if (p0 >= dst_off && p0 + 16 <= end) {
            const uint64_t q0 = src_off + (p0 - dst_off);  // source of this word's first base
            const uint32_t sh = 2u * (uint32_t)(q0 & 15);
            const uint32_t lo = __ldg(src + (q0 >> 4));
            // with sh > 0 the word's last base, q0 + 15 < src_off + n, lies in the next source word
            dst[w] = sh ? __funnelshift_r(lo, __ldg(src + (q0 >> 4) + 1), sh) : lo;
            continue;
        }
        uint32_t word = dst[w];
#pragma unroll
        for (int j = 0; j < 16; ++j) {
            const uint64_t p = p0 + j;
            if (p < dst_off || p >= end) continue;
            const uint64_t q = src_off + (p - dst_off);
            const uint32_t b = (__ldg(src + (q >> 4)) >> (2 * (q & 15))) & 3u;
            word = (word & ~(3u << (2 * j))) | (b << (2 * j));
        }
        dst[w] = word;
    }
}

// counts[p] = sum over states s with p in output(s) of hits[s]; with clear,
// each counter read is set back to 0 (for buffers that the next scan reuses).
__global__ void counts_kernel(const uint32_t* __restrict__ out_off, const uint2* __restrict__ out_ent,
                              uint32_t n_states, unsigned long long* hits, unsigned long long* counts, int clear) {
    const uint32_t stride = gridDim.x * blockDim.x;
    for (uint32_t s = blockIdx.x * blockDim.x + threadIdx.x; s < n_states; s += stride) {
        const unsigned long long h = hits[s];
        if (!h) continue;
        if (clear) hits[s] = 0ull;
        for (uint32_t k = out_off[s]; k < out_off[s + 1]; ++k) atomicAdd(&counts[out_ent[k].x], h);
    }
}

// ---- serving: one batch's occurrences split per request, on the device.
// Pass 1 counts every request's occurrences (n_per[t]) and its per-keyword
// counts (req_counts[t * P + keyword]); pass 2 turns n_per into exclusive
// offsets (one block); pass 3 writes each occurrence into its request's
// range of `out` with text_id 0 (the order inside a range is free, as in any
// scan result). Lanes of a warp that hold the same request combine their
// atomics through __match_any_sync.
__global__ void serve_count_kernel(const ac_match* __restrict__ in, uint64_t nm, uint32_t P,
                                   unsigned long long* n_per, unsigned long long* req_counts) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31;
    for (uint64_t base = t0 - lane; base < nm; base += stride) {  // whole warps step together
        const uint64_t i = base + lane;
        const bool ok = i < nm;
        const ac_match m = ok ? in[i] : ac_match{0, 0, 0xffffffffu};
        const uint32_t peers = __match_any_sync(FULL, m.text_id);
        if (ok) {
            if (lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&n_per[m.text_id], (unsigned long long)__popc(peers));
            atomicAdd(&req_counts[(uint64_t)m.text_id * P + m.pattern_id], 1ull);
        }
    }
}

// offs[0..B]: exclusive prefix sums of n_per (one block of 1024 threads).
__global__ void serve_offsets_kernel(const unsigned long long* __restrict__ n_per, uint32_t B,
                                     unsigned long long* offs) {
    __shared__ unsigned long long part[1024];
    const uint32_t per = (B + blockDim.x - 1) / blockDim.x;
    const uint32_t a = threadIdx.x * per, b = min(B, a + per);
    unsigned long long sum = 0;
    for (uint32_t t = a; t < b; ++t) sum += n_per[t];
    part[threadIdx.x] = sum;
    __syncthreads();
    for (uint32_t d = 1; d < blockDim.x; d <<= 1) {  // inclusive scan of the partial sums
        const unsigned long long v = threadIdx.x >= d ? part[threadIdx.x - d] : 0ull;
        __syncthreads();
        part[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned long long run = part[threadIdx.x] - sum;
    for (uint32_t t = a; t < b; ++t) {
        offs[t] = run;
        run += n_per[t];
    }
    if (threadIdx.x == blockDim.x - 1) offs[B] = part[threadIdx.x];
}

__global__ void serve_scatter_kernel(const ac_match* __restrict__ in, uint64_t nm,
                                     const unsigned long long* __restrict__ offs, unsigned long long* cursor,
                                     ac_match* __restrict__ out) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint32_t lane = threadIdx.x & 31;
    const uint32_t lt = lanemask_lt();
    for (uint64_t base = t0 - lane; base < nm; base += stride) {
        const uint64_t i = base + lane;
        const bool ok = i < nm;
        const ac_match m = ok ? in[i] : ac_match{0, 0, 0xffffffffu};
        const uint32_t peers = __match_any_sync(FULL, m.text_id);
        const uint32_t leader = __ffs(peers) - 1;
        unsigned long long first = 0;
        if (ok && lane == leader) first = atomicAdd(&cursor[m.text_id], (unsigned long long)__popc(peers));
        first = __shfl_sync(FULL, first, leader);
        if (ok) out[offs[m.text_id] + first + __popc(peers & lt)] = ac_match{m.pos, m.pattern_id, 0u};
    }
}

// Raises a kernel's dynamic shared-memory limit to `bytes`; the driver call is
// skipped when this device already has a limit at least that high for this
// kernel (keyed by the kernel's address: kernels of one signature share a type).
template <typename K>
int set_smem(K kern, size_t bytes) {
    static std::mutex mu;
    static std::map<std::pair<const void*, int>, int> done;
    int dev = 0;
    cudaGetDevice(&dev);
    const auto key = std::make_pair(reinterpret_cast<const void*>(kern), dev);
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = done.find(key);
        if (it != done.end() && (int)bytes <= it->second) return 0;
    }
    const int rc = (int)cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (rc == 0) {
        std::lock_guard<std::mutex> lk(mu);
        int& v = done[key];
        if ((int)bytes > v) v = (int)bytes;
    }
    return rc;
}

// The (interleave, stride) pairs that are compiled: stride 2 up to interleave 4,
// stride 3 up to interleave 2.
template <typename F>
int dispatch(uint32_t interleave, uint32_t stride, F&& f) {
    if (stride == 1) {
        switch (interleave) {
            case 1: return f.template operator()<1, 1>();
            case 2: return f.template operator()<2, 1>();
            case 4: return f.template operator()<4, 1>();
            case 8: return f.template operator()<8, 1>();
        }
    } else if (stride == 2) {
        switch (interleave) {
            case 1: return f.template operator()<1, 2>();
            case 2: return f.template operator()<2, 2>();
            case 4: return f.template operator()<4, 2>();
        }
    } else if (stride == 3) {
        switch (interleave) {
            case 1: return f.template operator()<1, 3>();
            case 2: return f.template operator()<2, 3>();
        }
    } else if (stride == 4) {  // three bases in lockstep (every state has a three-base row)
        switch (interleave) {
            case 1: return f.template operator()<1, 4>();
            case 2: return f.template operator()<2, 4>();
        }
    }
    return -1;
}

}  // namespace

const DeviceProps& ac_device_props() {
    static thread_local DeviceProps cache[64];
    static thread_local bool have[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (!have[dev]) {
        DeviceProps p;
        p.device = dev;
        cudaDeviceGetAttribute(&p.sms, cudaDevAttrMultiProcessorCount, dev);
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        p.smem_optin = (size_t)v;
        cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, dev);
        p.l2 = (size_t)v;
        cache[dev] = p;
        have[dev] = true;
    }
    return cache[dev];
}

uint32_t ac_max_threads(uint32_t interleave, uint32_t stride) {
    if (stride == 3) return interleave == 1 ? MaxThreads<1, 3>::value : (interleave == 2 ? MaxThreads<2, 3>::value : 0);
    switch (interleave) {
        case 1: return MaxThreads<1>::value;
        case 2: return MaxThreads<2>::value;
        case 4: return MaxThreads<4>::value;
        case 8: return MaxThreads<8>::value;
        default: return 0;
    }
}

uint32_t ac_wide_threads(uint32_t interleave, uint32_t stride) {
    return (interleave == 1 && stride == 3) ? kWideThreads : 0u;
}

bool ac_shape_compiled(uint32_t interleave, uint32_t stride) {
    return (stride == 1 && (interleave == 1 || interleave == 2 || interleave == 4 || interleave == 8)) ||
           (stride == 2 && (interleave == 1 || interleave == 2 || interleave == 4)) ||
           (stride == 3 && (interleave == 1 || interleave == 2));
}

// Shared memory each kernel declares statically (its Emit block), kept free
// of the dynamic allocation so the two fit the per-block limit together.
constexpr size_t kStaticSmem = 256;
static_assert(sizeof(Emit) <= kStaticSmem, "Emit fits the reserve");

static size_t row_bytes(uint32_t stride) { return stride >= 3 ? 256 : (stride == 2 ? 64 : 16); }

size_t ac_scan_smem_bytes(uint32_t hot, uint32_t threads, uint32_t stride) {
    return (size_t)hot * row_bytes(stride) + (size_t)(threads / 32) * QCAP * 16;
}

uint32_t ac_max_hot_states(uint32_t threads, uint32_t stride) {
    const DeviceProps& p = ac_device_props();
    const size_t queues = ac_scan_smem_bytes(0, threads, stride) + kStaticSmem;
    return p.smem_optin > queues ? (uint32_t)((p.smem_optin - queues) / row_bytes(stride)) : 0u;
}

namespace {
struct Occupancy {
    const ScanShape& sh;
    template <int I, int ST>
    int operator()() const {
        if constexpr (I == 1 && ST >= 3) {
            if (wide_build<I, ST>(sh.threads)) return blocks<I, ST, 1>();
        }
        return blocks<I, ST, 0>();
    }
    template <int I, int ST, int W>
    int blocks() const {
        const size_t smem = ac_scan_smem_bytes(sh.hot, sh.threads, ST);
        if (set_smem(scan_kernel<I, ST, W>, smem) != 0) return 0;
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, scan_kernel<I, ST, W>, (int)sh.threads, smem) !=
            cudaSuccess)
            return 0;
        return nb;
    }
};

struct ScanLaunch {
    const ScanArgs& a;
    const ScanShape& sh;
    uint64_t n_chunks;
    cudaStream_t st;
    template <int I, int ST>
    int operator()() const {
        if constexpr (I == 1 && ST >= 3) {
            if (wide_build<I, ST>(sh.threads)) return launch<I, ST, 1>();
        }
        return launch<I, ST, 0>();
    }
    template <int I, int ST, int W>
    int launch() const {
        const size_t smem = ac_scan_smem_bytes(sh.hot, sh.threads, ST);
        int rc = set_smem(scan_kernel<I, ST, W>, smem);
        if (rc) return rc;
        if (ac_fault_launch()) return (int)cudaErrorLaunchFailure;
        scan_kernel<I, ST, W><<<sh.grid, sh.threads, smem, st>>>(a, sh.chunk, sh.hot, n_chunks);
        return (int)cudaGetLastError();
    }
};

struct BatchLaunch {
    const BatchArgs& a;
    const ScanShape& sh;
    cudaStream_t st;
    bool prepare_only;
    template <int I, int ST>
    int operator()() const {
        if constexpr (I == 1 && ST >= 3) {
            if (wide_build<I, ST>(sh.threads)) return launch<I, ST, 1>();
        }
        return launch<I, ST, 0>();
    }
    template <int I, int ST, int W>
    int launch() const {
        const size_t smem = ac_scan_smem_bytes(sh.hot, sh.threads, ST);
        int rc = set_smem(batch_kernel<I, ST, W>, smem);
        if (rc || prepare_only) return rc;
        if (ac_fault_launch()) return (int)cudaErrorLaunchFailure;
        batch_kernel<I, ST, W><<<sh.grid, sh.threads, smem, st>>>(a, sh.hot);
        return (int)cudaGetLastError();
    }
};
}  // namespace

uint32_t ac_blocks_per_sm(const ScanShape& sh, bool all_rows3) {
    // occupancy depends on (device, interleave, kernel variant, threads, shared memory): memoised
    static std::mutex mu;
    static std::map<std::tuple<int, uint32_t, uint32_t, uint32_t, size_t>, uint32_t> memo;
    int dev = 0;
    cudaGetDevice(&dev);
    const uint32_t stride = sh.stride ? sh.stride : 1u;
    // the kernel the launch will run: three bases per lookup runs the lockstep
    // walk (variant 4) when every state has a three-base row
    const uint32_t code = (stride == 3 && all_rows3) ? 4u : stride;
    const auto key = std::make_tuple(dev, sh.interleave, code, sh.threads,
                                     ac_scan_smem_bytes(sh.hot, sh.threads, stride));
    {
        std::lock_guard<std::mutex> lk(mu);
        auto it = memo.find(key);
        if (it != memo.end()) return it->second;
    }
    const int nb = dispatch(sh.interleave, code, Occupancy{sh});
    const uint32_t r = nb > 0 ? (uint32_t)nb : 0u;
    std::lock_guard<std::mutex> lk(mu);
    memo[key] = r;
    return r;
}

int ac_launch_pack(const uint8_t* ascii, uint64_t n, uint32_t* packed, bool fold, unsigned long long* bad,
                   void* stream) {
    if (n == 0) return 0;
    const uint64_t nw = (n + 15) >> 4;
    const DeviceProps& p = ac_device_props();
    // one wave of resident blocks (each strides over the text), no more
    static std::atomic<int> resident{0};
    if (resident.load() == 0) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pack_kernel, 256, 0) != cudaSuccess || nb < 1) nb = 1;
        resident.store(nb);
    }
    uint64_t blocks = (nw + 4 * 256 - 1) / (4 * 256);  // four words a thread per pass
    const uint64_t cap = (uint64_t)p.sms * (uint64_t)resident.load();
    if (blocks > cap) blocks = cap;
    if (blocks < 1) blocks = 1;
    if (ac_fault_launch()) return (int)cudaErrorLaunchFailure;
    pack_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(ascii, n, packed, fold ? 1 : 0, bad);
    return (int)cudaGetLastError();
}

int ac_launch_scan(const ScanArgs& a, const ScanShape& sh, void* stream) {
    const uint64_t owned = a.own_end > a.own_begin ? a.own_end - a.own_begin : 0;
    if (owned == 0) return 0;
    if ((sh.stride == 2 && !a.delta2) || (sh.stride == 3 && !a.delta3)) return (int)cudaErrorInvalidValue;
    const uint64_t n_chunks = (owned + sh.chunk - 1) / sh.chunk;
    const uint32_t code = (sh.stride == 3 && a.s3_rows >= a.n_states) ? 4u : sh.stride;
    const int rc = dispatch(sh.interleave, code, ScanLaunch{a, sh, n_chunks, (cudaStream_t)stream});
    return rc < 0 ? (int)cudaErrorInvalidValue : rc;
}

int ac_launch_batch(const BatchArgs& a, const ScanShape& sh, void* stream) {
    if (a.n_items == 0) return 0;
    if ((sh.stride == 2 && !a.delta2) || (sh.stride == 3 && !a.delta3)) return (int)cudaErrorInvalidValue;
    const uint32_t code = (sh.stride == 3 && a.s3_rows >= a.n_states) ? 4u : sh.stride;
    const int rc = dispatch(sh.interleave, code, BatchLaunch{a, sh, (cudaStream_t)stream, false});
    return rc < 0 ? (int)cudaErrorInvalidValue : rc;
}

int ac_prepare_batch(const ScanShape& sh) {
    BatchArgs dummy{};
    int rc = dispatch(sh.interleave, sh.stride, BatchLaunch{dummy, sh, nullptr, true});
    if (rc == 0 && sh.stride == 3) rc = dispatch(sh.interleave, 4u, BatchLaunch{dummy, sh, nullptr, true});
    return rc < 0 ? (int)cudaErrorInvalidValue : rc;
}

int ac_launch_part_scan(const PartArgs& a, uint32_t n_parts, uint32_t grid_x, uint32_t threads, uint32_t chunk,
                        void* stream) {
    const uint64_t owned = a.own_end > a.own_begin ? a.own_end - a.own_begin : 0;
    if (owned == 0 || n_parts == 0) return 0;
    const uint64_t n_chunks = (owned + chunk - 1) / chunk;
    const size_t smem = ac_scan_smem_bytes(a.max_states, threads, 1);
    int rc = set_smem(part_scan_kernel<1>, smem);
    if (rc) return rc;
    if (ac_fault_launch()) return (int)cudaErrorLaunchFailure;
    part_scan_kernel<1><<<dim3(grid_x, n_parts), threads, smem, (cudaStream_t)stream>>>(a, chunk, n_chunks);
    return (int)cudaGetLastError();
}

int ac_launch_failureless(const FlArgs& a, uint32_t hot, void* stream) {
    if (a.own_end <= a.own_begin) return 0;
    const size_t smem = ac_scan_smem_bytes(hot, 1024, 1);
    int rc = set_smem(failureless_kernel, smem);
    if (rc) return rc;
    const DeviceProps& p = ac_device_props();
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, failureless_kernel, 1024, smem);
    const uint64_t span = a.own_end - (a.own_begin > a.halo ? a.own_begin - a.halo : 0);
    const uint64_t want = (span + 1023) / 1024;
    const uint32_t grid = (uint32_t)std::min<uint64_t>(want, (uint64_t)p.sms * std::max(nb, 1));
    if (ac_fault_launch()) return (int)cudaErrorLaunchFailure;
    failureless_kernel<<<grid, 1024, smem, (cudaStream_t)stream>>>(a, hot);
    return (int)cudaGetLastError();
}

int ac_launch_splice(uint32_t* dst, uint64_t dst_off, const uint32_t* src, uint64_t src_off, uint64_t n,
                     void* stream) {
    if (n == 0) return 0;
    const uint64_t words = ((dst_off + n + 15) >> 4) - (dst_off >> 4);
    const DeviceProps& p = ac_device_props();
    uint64_t blocks = (words + 255) / 256;
    const uint64_t cap = (uint64_t)p.sms * 8;
    if (blocks > cap) blocks = cap;
    if (ac_fault_launch()) return (int)cudaErrorLaunchFailure;
    splice_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(dst, dst_off, src, src_off, n);
    return (int)cudaGetLastError();
}

int ac_launch_counts(const uint32_t* out_off, const uint2* out_ent, uint32_t n_states,
                     const unsigned long long* hits, unsigned long long* counts, void* stream, bool clear_hits) {
    if (n_states == 0) return 0;
    const DeviceProps& p = ac_device_props();
    uint32_t blocks = (n_states + 255) / 256;
    const uint32_t cap = (uint32_t)p.sms * 8;
    if (blocks > cap) blocks = cap;
    if (ac_fault_launch()) return (int)cudaErrorLaunchFailure;
    counts_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(out_off, out_ent, n_states,
                                                            const_cast<unsigned long long*>(hits), counts,
                                                            clear_hits ? 1 : 0);
    return (int)cudaGetLastError();
}

int ac_launch_serve_split(const ac_match* in, uint64_t nm, uint32_t n_req, uint32_t n_patterns, ac_match* out,
                          unsigned long long* req_counts, unsigned long long* n_per, unsigned long long* offs,
                          unsigned long long* cursor, void* stream) {
    const cudaStream_t st = (cudaStream_t)stream;
    const DeviceProps& p = ac_device_props();
    const uint64_t want = (nm + 255) / 256;
    const uint32_t blocks = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(want, (uint64_t)p.sms * 8));
    if (nm) {
        if (ac_fault_launch()) return (int)cudaErrorLaunchFailure;
        serve_count_kernel<<<blocks, 256, 0, st>>>(in, nm, n_patterns, n_per, req_counts);
    }
    if (ac_fault_launch()) return (int)cudaErrorLaunchFailure;
    serve_offsets_kernel<<<1, 1024, 0, st>>>(n_per, n_req, offs);
    if (nm) {
        if (ac_fault_launch()) return (int)cudaErrorLaunchFailure;
        serve_scatter_kernel<<<blocks, 256, 0, st>>>(in, nm, offs, cursor, out);
    }
    return (int)cudaGetLastError();
}
