// ac_builder.cpp - stage 1 of Sec. III.A on the host: the goto / failure /
// output machine, then flattened into a full transition table over
// {A,C,G,T} with states renumbered breadth first.
//
// goto:    a trie with a 4-way child array per state.
// failure: breadth first; depth-1 states fail to the root; for a child u of r
//          reached on a, fail(u) = goto(f, a) for the first f on r's failure
//          chain (fail(r), fail(fail(r)), ..., root) that has an a-edge, else
//          the root.
// output:  the keywords ending at s plus output(fail(s)).
// stride 2: delta2(s, xy) = delta(delta(s, x), y) for the 16 base pairs, with
//          one flag for each of the two states entered (a scan that reads two
//          bases per lookup must still report keywords ending at the first).
// stride 3: delta3(s, xyz) = delta(delta(delta(s, x), y), z) for the 64 base
//          triples, with one flag for each of the three states entered.
// flatten: delta(s, a) = goto(s, a) if the edge exists, else delta(fail(s), a)
//          (the root's missing edges loop to the root). Computed breadth
//          first, so delta(fail(s), .) is final before s is visited. A scan
//          over delta makes exactly one lookup per base and visits the same
//          states as the paper's failure-following scan (Sec. III.A), which
//          re-reads a character after each failure hop.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <deque>
#include <new>
#include <system_error>
#include <thread>
#include <vector>

#include "ac_internal.h"

namespace {

inline int base_code(uint8_t c, bool fold) {
    switch (c) {
        case 'A': return 0;
        case 'C': return 1;
        case 'G': return 2;
        case 'T': return 3;
        case 'a': return fold ? 0 : -1;
        case 'c': return fold ? 1 : -1;
        case 'g': return fold ? 2 : -1;
        case 't': return fold ? 3 : -1;
        default: return -1;
    }
}

// Runs f(s) for s in [0, rows) on the host's cores (rows are independent).
template <typename F>
void parallel_rows(uint32_t rows, F&& f) {
    const uint32_t hw = std::max(1u, std::min(16u, std::thread::hardware_concurrency()));
    const uint32_t T = rows < 4096 ? 1u : hw;
    if (T == 1) {
        for (uint32_t s = 0; s < rows; ++s) f(s);
        return;
    }
    auto range = [&](uint32_t t) {
        const uint32_t a = (uint32_t)((uint64_t)rows * t / T), b = (uint32_t)((uint64_t)rows * (t + 1) / T);
        for (uint32_t s = a; s < b; ++s) f(s);
    };
    std::vector<std::thread> pool;
    uint32_t spawned = 0;
    try {
        for (; spawned < T; ++spawned) pool.emplace_back(range, spawned);
    } catch (const std::system_error&) {  // no more threads: the rest on this one
    }
    for (uint32_t t = spawned; t < T; ++t) range(t);
    for (auto& th : pool) th.join();
}

}  // namespace

int ac_build_host(const char* const* patterns, const uint32_t* lens, uint32_t n, bool fold_case,
                  bool with_stride2, uint32_t stride2_states, bool with_stride3, uint32_t stride3_states,
                  bool with_failureless, HostTables* t, uint32_t* bad_pattern) {
    if (!patterns || !lens || n == 0 || !t) return AC_ERR_INVALID_ARG;
    uint64_t total = 0;
    for (uint32_t p = 0; p < n; ++p) {
        if (lens[p] == 0) {
            if (bad_pattern) *bad_pattern = p;
            return AC_ERR_EMPTY_PATTERN;
        }
        if (!patterns[p]) return AC_ERR_INVALID_ARG;
        for (uint32_t j = 0; j < lens[p]; ++j)
            if (base_code((uint8_t)patterns[p][j], fold_case) < 0) {
                if (bad_pattern) *bad_pattern = p;
                return AC_ERR_ALPHABET;
            }
        total += lens[p];
    }
    try {
        // ---- goto (trie), states in creation order
        std::vector<int32_t> child;  // [S*4], -1 = no edge
        child.reserve(std::min<uint64_t>(total + 1, AC_MAX_STATES) * 4);
        child.assign(4, -1);
        std::vector<std::vector<uint32_t>> own(1);
        std::vector<uint32_t> pat_node(n);
        uint32_t max_len = 0, min_len = UINT32_MAX;
        for (uint32_t p = 0; p < n; ++p) {
            int32_t s = 0;
            for (uint32_t j = 0; j < lens[p]; ++j) {
                int c = base_code((uint8_t)patterns[p][j], fold_case);
                int32_t nx = child[(size_t)s * 4 + c];
                if (nx < 0) {
                    if (own.size() >= AC_MAX_STATES) return AC_ERR_TOO_LARGE;
                    nx = (int32_t)own.size();
                    child[(size_t)s * 4 + c] = nx;
                    child.insert(child.end(), {-1, -1, -1, -1});
                    own.emplace_back();
                }
                s = nx;
            }
            own[s].push_back(p);
            pat_node[p] = (uint32_t)s;
            max_len = std::max(max_len, lens[p]);
            min_len = std::min(min_len, lens[p]);
        }
        const uint32_t S = (uint32_t)own.size();

        // ---- breadth-first order (children visited A, C, G, T)
        std::vector<uint32_t> order;  // bfs position -> creation id
        order.reserve(S);
        std::vector<uint32_t> depth_c(S, 0);
        order.push_back(0);
        for (size_t h = 0; h < order.size(); ++h) {
            uint32_t r = order[h];
            for (int c = 0; c < 4; ++c) {
                int32_t u = child[(size_t)r * 4 + c];
                if (u >= 0) {
                    depth_c[u] = depth_c[r] + 1;
                    order.push_back((uint32_t)u);
                }
            }
        }
        std::vector<uint32_t> bfs_id(S);
        for (uint32_t i = 0; i < S; ++i) bfs_id[order[i]] = i;

        // ---- failure + flattened delta in one breadth-first pass (creation ids).
        // When r is visited, fail(r) was set by r's parent and the row of
        // fail(r) (a shallower state, visited earlier) is final. For a child u of
        // r on c, delta(fail(r), c) is exactly "follow r's failure chain until a
        // c-edge exists, else the root", i.e. fail(u).
        std::vector<uint32_t> fail_c(S, 0);
        std::vector<uint32_t> delta_c((size_t)S * 4, 0);
        for (uint32_t h = 0; h < S; ++h) {
            uint32_t r = order[h];
            for (int c = 0; c < 4; ++c) {
                int32_t u = child[(size_t)r * 4 + c];
                uint32_t via_fail = (r == 0) ? 0u : delta_c[(size_t)fail_c[r] * 4 + c];
                if (u >= 0) {
                    delta_c[(size_t)r * 4 + c] = (uint32_t)u;
                    fail_c[u] = via_fail;  // depth-1 states: the root
                } else {
                    delta_c[(size_t)r * 4 + c] = via_fail;  // the root loops on itself
                }
            }
        }

        // ---- output sets: own(s) then output(fail(s)), breadth first
        // (stored per breadth-first id as CSR)
        std::vector<uint32_t> out_n(S, 0);
        uint64_t E = 0;
        for (uint32_t h = 0; h < S; ++h) {
            uint32_t s = order[h];
            out_n[s] = (uint32_t)own[s].size() + (s ? out_n[fail_c[s]] : 0u);
            E += out_n[s];
        }
        if (E > 0xffffffffull) return AC_ERR_TOO_LARGE;

        t->n_states = S;
        t->n_patterns = n;
        t->max_len = max_len;
        t->min_len = min_len;
        t->max_depth = depth_c[order[S - 1]];
        t->out_off.assign((size_t)S + 1, 0);
        for (uint32_t i = 0; i < S; ++i) t->out_off[i + 1] = t->out_off[i] + out_n[order[i]];
        t->out_pid.assign(E, 0);
        for (uint32_t i = 0; i < S; ++i) {
            uint32_t s = order[i];
            uint32_t w = t->out_off[i];
            for (uint32_t p : own[s]) t->out_pid[w++] = p;
            if (s) {
                uint32_t f = bfs_id[fail_c[s]];  // already written: f < i
                for (uint32_t k = t->out_off[f]; k < t->out_off[f + 1]; ++k) t->out_pid[w++] = t->out_pid[k];
            }
        }

        // ---- renumber the flattened table to breadth-first ids, add the flag
        t->delta.assign((size_t)S * 4, 0);
        t->depth.assign(S, 0);
        t->fail.assign(S, 0);
        for (uint32_t i = 0; i < S; ++i) {
            uint32_t s = order[i];
            t->depth[i] = depth_c[s];
            t->fail[i] = bfs_id[fail_c[s]];
            for (int c = 0; c < 4; ++c) {
                uint32_t nx = bfs_id[delta_c[(size_t)s * 4 + c]];
                uint32_t flag = (t->out_off[nx + 1] > t->out_off[nx]) ? AC_FLAG : 0u;
                t->delta[(size_t)i * 4 + c] = nx | flag;
            }
        }
        t->pat_len.assign(lens, lens + n);
        t->pat_state.resize(n);
        for (uint32_t p = 0; p < n; ++p) t->pat_state[p] = bfs_id[pat_node[p]];
        t->out_ent.resize(2 * E);
        for (uint64_t k = 0; k < E; ++k) {
            t->out_ent[2 * k] = t->out_pid[k];
            t->out_ent[2 * k + 1] = lens[t->out_pid[k]];
        }

        // ---- failure-less form (trie edges only): goto[s][c] = child or AC_NO_EDGE,
        // bit 31 = the child is where some keyword ends; own keywords per state as CSR
        t->gotos.clear();
        t->own_off.clear();
        t->own_pid.clear();
        t->own_ent.clear();
        if (with_failureless) {
            t->gotos.assign((size_t)S * 4, AC_NO_EDGE);
            t->own_off.assign((size_t)S + 1, 0);
            for (uint32_t p = 0; p < n; ++p) t->own_off[t->pat_state[p] + 1]++;
            for (uint32_t i = 0; i < S; ++i) t->own_off[i + 1] += t->own_off[i];
            t->own_pid.assign(n, 0);
            std::vector<uint32_t> fill(t->own_off.begin(), t->own_off.end() - 1);
            for (uint32_t p = 0; p < n; ++p) t->own_pid[fill[t->pat_state[p]]++] = p;  // ids ascending per state
            t->own_ent.resize(2 * (size_t)n);
            for (uint32_t j = 0; j < n; ++j) {
                t->own_ent[2 * j] = t->own_pid[j];
                t->own_ent[2 * j + 1] = lens[t->own_pid[j]];
            }
            for (uint32_t i = 0; i < S; ++i) {
                const uint32_t s = order[i];
                for (int c = 0; c < 4; ++c) {
                    const int32_t u = child[(size_t)s * 4 + c];
                    if (u < 0) continue;
                    const uint32_t b = bfs_id[u];
                    t->gotos[(size_t)i * 4 + c] = b | (t->own_off[b + 1] > t->own_off[b] ? AC_FLAG : 0u);
                }
            }
        }

        // ---- two bases per lookup: delta2[s][x | y << 2] = delta(delta(s, x), y),
        // bit 31 = the final state has output, bit 30 = the state after x has output
        t->delta2.clear();
        t->s2_rows = 0;
        if (with_stride2) {
            const uint32_t rows = std::min<uint32_t>(S, stride2_states ? stride2_states : AC_DEFAULT_STRIDE2_ROWS);
            t->s2_rows = std::min<uint32_t>(rows, AC_MAX_STATES_STRIDE2);
            t->delta2.assign((size_t)t->s2_rows * 16, 0);
            auto has_out = [&](uint32_t u) { return t->out_off[u + 1] > t->out_off[u]; };
            parallel_rows(t->s2_rows, [&](uint32_t s) {
                for (uint32_t x = 0; x < 4; ++x) {
                    const uint32_t m = t->delta[(size_t)s * 4 + x] & AC_STATE_MASK;
                    for (uint32_t y = 0; y < 4; ++y) {
                        const uint32_t f = t->delta[(size_t)m * 4 + y] & AC_STATE_MASK;
                        t->delta2[(size_t)s * 16 + (x | (y << 2))] =
                            f | (has_out(f) ? AC_FLAG : 0u) | (has_out(m) ? AC_FLAG_MID : 0u);
                    }
                }
            });
        }

        // ---- three bases per lookup: delta3[s][x | y << 2 | z << 4], bits 0-28 the
        // state after z; bits 31 / 30 / 29 = the states after z / y / x have output
        t->delta3.clear();
        t->s3_rows = 0;
        if (with_stride3) {
            const uint32_t rows = std::min<uint32_t>(S, stride3_states ? stride3_states : AC_DEFAULT_STRIDE3_ROWS);
            t->s3_rows = std::min<uint32_t>(rows, AC_MAX_STATES_STRIDE3);
            t->delta3.assign((size_t)t->s3_rows * 64, 0);
            auto has_out = [&](uint32_t u) { return t->out_off[u + 1] > t->out_off[u]; };
            parallel_rows(t->s3_rows, [&](uint32_t s) {
                for (uint32_t x = 0; x < 4; ++x) {
                    const uint32_t a = t->delta[(size_t)s * 4 + x] & AC_STATE_MASK;
                    for (uint32_t y = 0; y < 4; ++y) {
                        const uint32_t b = t->delta[(size_t)a * 4 + y] & AC_STATE_MASK;
                        for (uint32_t z = 0; z < 4; ++z) {
                            const uint32_t c = t->delta[(size_t)b * 4 + z] & AC_STATE_MASK;
                            t->delta3[(size_t)s * 64 + (x | (y << 2) | (z << 4))] =
                                c | (has_out(c) ? AC_FLAG : 0u) | (has_out(b) ? AC_FLAG_MID : 0u) |
                                (has_out(a) ? AC_FLAG_MID1 : 0u);
                        }
                    }
                }
            });
        }
    } catch (const std::bad_alloc&) {
        return AC_ERR_OOM;
    }
    return AC_OK;
}
