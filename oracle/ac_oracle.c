/*
 * ac_oracle.c - plain, slow, single-threaded Aho-Corasick (Sec. III.A of the
 * paper) and a brute-force matcher.
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the test suite, the package's smoke
 * check and the benchmark's CPU-baseline leg; never by the product path.
 * It shares no code with the CUDA library.
 *
 * Data structures are deliberately the textbook ones: a trie with child
 * lists (goto), one failure pointer per state (fail) and one explicit list of
 * keyword ids per state (output). No flattening, no renumbering, no
 * precomputed full transition table: the scan follows failure transitions at
 * run time exactly as the paper's stage 2 describes.
 *
 * ORC_MUTANT (compile-time, default 0) plants one known mistake; it exists
 * only so the test suite can show that its pins catch each such mistake.
 */
#include "ac_oracle.h"

#include <stdlib.h>
#include <string.h>

#ifndef ORC_MUTANT
#define ORC_MUTANT 0
#endif

#define ORC_FAIL (-1)

struct orc_machine {
    int32_t n_states, cap_states;
    int32_t* first_child;  /* first child in the child list, -1 if none */
    int32_t* next_sibling; /* next child of the same parent, -1 if none */
    uint8_t* label;        /* character on the edge into the state      */
    int32_t* depth;        /* distance from the root                    */
    int32_t* fail;         /* failure transition                        */
    /* output(s): own keywords first, then output(fail(s)) */
    uint32_t** out_ids;
    int32_t* out_n;
    int32_t* own_n; /* how many of out_ids[s] end at s itself */
    uint32_t n_pats;
    uint32_t* pat_len;
};

struct orc_matches {
    uint64_t n, cap;
    uint64_t* pos;
    uint32_t* pid;
};

/* ---------------------------------------------------------------- helpers */

static int grow_states(orc_machine* m) {
    int32_t nc = m->cap_states ? m->cap_states * 2 : 64;
#define GROW(f, T)                                                   \
    do {                                                             \
        T* p = (T*)realloc(m->f, (size_t)nc * sizeof(T));            \
        if (!p) return 0;                                            \
        m->f = p;                                                    \
    } while (0)
    GROW(first_child, int32_t);
    GROW(next_sibling, int32_t);
    GROW(label, uint8_t);
    GROW(depth, int32_t);
    GROW(fail, int32_t);
    GROW(out_ids, uint32_t*);
    GROW(out_n, int32_t);
    GROW(own_n, int32_t);
#undef GROW
    m->cap_states = nc;
    return 1;
}

static int32_t new_state(orc_machine* m, int32_t parent, uint8_t c) {
    if (m->n_states == m->cap_states && !grow_states(m)) return -1;
    int32_t s = m->n_states++;
    m->first_child[s] = -1;
    m->next_sibling[s] = -1;
    m->label[s] = c;
    m->depth[s] = parent < 0 ? 0 : m->depth[parent] + 1;
    m->fail[s] = 0;
    m->out_ids[s] = NULL;
    m->out_n[s] = 0;
    m->own_n[s] = 0;
    if (parent >= 0) { /* append at the end of the parent's child list */
        int32_t* link = &m->first_child[parent];
        while (*link >= 0) link = &m->next_sibling[*link];
        *link = s;
    }
    return s;
}

/* goto(s, c): the trie edge, or ORC_FAIL. The root's missing edges are
 * handled by the scan (the root accepts every character and stays). */
static int32_t go(const orc_machine* m, int32_t s, uint8_t c) {
    for (int32_t t = m->first_child[s]; t >= 0; t = m->next_sibling[t])
        if (m->label[t] == c) return t;
    return ORC_FAIL;
}

static int push_id(uint32_t** ids, int32_t* n, uint32_t id) {
    uint32_t* p = (uint32_t*)realloc(*ids, (size_t)(*n + 1) * sizeof(uint32_t));
    if (!p) return 0;
    p[*n] = id;
    *ids = p;
    *n += 1;
    return 1;
}

static int push_match(orc_matches* r, uint64_t pos, uint32_t pid) {
    if (r->n == r->cap) {
        uint64_t nc = r->cap ? r->cap * 2 : 1024;
        uint64_t* p = (uint64_t*)realloc(r->pos, nc * sizeof(uint64_t));
        if (!p) return 0;
        r->pos = p;
        uint32_t* q = (uint32_t*)realloc(r->pid, nc * sizeof(uint32_t));
        if (!q) return 0;
        r->pid = q;
        r->cap = nc;
    }
    r->pos[r->n] = pos;
    r->pid[r->n] = pid;
    r->n += 1;
    return 1;
}

/* ---------------------------------------------------------------- stage 1 */

orc_machine* orc_build(const uint8_t* const* pats, const uint32_t* lens, uint32_t n_pats) {
    if (!pats || !lens || n_pats == 0) return NULL;
    for (uint32_t p = 0; p < n_pats; ++p)
        if (lens[p] == 0 || !pats[p]) return NULL;

    orc_machine* m = (orc_machine*)calloc(1, sizeof(orc_machine));
    if (!m) return NULL;
    m->n_pats = n_pats;
    m->pat_len = (uint32_t*)malloc(n_pats * sizeof(uint32_t));
    if (!m->pat_len || new_state(m, -1, 0) != 0) goto oom;

    /* goto: insert each keyword, creating states in order of need */
    for (uint32_t p = 0; p < n_pats; ++p) {
        m->pat_len[p] = lens[p];
        int32_t s = 0;
        for (uint32_t j = 0; j < lens[p]; ++j) {
            int32_t t = go(m, s, pats[p][j]);
            if (t == ORC_FAIL) {
                t = new_state(m, s, pats[p][j]);
                if (t < 0) goto oom;
            }
            s = t;
        }
        if (!push_id(&m->out_ids[s], &m->out_n[s], p)) goto oom;
        m->own_n[s] += 1;
    }

    /* fail + output: breadth-first from the root, so that fail(r) and
     * output(fail(r)) are final before any child of r is visited. */
    int32_t* queue = (int32_t*)malloc((size_t)m->n_states * sizeof(int32_t));
    if (!queue) goto oom;
    int32_t head = 0, tail = 0;
    for (int32_t t = m->first_child[0]; t >= 0; t = m->next_sibling[t]) {
        m->fail[t] = 0; /* depth-1 states fail to the root */
        queue[tail++] = t;
    }
    while (head < tail) {
        int32_t r = queue[head++];
        /* output(r) = own(r) U output(fail(r)); fail(r) is shallower, so done */
        int32_t f = m->fail[r];
#if ORC_MUTANT != 1 /* mutant 1: drop the inherited term of the output function */
        for (int32_t k = 0; k < m->out_n[f]; ++k)
            if (!push_id(&m->out_ids[r], &m->out_n[r], m->out_ids[f][k])) { free(queue); goto oom; }
#endif
        for (int32_t u = m->first_child[r]; u >= 0; u = m->next_sibling[u]) {
            uint8_t a = m->label[u];
            int32_t v = m->fail[r];
#if ORC_MUTANT == 4 /* mutant 4: a single failure hop instead of following the chain */
            if (v != 0 && go(m, v, a) == ORC_FAIL) v = m->fail[v];
#else
            while (v != 0 && go(m, v, a) == ORC_FAIL) v = m->fail[v];
#endif
            int32_t g = go(m, v, a);
#if ORC_MUTANT == 5 /* mutant 5: ignore the root's own edges when the chain ends there */
            if (v == 0) g = ORC_FAIL;
#endif
            m->fail[u] = (g == ORC_FAIL) ? 0 : g;
            queue[tail++] = u;
        }
    }
    free(queue);
    return m;

oom:
    orc_free(m);
    return NULL;
}

void orc_free(orc_machine* m) {
    if (!m) return;
    for (int32_t s = 0; s < m->n_states; ++s) free(m->out_ids[s]);
    free(m->first_child);
    free(m->next_sibling);
    free(m->label);
    free(m->depth);
    free(m->fail);
    free(m->out_ids);
    free(m->out_n);
    free(m->own_n);
    free(m->pat_len);
    free(m);
}

int32_t orc_num_states(const orc_machine* m) { return m->n_states; }

int32_t orc_goto(const orc_machine* m, int32_t s, int32_t c) {
    if (s < 0 || s >= m->n_states || c < 0 || c > 255) return ORC_FAIL;
    return go(m, s, (uint8_t)c);
}

int32_t orc_fail(const orc_machine* m, int32_t s) {
    return (s < 0 || s >= m->n_states) ? ORC_FAIL : m->fail[s];
}

int32_t orc_depth(const orc_machine* m, int32_t s) {
    return (s < 0 || s >= m->n_states) ? ORC_FAIL : m->depth[s];
}

int32_t orc_output(const orc_machine* m, int32_t s, uint32_t* ids, int32_t cap) {
    if (s < 0 || s >= m->n_states) return 0;
    for (int32_t k = 0; k < m->out_n[s] && k < cap; ++k) ids[k] = m->out_ids[s][k];
    return m->out_n[s];
}

/* ---------------------------------------------------------------- stage 2 */

/* One character of stage 2: follow failure transitions until a valid
 * transition exists (the root always has one: itself), then take it.
 * Every state entered is passed to rec (failure hops included). */
static int32_t step(const orc_machine* m, int32_t s, uint8_t c, int32_t* rec, int64_t* nrec,
                    int64_t cap) {
    int32_t t;
    while ((t = go(m, s, c)) == ORC_FAIL && s != 0) {
        s = m->fail[s];
        if (rec) {
            if (*nrec < cap) rec[*nrec] = s;
            *nrec += 1;
        }
#if ORC_MUTANT == 3 /* mutant 3: do not read the same character again after a failure hop */
        return s;
#endif
    }
    s = (t == ORC_FAIL) ? 0 : t;
    if (rec) {
        if (*nrec < cap) rec[*nrec] = s;
        *nrec += 1;
    }
    return s;
}

int64_t orc_trace(const orc_machine* m, const uint8_t* text, uint64_t n, int32_t* states,
                  int64_t cap) {
    int64_t k = 0;
    if (cap > 0) states[0] = 0;
    k = 1;
    int32_t s = 0;
    for (uint64_t i = 0; i < n; ++i) s = step(m, s, text[i], states, &k, cap);
    return k;
}

orc_matches* orc_scan(const orc_machine* m, const uint8_t* text, uint64_t n, uint64_t* counts) {
    orc_matches* r = (orc_matches*)calloc(1, sizeof(orc_matches));
    if (!r) return NULL;
    if (counts) memset(counts, 0, m->n_pats * sizeof(uint64_t));
    int32_t s = 0;
    for (uint64_t i = 0; i < n; ++i) {
        s = step(m, s, text[i], NULL, NULL, 0);
        for (int32_t k = 0; k < m->out_n[s]; ++k) {
            uint32_t p = m->out_ids[s][k];
#if ORC_MUTANT == 2 /* mutant 2: off-by-one start position */
            uint64_t start = i + 2 - m->pat_len[p];
#else
            uint64_t start = i + 1 - m->pat_len[p];
#endif
            if (!push_match(r, start, p)) {
                orc_matches_free(r);
                return NULL;
            }
#if ORC_MUTANT == 6 /* mutant 6: inherited keywords not counted */
            if (counts && k < m->own_n[s]) counts[p] += 1;
#else
            if (counts) counts[p] += 1;
#endif
        }
    }
    return r;
}

orc_matches* orc_naive(const uint8_t* const* pats, const uint32_t* lens, uint32_t n_pats,
                       const uint8_t* text, uint64_t n) {
    orc_matches* r = (orc_matches*)calloc(1, sizeof(orc_matches));
    if (!r) return NULL;
    for (uint64_t i = 0; i < n; ++i) {
        for (uint32_t p = 0; p < n_pats; ++p) {
            if (lens[p] == 0 || lens[p] > n - i) continue;
            if (memcmp(text + i, pats[p], lens[p]) == 0 && !push_match(r, i, p)) {
                orc_matches_free(r);
                return NULL;
            }
        }
    }
    return r;
}

uint64_t orc_matches_size(const orc_matches* r) { return r ? r->n : 0; }

void orc_matches_copy(const orc_matches* r, uint64_t* pos, uint32_t* pid) {
    if (!r) return;
    if (r->n) {
        memcpy(pos, r->pos, r->n * sizeof(uint64_t));
        memcpy(pid, r->pid, r->n * sizeof(uint32_t));
    }
}

void orc_matches_free(orc_matches* r) {
    if (!r) return;
    free(r->pos);
    free(r->pid);
    free(r);
}
