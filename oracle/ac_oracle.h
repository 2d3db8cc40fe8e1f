/*
 * ac_oracle.h - the CPU oracle for the Aho-Corasick scan.
 *
 * TEST INFRASTRUCTURE ONLY. Only the test suite, the package's smoke check and
 * the benchmark's CPU-baseline leg may load this library. The product path
 * (the CUDA library and its Python binding) never links, imports or calls it,
 * and the two share no code, header, table or helper.
 *
 * What it computes (Aho-Corasick, as described in Sec. III.A of the paper):
 *   stage 1 builds the pattern matching machine from the keywords:
 *     goto   - a trie; state 0 is the root; states are numbered in the order
 *              they are created while the keywords are inserted one after
 *              another (this reproduces the state numbers of Fig. 1/Fig. 2);
 *     fail   - the failure transition of every state (Fig. 1, dotted lines);
 *     output - the keywords recognised on entering a state ("final states"
 *              of Fig. 2), i.e. the keywords ending at the state itself plus
 *              the output of its failure state;
 *   stage 2 reads the text once: on a character with no valid transition the
 *   machine follows failure transitions and reads the same character again
 *   until a valid transition exists (the root accepts every character).
 *   After each character it reports every keyword of output(state); all
 *   overlapping occurrences are reported (Fig. 2, text "SHERS").
 *
 * Conventions fixed where the paper is silent:
 *   - an occurrence is (start position, pattern id), start 0-based;
 *   - pattern ids are 0-based indices in the caller's order; duplicate
 *     keywords are separate ids that share a state and are all reported;
 *   - the alphabet is bytes (0..255), so the paper's example runs verbatim.
 *
 * Parity pins live in the test suite: the worked example of Fig. 1/2,
 * brute force on small inputs, closed forms and invariants.
 */
#ifndef AC_ORACLE_H
#define AC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct orc_machine orc_machine;
typedef struct orc_matches orc_matches;

/* Stage 1. Returns NULL on an empty keyword, n_pats == 0 or allocation failure. */
orc_machine* orc_build(const uint8_t* const* pats, const uint32_t* lens, uint32_t n_pats);
void orc_free(orc_machine* m);

int32_t orc_num_states(const orc_machine* m);
int32_t orc_goto(const orc_machine* m, int32_t s, int32_t c); /* -1 = fail (no edge) */
int32_t orc_fail(const orc_machine* m, int32_t s);
int32_t orc_depth(const orc_machine* m, int32_t s);
/* Writes up to cap ids of output(s) (own keywords first, then inherited),
 * returns |output(s)|. */
int32_t orc_output(const orc_machine* m, int32_t s, uint32_t* ids, int32_t cap);

/* Stage 2 with every state entered recorded, failure hops included
 * (states[0] is the start state 0). Returns the number of states entered,
 * writing at most cap of them. */
int64_t orc_trace(const orc_machine* m, const uint8_t* text, uint64_t n,
                  int32_t* states, int64_t cap);

/* Stage 2. counts[n_pats] (may be NULL) receives per-keyword occurrence counts.
 * Returns the occurrence list in scan order (end position ascending, then the
 * order of output(state)). */
orc_matches* orc_scan(const orc_machine* m, const uint8_t* text, uint64_t n, uint64_t* counts);

/* Brute force: every (i, p) with text[i .. i+len_p-1] == pat_p, ordered by
 * start i, then p. */
orc_matches* orc_naive(const uint8_t* const* pats, const uint32_t* lens, uint32_t n_pats,
                       const uint8_t* text, uint64_t n);

uint64_t orc_matches_size(const orc_matches* r);
void orc_matches_copy(const orc_matches* r, uint64_t* pos, uint32_t* pid);
void orc_matches_free(orc_matches* r);

#ifdef __cplusplus
}
#endif
#endif
