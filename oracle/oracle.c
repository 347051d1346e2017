/*
 * ORACLE - test infrastructure only.
 *
 * A plain, slow, obviously correct CPU statement of what the speculative DFA
 * membership test of Ko, Jung, Han & Burgstaller ("A Speculative Parallel DFA
 * Membership Test for Multicore, SIMD and Cloud Computing Environments")
 * computes.  Only the tests, the smoke check and the benchmark's CPU-baseline
 * leg may call it; the product path never does.  It shares no code, header or
 * table with the CUDA path: it works on the user's uint32 transition function
 * directly, with no alphabet classes, no initial-state tables built ahead of
 * time and no blocking.
 *
 * Conventions (Sec. 2.1 of the paper): a DFA is (Q, Sigma, delta, q0, F) with
 * delta: Q x Sigma -> Q.  The paper assumes a unique error (sink) state q_e.
 * A delta entry of -1 means "go to q_e"; q_e is numbered |Q| (one past the
 * user's states), loops on every symbol and is not accepting.  An input byte
 * b is the symbol byte_to_symbol[b] (identity when the map is NULL); a byte
 * mapped to 0xFF is not in Sigma and the run reports ORACLE_ESYMBOL.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_OK 0
#define ORACLE_EINVAL (-1)
#define ORACLE_ESYMBOL (-2)
#define ORACLE_ENOMEM (-3)

/* delta extended by the error-state row (Sec. 2.1). */
static uint32_t step(uint32_t Q, uint32_t S, const int32_t *delta, uint32_t q, uint32_t a) {
    if (q == Q) return Q;
    int32_t t = delta[(uint64_t)q * S + a];
    return t < 0 ? Q : (uint32_t)t;
}

static int symbol(const uint8_t *map, uint8_t b) {
    if (!map) return b;
    return map[b] == 0xFF ? -1 : map[b];
}

static int is_final(const uint8_t *final_flags, uint32_t Q, uint32_t s) {
    return s < Q && final_flags[s];
}

/*
 * Algorithm 1 (Sec. 1, "Sequential DFA matching"): state <- q0; for every
 * input position i: state <- delta(state, Str[i]); accept iff state in F.
 * No early exit at q_e (the paper's Sec. 3 remark makes it optional).
 */
int oracle_run(uint32_t Q, uint32_t S, const int32_t *delta, uint32_t q0,
               const uint8_t *final_flags, const uint8_t *byte_to_symbol,
               const uint8_t *str, uint64_t n, uint32_t *final_out, int32_t *accept_out) {
    uint32_t state = q0;
    for (uint64_t i = 0; i < n; ++i) {
        int a = symbol(byte_to_symbol, str[i]);
        if (a < 0) return ORACLE_ESYMBOL;
        state = step(Q, S, delta, state, (uint32_t)a);
    }
    *final_out = state;
    *accept_out = is_final(final_flags, Q, state);
    return ORACLE_OK;
}

/*
 * States left out of every initial-state set.  Algorithm 3 drops the error
 * state q_e from its initial-state sets because a run that reached it never leaves it (Sec. 3,
 * Sec. 4.2).  For a DFA that is not minimal the same argument holds for every
 * state that loops on all symbols and is not accepting, so those are the
 * states excluded here: excluded[s] = 1 iff delta(s, a) == s for all a and
 * s is not final.  excluded has Q+1 entries (index Q is q_e).
 */
void oracle_excluded(uint32_t Q, uint32_t S, const int32_t *delta, const uint8_t *final_flags,
                     uint8_t *excluded) {
    for (uint32_t s = 0; s <= Q; ++s) {
        int loops = 1;
        for (uint32_t a = 0; a < S && loops; ++a)
            if (step(Q, S, delta, s, a) != s) loops = 0;
        excluded[s] = (uint8_t)(loops && !is_final(final_flags, Q, s));
    }
}

/*
 * Eq. (11): I_sigma = { s : delta(x, sigma) = s for some x in Q }, minus the
 * excluded states (Algorithm 3's initial-state sets).  iset is S x (Q+1) flags,
 * iset[a*(Q+1)+s] = 1 iff s in I_a.  Returns I_max of Eq. (12): the largest
 * cardinality (Algorithm 3's maximum over the sets, read as cardinalities).
 */
uint32_t oracle_isets(uint32_t Q, uint32_t S, const int32_t *delta, const uint8_t *final_flags,
                      uint8_t *iset) {
    uint8_t *excl = (uint8_t *)malloc(Q + 1);
    oracle_excluded(Q, S, delta, final_flags, excl);
    uint32_t imax = 0;
    for (uint32_t a = 0; a < S; ++a) {
        uint8_t *row = iset + (uint64_t)a * (Q + 1);
        memset(row, 0, Q + 1);
        for (uint32_t x = 0; x <= Q; ++x) {
            uint32_t t = step(Q, S, delta, x, a);
            if (!excl[t]) row[t] = 1;
        }
        uint32_t card = 0;
        for (uint32_t s = 0; s <= Q; ++s) card += row[s];
        if (card > imax) imax = card;
    }
    free(excl);
    return imax;
}

/*
 * Algorithm 3 ("DFA matching applying initial state sets") for a given
 * partition, followed by the sequential merge of Eq. (8).
 *
 * starts[0..P] are the chunk boundaries: chunk i covers [starts[i], starts[i+1]).
 * The vectors L_i (Sec. 4.1) are dense over Q+1 and start as the identity.
 * Chunk 0 is matched from q0 only.  Chunk i >= 1 is matched from every j in
 * I_sigma where sigma = Str[starts[i]-1] is its reverse lookahead symbol; if
 * starts[i] == 0 every earlier chunk is empty and the only possible initial
 * state is q0.  maps_out (optional) receives P x (Q+1) entries.
 */
int oracle_chunked(uint32_t Q, uint32_t S, const int32_t *delta, uint32_t q0,
                   const uint8_t *final_flags, const uint8_t *byte_to_symbol,
                   const uint8_t *str, uint64_t n, uint32_t P, const uint64_t *starts,
                   uint32_t *maps_out, uint32_t *final_out, int32_t *accept_out) {
    if (P == 0 || starts[0] != 0 || starts[P] != n) return ORACLE_EINVAL;
    for (uint32_t i = 0; i < P; ++i)
        if (starts[i] > starts[i + 1]) return ORACLE_EINVAL;
    for (uint64_t t = 0; t < n; ++t)
        if (symbol(byte_to_symbol, str[t]) < 0) return ORACLE_ESYMBOL;

    uint8_t *iset = (uint8_t *)malloc((uint64_t)S * (Q + 1));
    uint32_t *L = (uint32_t *)malloc((uint64_t)P * (Q + 1) * sizeof(uint32_t));
    if (!iset || !L) { free(iset); free(L); return ORACLE_ENOMEM; }
    oracle_isets(Q, S, delta, final_flags, iset);

    for (uint32_t i = 0; i < P; ++i) {
        uint32_t *Li = L + (uint64_t)i * (Q + 1);
        for (uint32_t j = 0; j <= Q; ++j) Li[j] = j;           /* identity */
        uint64_t start = starts[i], end = starts[i + 1];        /* [start, end) */
        if (i == 0 || start == 0) {
            /* chunk 0 (or a chunk preceded only by empty chunks): from q0 */
            uint32_t s = q0;
            for (uint64_t k = start; k < end; ++k)
                s = step(Q, S, delta, s, (uint32_t)symbol(byte_to_symbol, str[k]));
            Li[q0] = s;
        } else {
            uint32_t sigma = (uint32_t)symbol(byte_to_symbol, str[start - 1]);
            const uint8_t *I = iset + (uint64_t)sigma * (Q + 1);
            for (uint32_t j = 0; j <= Q; ++j) {
                if (!I[j]) continue;
                uint32_t s = j;
                for (uint64_t k = start; k < end; ++k)
                    s = step(Q, S, delta, s, (uint32_t)symbol(byte_to_symbol, str[k]));
                Li[j] = s;
            }
        }
    }
    /* Eq. (8): last = L_{P-1}[ ... L_1[ L_0[q0] ] ... ] */
    uint32_t last = L[q0];
    for (uint32_t i = 1; i < P; ++i) last = L[(uint64_t)i * (Q + 1) + last];
    *final_out = last;
    *accept_out = is_final(final_flags, Q, last);
    if (maps_out) memcpy(maps_out, L, (uint64_t)P * (Q + 1) * sizeof(uint32_t));
    free(iset);
    free(L);
    return ORACLE_OK;
}

/* Eq. (9): L_{i,j}[k] = L_j[ L_i[k] ] for k in 0..m-1. */
void oracle_compose(uint32_t m, const uint32_t *Li, const uint32_t *Lj, uint32_t *out) {
    for (uint32_t k = 0; k < m; ++k) out[k] = Lj[Li[k]];
}

/*
 * Eq. (13): I_{sigma_1..sigma_r} = { delta*(x, sigma_1..sigma_r) : x in Q },
 * minus the excluded states (the same exclusion as Algorithm 3 and 4).
 * out has Q+1 flags; returns the set's cardinality.
 */
uint32_t oracle_iset_word(uint32_t Q, uint32_t S, const int32_t *delta, const uint8_t *final_flags,
                          const uint32_t *word, uint32_t len, uint8_t *out) {
    uint8_t *excl = (uint8_t *)malloc(Q + 1);
    oracle_excluded(Q, S, delta, final_flags, excl);
    memset(out, 0, Q + 1);
    for (uint32_t x = 0; x <= Q; ++x) {
        uint32_t s = x;
        for (uint32_t i = 0; i < len; ++i) s = step(Q, S, delta, s, word[i]);
        if (!excl[s]) out[s] = 1;
    }
    uint32_t card = 0;
    for (uint32_t s = 0; s <= Q; ++s) card += out[s];
    free(excl);
    return card;
}

/* delta*(q, w) over a symbol word (Sec. 2.1), used for the r-symbol sets of Eq. (13). */
uint32_t oracle_delta_star(uint32_t Q, uint32_t S, const int32_t *delta, uint32_t q,
                           const uint32_t *word, uint32_t len) {
    for (uint32_t i = 0; i < len; ++i) q = step(Q, S, delta, q, word[i]);
    return q;
}
