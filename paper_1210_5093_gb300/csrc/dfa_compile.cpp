// DFA compilation (done once per DFA, off the timed path).
//
// The first part of Algorithm 3 computes the initial-state sets
// I_sigma = { delta(x, sigma) : x in Q } \ {q_e} (Eq. 11) and
// I_max = max_sigma |I_sigma| (Eq. 12).  Because I_max is a static property of
// the DFA it may be computed off-line (Sec. 4.2); this file does it once at
// dfa_create, together with the GPU data layout:
//   * symbols (and bytes) whose delta columns are identical form one alphabet
//     class, so the table has C columns instead of |Sigma|;
//   * every state that loops on all symbols and is not accepting is left out
//     of the I sets (the error state q_e is one; a run that reaches such a
//     state never leaves it, which is the paper's reason for dropping q_e);
//   * the table is stored class-major with entries pre-multiplied by the
//     entry size, so one lookup is T[row_offset(class) + state_offset].
#include <algorithm>
#include <cstring>
#include <map>

#include "dfa_internal.h"

namespace dfam {

uint64_t chunk_start(uint64_t n, uint32_t P, uint32_t m, uint32_t k) {
    // Eq. (6) with unit weights and m states per later chunk: L_0 = n*m/(m+P-1)
    // and chunk k >= 1 starts at floor(L_0 + (k-1)*L_0/m) = floor(n*(m+k-1)/(m+P-1)).
    if (k == 0) return 0;
    if (k >= P) return n;
    unsigned __int128 num = (unsigned __int128)n * (uint64_t)(m + k - 1);
    return (uint64_t)(num / (uint64_t)(m + P - 1));
}

int compile_dfa(uint32_t Q, uint32_t S, const int32_t* delta, uint32_t q0, const uint32_t* finals,
                uint32_t nf, const uint8_t* b2s, HostDfa* out) {
    if (!out || !delta || Q == 0 || Q > kMaxStates || S == 0 || S > 256 || q0 >= Q) return DFA_EINVAL;
    if (nf && !finals) return DFA_EINVAL;
    if (!b2s && S != 256) return DFA_EINVAL;
    HostDfa h;
    h.Q = Q;
    h.S = S;
    h.qe = Q + 1;  // q_e = Q, always present (unreachable when delta has no -1)
    h.q0 = q0;
    const uint32_t qe = h.qe;
    for (uint64_t i = 0; i < (uint64_t)Q * S; ++i)
        if (delta[i] < -1 || delta[i] >= (int32_t)Q) return DFA_EINVAL;
    h.accept.assign(qe, 0);
    for (uint32_t i = 0; i < nf; ++i) {
        if (finals[i] >= Q) return DFA_EINVAL;
        h.accept[finals[i]] = 1;
    }
    if (b2s)
        for (int b = 0; b < 256; ++b)
            if (b2s[b] != 0xFF && b2s[b] >= S) return DFA_EINVAL;

    auto target = [&](uint32_t q, uint32_t a) -> uint32_t {
        if (q == Q) return Q;
        int32_t t = delta[(uint64_t)q * S + a];
        return t < 0 ? Q : (uint32_t)t;
    };

    // Excluded states: absorbing on every symbol of Sigma and not accepting.
    h.excluded.assign(qe, 0);
    for (uint32_t s = 0; s < qe; ++s) {
        bool loops = true;
        for (uint32_t a = 0; a < S && loops; ++a) loops = target(s, a) == s;
        h.excluded[s] = (loops && !h.accept[s]) ? 1 : 0;
        h.num_excluded += h.excluded[s];
    }

    // Alphabet classes: bytes whose symbols have identical columns share a class.
    std::map<std::vector<uint32_t>, uint32_t> col_id;
    std::vector<std::vector<uint32_t>> cols;
    h.byte_class.assign(256, kNone16);
    std::vector<int> class_of_symbol(S, -1);
    for (int b = 0; b < 256; ++b) {
        int a = b2s ? (b2s[b] == 0xFF ? -1 : b2s[b]) : b;
        if (a < 0) continue;
        if (class_of_symbol[a] < 0) {
            std::vector<uint32_t> col(qe);
            for (uint32_t q = 0; q < qe; ++q) col[q] = target(q, (uint32_t)a);
            auto it = col_id.find(col);
            if (it == col_id.end()) {
                uint32_t id = (uint32_t)cols.size();
                col_id.emplace(col, id);
                cols.push_back(std::move(col));
                class_of_symbol[a] = (int)id;
            } else {
                class_of_symbol[a] = (int)it->second;
            }
        }
        h.byte_class[b] = (uint16_t)class_of_symbol[a];
    }
    const uint32_t C = (uint32_t)cols.size();
    h.C = C;

    // Initial-state sets per class (Eq. 11) plus the start set {q0} as set C.
    h.iset_off.assign(C + 3, 0);
    h.iset.clear();
    std::vector<uint8_t> mark(qe);
    double sum = 0;
    for (uint32_t c = 0; c < C; ++c) {
        std::fill(mark.begin(), mark.end(), 0);
        for (uint32_t x = 0; x < qe; ++x) {
            uint32_t t = cols[c][x];
            if (!h.excluded[t]) mark[t] = 1;
        }
        for (uint32_t s = 0; s < qe; ++s)
            if (mark[s]) h.iset.push_back((uint16_t)s);
        h.iset_off[c + 1] = (uint32_t)h.iset.size();
        uint32_t card = h.iset_off[c + 1] - h.iset_off[c];
        h.imax = std::max(h.imax, card);
        sum += card;
    }
    h.iset.push_back((uint16_t)q0);                  // set C: the start set {q0}
    h.iset_off[C + 1] = (uint32_t)h.iset.size();
    for (uint32_t s = 0; s < qe; ++s) h.iset.push_back((uint16_t)s);  // set C+1: all of Q (Algorithm 2)
    h.iset_off[C + 2] = (uint32_t)h.iset.size();
    h.gamma = (double)h.imax / (double)Q;
    h.mean_iset = C ? sum / C : 0.0;

    // pos[c][s]: index of s within I_c (kNone16 if s is not a member).
    h.pos.assign((size_t)(C + 2) * qe, kNone16);
    for (uint32_t c = 0; c <= C + 1; ++c)
        for (uint32_t i = h.iset_off[c]; i < h.iset_off[c + 1]; ++i)
            h.pos[(size_t)c * qe + h.iset[i]] = (uint16_t)(i - h.iset_off[c]);

    // Table image: class-major, entries pre-scaled by the entry size; row C = identity.
    // 16-bit entries hold 2 * state, so above 32768 states (q_e included) they are 32-bit.
    h.sb = qe <= 256 ? 1 : (qe <= 32768 ? 2 : 4);
    const uint32_t align = 4 / h.sb;  // rows start on a 4-byte boundary
    h.qpad = (qe + align - 1) / align * align;
    const uint64_t tbytes = (uint64_t)(C + 1) * h.qpad * h.sb;
    h.table.assign(tbytes, 0);
    for (uint32_t c = 0; c <= C; ++c)
        for (uint32_t q = 0; q < h.qpad; ++q) {
            uint32_t nxt = q < qe ? (c < C ? cols[c][q] : q) : 0;
            uint64_t at = ((uint64_t)c * h.qpad + q) * h.sb;
            uint32_t v = nxt * h.sb;
            for (uint32_t i = 0; i < h.sb; ++i) h.table[at + i] = (uint8_t)(v >> (8 * i));
        }
    // Shared-memory placement needs a table that leaves room for the rest of
    // the CTA's shared memory, and a way to address its rows from the staged
    // input: 8-bit class indices (at most 254 classes, 255 marks a byte
    // outside Sigma) or else 16-bit row offsets (kNone16 reserved).
    bool fits16 = (uint64_t)C * h.qpad * h.sb < kNone16;
    h.placement = (tbytes <= kSmemTableMax && (C + 1 <= 255 || fits16)) ? kSmem : kGlobal;
    h.byte_off16.assign(256, kNone16);
    h.byte_off32.assign(256, kNone32);
    for (int b = 0; b < 256; ++b) {
        if (h.byte_class[b] == kNone16) continue;
        uint64_t off = (uint64_t)h.byte_class[b] * h.qpad * h.sb;
        h.byte_off32[b] = (uint32_t)off;
        if (fits16) h.byte_off16[b] = (uint16_t)off;
    }
    // Byte rows (nib_code) when chains visit at most 16 states: every state
    // including q_e fits, or q_e is unreachable (no -1 in delta; chains start
    // in Q, as q_e is excluded from every set).  Row C is the identity.
    bool qe_reachable = false;
    for (uint64_t i = 0; i < (uint64_t)Q * S && !qe_reachable; ++i) qe_reachable = delta[i] < 0;
    const uint32_t live = qe_reachable ? qe : Q;
    if (live <= 16 && h.placement == kSmem) {
        h.nib_rows.assign((size_t)(C + 1) * 16, 0);
        for (uint32_t c = 0; c <= C; ++c)
            for (uint32_t q = 0; q < live; ++q)
                h.nib_rows[(size_t)c * 16 + q] = (uint8_t)nib_code(c < C ? cols[c][q] : q);
    }
    // States per thread: enough chains per thread for latency hiding, few
    // enough that the padding of the last thread of a chunk stays small.
    double mean = std::max(1.0, h.mean_iset);
    h.K = k_for_set_size(mean);
    // a chunk's chains should fit in one tile, ceil(I_max/K) <= kThreads/2, up
    // to K = 16 (launches of Algorithm 2, which match all of Q, raise K
    // further); a chunk with more chains than a tile holds runs its chains in
    // several passes over the chunk (large DFAs)
    while ((std::max(h.imax, 1u) + h.K - 1) / h.K > (uint32_t)kThreads / 2 && h.K < 16) h.K *= 2;
    h.K0 = h.K;
    // single tests of byte-row DFAs are latency-bound when they use the rows (a
    // step is a short dependent chain of permutes that other chains cannot
    // hide): one chain per thread.  Batched launches keep K0.
    if (!h.nib_rows.empty()) h.K = 1;
    *out = std::move(h);
    return DFA_OK;
}

}  // namespace dfam
