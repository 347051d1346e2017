// Device side of the speculative chunked DFA membership test (sm_103a).
//
// A launch covers `ntests` independent membership tests.  Work flows through
// four planning kernels (or k_plan_small, all of them in one CTA, for small
// launches) and one persistent match kernel, all on one stream:
//
//   k_boundaries   (placement only) moves each chunk start within a window to
//                  just after the symbol with the smallest initial set (Sec. 4.2)
//   k_lookahead    (r >= 2 only) per chunk: the Eq. 13 set of r symbols
//   k_count        per chunk: test, reverse-lookahead class, thread slots, work  (Alg. 3, Eq. 11)
//   k_offsets      per-chunk slot offsets, CTA shares of the work, share bounds
//   k_pack (x2)    greedy packing of each share into tiles, tile ranges
//   k_match        persistent: stage chunks, advance every (chunk, state) chain,
//                  compose the chunk maps, combine per test             (Alg. 3, Eqs. 8-9)
//
// Layout of the work: chunk k of a test is matched from every state of its
// initial-state set I_k (the image of its reverse-lookahead symbol's class).
// Each thread advances K of those chains together (one "lane task" per
// (chunk, state) pair, K per thread so the class stream is read once for K
// lookups).  Each CTA owns an equal share of the launch's work (a contiguous
// run of chunks), packed into tiles whose threads fit the CTA; it composes
// the maps of its chunks in order (Eq. 9) into one running map per test;
// tests that span several CTAs are finished by the CTA that completes last.
#include <cuda_runtime.h>

#include <cstdio>
#include <algorithm>

#include "dfa_internal.h"

namespace dfam {

// ------------------------------------------------------------ debug checks

// The debug build (DFA_DEBUG_BOUNDS) checks every state, class, set slot and
// chunk bound before the kernels use it.  A failed check sets bit 1 of the
// test's error word (reported as DFA_EBOUNDS) and the caller skips or clamps
// the access; in the release build the checks compile to nothing.
#ifdef DFA_DEBUG_BOUNDS
// the error word keeps the largest source line of a failed check above bit 8;
// a DFA_EBOUNDS result reports it as its final_state
#define DFAM_OK(cond, err_word) \
    ((cond) ? true : (atomicMax((err_word), ((uint32_t)__LINE__ << 8) | 2u), false))
#else
#define DFAM_OK(cond, err_word) true
#endif

// Result status of a test from its error word: bit 0 = a byte outside Sigma,
// bit 1 = a failed debug check.
__device__ __forceinline__ int32_t status_of(uint32_t err) {
    return (err & 2u) ? DFA_EBOUNDS : (err ? DFA_ESYMBOL : DFA_OK);
}
// final_state of a result: the state, 0 for a failed test, or (debug build,
// DFA_EBOUNDS) the source line of the failed check.
__device__ __forceinline__ uint32_t final_of(uint32_t err, uint32_t s) {
    return err ? ((err & 2u) ? err >> 8 : 0u) : s;
}
// The error word a continuation test inherits from its predecessor's status.
__device__ __forceinline__ uint32_t err_of(int32_t status) {
    return status == DFA_OK ? 0u : (status == DFA_EBOUNDS ? 2u : 1u);
}

// ------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t sa(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t lds_u8(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u8 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t lds_u16(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint4 lds_v4(uint32_t a) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
}
__device__ __forceinline__ void sts_v4(uint32_t a, uint4 v) {
    asm volatile("st.shared.v4.u32 [%0], {%1,%2,%3,%4};"
                 :: "r"(a), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w) : "memory");
}
__device__ __forceinline__ uint32_t ldg_u8(const uint8_t* p) {
    uint32_t v;
    asm volatile("ld.global.nc.u8 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint32_t ldg_u16(const uint8_t* p) {
    uint32_t v;
    asm volatile("ld.global.nc.u16 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}
__device__ __forceinline__ uint32_t ldg_u32(const uint8_t* p) {
    uint32_t v;
    asm volatile("ld.global.nc.u32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

// floor(x / q) given qinv = floor((2^64 - 1) / q): the multiply-high estimate
// is at most 2 below the quotient (division by an invariant integer).
__device__ __forceinline__ uint64_t div_by_recip(uint64_t x, uint64_t q, uint64_t qinv) {
    uint64_t s = __umul64hi(x, qinv);
    uint64_t r = x - s * q;
    if (r >= q) {
        ++s;
        r -= q;
    }
    if (r >= q) ++s;
    return s;
}

// Eq. (6) with unit weights and m states per later chunk (see chunk_start on
// the host): Start(k) = floor(n (m + k - 1) / (m + P - 1)), exact.
__device__ __forceinline__ uint64_t dstart(const DevTest& t, uint32_t k) {
    if (k == 0) return 0;
    if (k >= t.P) return t.n;
    const uint64_t a = (uint64_t)t.m + k - 1, q = (uint64_t)t.m + t.P - 1;
    if (__umul64hi(t.n, a) == 0) return div_by_recip(t.n * a, q, t.qinv);
    const unsigned __int128 num = (unsigned __int128)t.n * a;
    return (uint64_t)(num / q);
}

template <int NTH, typename T>
__device__ __forceinline__ T block_excl_scan(T v, T* tmp, T* total) {
    // tmp: NTH/32 + 1 entries of shared memory
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T w = lane < NTH / 32 ? tmp[lane] : 0, z = w;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            T y = __shfl_up_sync(0xffffffffu, z, o);
            if (lane >= o) z += y;
        }
        if (lane < NTH / 32) tmp[lane] = z - w;
        if (lane == NTH / 32 - 1) tmp[NTH / 32] = z;
    }
    __syncthreads();
    T r = tmp[warp] + x - v;
    if (total) *total = tmp[NTH / 32];
    __syncthreads();
    return r;
}

constexpr int kPlanThreads = 1024;

__device__ __forceinline__ DevTest test_at(const LaunchPlan& lp, uint32_t i) {
    return lp.tests ? lp.tests[i] : lp.test1;
}
__device__ __forceinline__ DevGroup group_at(const LaunchPlan& lp, uint32_t i) {
    return lp.groups ? lp.groups[i] : lp.group1;
}

// ------------------------------------------------------------ planning

__device__ __forceinline__ uint32_t find_test(const LaunchPlan& lp, uint32_t g) {
    uint32_t lo = 0, hi = lp.ntests - 1;
    while (lo < hi) {
        uint32_t mid = (lo + hi + 1) >> 1;
        if (test_at(lp, mid).chunk_base <= g) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Start of chunk k of test t: placed by k_boundaries (Sec. 4.2) when the test
// has a placement window, else Eqs. (6)-(7).
__device__ __forceinline__ uint64_t cstart(const LaunchPlan& lp, const DevTest& t, uint32_t k) {
    if (k == 0) return 0;
    if (k >= t.P) return t.n;
    return t.window ? lp.starts[t.chunk_base + k] : dstart(t, k);
}

// Readable bytes of the string before position st of test t (unbounded for
// a continuation segment, whose predecessor is in the same device buffer).
__device__ __forceinline__ uint64_t bytes_before(const DevTest& t, uint64_t st) {
    return (t.flags & kTestCont) ? (~0ull >> 1) : st;
}

constexpr int kLaWarps = 8;
constexpr int kBndWarps = 8;

// Boundary placement, which Sec. 4.2 suggests: cut the input right after
// symbols with small initial-state sets.  One warp per chunk k >= 1 of a test
// with a window w: among the positions p in [S - w, S + w] around the
// Eqs. (6)-(7) start S, chunk k starts at the one whose preceding byte's class
// has the smallest |I_class| (a byte outside Sigma costs more than any set),
// then the one nearest S, then the smaller p.  The host keeps w at most a
// quarter of the shortest later chunk, so the window lies inside the string
// and placed starts stay increasing.  Each lane scores every 32nd candidate
// (coalesced byte reads, one byte_plan load each); a warp minimum picks p.
__global__ void __launch_bounds__(kBndWarps * 32) k_boundaries(LaunchPlan lp) {
    const int lane = threadIdx.x & 31;
    const uint32_t g = blockIdx.x * kBndWarps + (threadIdx.x >> 5);
    if (g >= lp.ptot) return;  // warp-uniform
    const DevTest t = test_at(lp, find_test(lp, g));
    const uint32_t k = g - t.chunk_base;
    if (t.window == 0 || k == 0) return;
    const uint64_t S = dstart(t, k), w = t.window;
    const uint32_t* bp = lp.dfas[t.dfa].byte_plan;
    const uint8_t* before = t.str - 1;  // before[p] = Str[p - 1]
    // key: |I| (bits 18-34), distance (bits 1-17), past S (bit 0); lower is better
    uint64_t best = ~0ull;
    for (uint64_t p = S - w + (uint64_t)lane; p <= S + w; p += 32) {
        const uint32_t v = __ldg(bp + __ldg(before + p));
        const uint64_t cost = v == kNone32 ? 0x10000u : (v & 0xFFFFu);
        const uint64_t dist = p < S ? S - p : p - S;
        const uint64_t key = (cost << 18) | (dist << 1) | (p > S ? 1u : 0u);
        best = key < best ? key : best;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const uint64_t y = __shfl_xor_sync(0xffffffffu, best, o);
        best = y < best ? y : best;
    }
    if (lane == 0) {
        const uint64_t dist = (best >> 1) & 0x1FFFFu;
        lp.starts[g] = (best & 1u) ? S + dist : S - dist;
    }
}

// r-symbol reverse lookahead (Eq. 13), one warp per chunk: with sigma_1..sigma_j
// the j = min(r, Start(k)) bytes before the chunk, I = delta*(Q, sigma_1..sigma_j)
// minus the excluded states, computed as I_{sigma_1} pushed through
// sigma_2..sigma_j (excluded states are absorbing, so dropping them at every
// step is exact).  A bitmap over Q removes duplicates and yields the set in
// ascending order.  Chunks with j < 2 are left to k_count (start set or one
// symbol).  Shared memory per warp: qe_words bitmap words + vcap set entries.
__global__ void __launch_bounds__(kLaWarps * 32) k_lookahead(LaunchPlan lp, uint32_t qe_words,
                                                          uint32_t set_words) {
    extern __shared__ uint32_t la_sm[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    uint32_t* bm = la_sm + (size_t)w * (qe_words + set_words);
    uint16_t* buf = reinterpret_cast<uint16_t*>(bm + qe_words);
    const uint32_t g = blockIdx.x * kLaWarps + (uint32_t)w;
    if (g >= lp.ptot) return;  // warp-uniform
    const uint32_t ti = find_test(lp, g);
    const DevTest t = test_at(lp, ti);
    if (t.lookahead < 2) return;
    const DevDfa& d = lp.dfas[t.dfa];
    const uint64_t st = cstart(lp, t, g - t.chunk_base);
    const uint64_t avail = bytes_before(t, st);
    const uint32_t j = (uint32_t)(avail < t.lookahead ? avail : t.lookahead);
    if (j < 2) return;
    const DevGroup gr = group_at(lp, t.group);
    uint16_t* out = lp.sets + gr.set_base + (uint64_t)(g - gr.first_chunk) * gr.set_stride;
    const uint8_t* p = t.str + ((int64_t)st - (int64_t)j);
    uint32_t c = d.byte_class[p[0]];
    if (c == kNone16) {
        if (lane == 0) { atomicOr(lp.test_err + ti, 1u); lp.set_size[g] = 0; }
        return;
    }
    uint32_t n = d.iset_off[c + 1] - d.iset_off[c];
    for (uint32_t x = lane; x < n; x += 32) buf[x] = d.iset[d.iset_off[c] + x];
    __syncwarp();
    const uint32_t words = (d.qe + 31) / 32;
    const uint32_t wpl = (words + 31) / 32;  // bitmap words per lane
    for (uint32_t i = 1; i < j; ++i) {
        c = d.byte_class[p[i]];
        if (c == kNone16) {
            if (lane == 0) { atomicOr(lp.test_err + ti, 1u); lp.set_size[g] = 0; }
            return;
        }
        for (uint32_t x = lane; x < words; x += 32) bm[x] = 0;
        __syncwarp();
        const uint8_t* row = d.table + (size_t)c * d.qpad * d.sb;
        for (uint32_t x = lane; x < n; x += 32) {
            const uint32_t s = buf[x];
            const uint32_t nx = d.sb == 1 ? row[s]
                                : (d.sb == 2 ? (uint32_t)(reinterpret_cast<const uint16_t*>(row)[s] >> 1)
                                             : reinterpret_cast<const uint32_t*>(row)[s] >> 2);
            if (!DFAM_OK(nx < d.qe, lp.test_err + ti)) continue;
            if (!d.excluded[nx]) atomicOr(bm + (nx >> 5), 1u << (nx & 31));
        }
        __syncwarp();
        // ascending compaction: lane L owns bitmap words [L*wpl, (L+1)*wpl)
        uint32_t cnt = 0;
        for (uint32_t k = 0; k < wpl; ++k) {
            const uint32_t wi = lane * wpl + k;
            if (wi < words) cnt += __popc(bm[wi]);
        }
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t total = __shfl_sync(0xffffffffu, incl, 31);
        uint32_t pos = incl - cnt;
        __syncwarp();
        for (uint32_t k = 0; k < wpl; ++k) {
            const uint32_t wi = lane * wpl + k;
            if (wi >= words) break;
            uint32_t bits = bm[wi];
            while (bits) {
                const uint32_t b = __ffs(bits) - 1;
                bits &= bits - 1;
                if (DFAM_OK(pos < gr.set_stride, lp.test_err + ti)) buf[pos] = (uint16_t)(wi * 32 + b);
                ++pos;
            }
        }
        n = total;
        if (!DFAM_OK(n <= gr.set_stride, lp.test_err + ti)) n = gr.set_stride;
        __syncwarp();
    }
    for (uint32_t x = lane; x < n; x += 32) out[x] = buf[x];
    if (lane == 0) lp.set_size[g] = n;
}

// Per-chunk packing word: thread slots (bits 0-19: ceil(|I| / K) <= 32768)
// and kOpensTile, set when the chunk starts a new DFA group or the share of a
// new CTA.  A chunk with more slots than a CTA has threads fills a tile of its
// own and runs its chains in several passes.
constexpr uint32_t kOpensTile = 1u << 20;
__device__ __forceinline__ uint32_t word_cost(uint32_t w) { return w & 0xFFFFFu; }

// CTA shares.  The launch's work W (lane-steps: thread slots x chunk length,
// summed over its chunks) is cut into G equal shares, one per CTA of the
// match kernel; chunk g goes to the share holding its midpoint.  With mid2 =
// twice that midpoint (2 x work before g + work of g) the share is
// floor(mid2 * G / (2 W)), so every CTA gets W / G +- one chunk; when W / G is
// below the heaviest chunk's work some CTAs get no chunk.
__device__ __forceinline__ uint32_t cta_of_mid2(uint64_t mid2, uint64_t W, uint32_t G,
                                                uint64_t winv) {
    if (W == 0) return 0;
    uint64_t c;
    if (W < (1ull << 50) && G <= 4096)  // mid2 <= 2W, so mid2 * G < 2^63: 64-bit is exact
        c = div_by_recip(mid2 * G, 2 * W, winv);
    else
        c = (uint64_t)((unsigned __int128)mid2 * G / ((unsigned __int128)W * 2));
    return (uint32_t)(c < G ? c : G - 1);
}

// The reciprocal cta_of_mid2 takes (one real division per thread).
__device__ __forceinline__ uint64_t share_recip(uint64_t W) { return W ? ~0ull / (2 * W) : 0; }

// Per chunk g: owning test, reverse-lookahead class (Algorithm 3, Sec. 4.2)
// and the thread slots it is charged: ceil(|I_k| / K), at least 2.  Writes
// chunk_test, chunk_cls and the packing word; returns in cost[i] and work[i]
// the slots and cost x chunk length (the lane-steps the chunk occupies, used
// to give every CTA an equal share) of chunks g0 .. g0+N-1 (those below
// ptot).  The N chunks go through each step together so their dependent
// global loads (lookahead byte, class, set size) overlap.
template <int N>
__device__ __forceinline__ void chunk_count_n(const LaunchPlan& lp, uint32_t g0, uint32_t* cost,
                                              uint64_t* work) {
    constexpr uint32_t kNoByte = 0x100;
    uint32_t lo[N], b[N], C[N], K[N], dyn[N];
    uint64_t st[N], en[N];
    const uint32_t* bp[N];
    // Two dependent load levels per chunk, issued for all N chunks together:
    // (1) the byte before the chunk, the DFA's fields and the Eq. 13 set size;
    // (2) that byte's class and |I_class| from the DFA's byte_plan.
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const uint32_t g = g0 + i;
        const bool ok = g < lp.ptot;
        lo[i] = ok ? find_test(lp, g) : 0;
        const DevTest t = test_at(lp, lo[i]);
        const DevDfa* d = lp.dfas + t.dfa;
        C[i] = __ldg(&d->C);
        K[i] = __ldg(&d->K);
        bp[i] = (const uint32_t*)__ldg((const unsigned long long*)&d->byte_plan);
        const uint32_t k = g - t.chunk_base;
        st[i] = ok ? cstart(lp, t, k) : 0;
        en[i] = ok ? cstart(lp, t, k + 1) : 0;
        const uint64_t avail = bytes_before(t, st[i]);
        b[i] = (ok && avail && t.lookahead) ? (uint32_t)__ldg(t.str + ((int64_t)st[i] - 1)) : kNoByte;
        // Eq. 13 sets (r >= 2) were sized by k_lookahead
        dyn[i] = (ok && avail >= 2 && t.lookahead >= 2) ? lp.set_size[g] + 1 : 0;
        if (!ok) b[i] = kNoByte;
        if (ok && avail == 0) C[i] |= 0x80000000u;  // chunk 0 (or after empty chunks): start set
        if (ok && !t.lookahead) K[i] |= 0x80000000u;  // Algorithm 2
    }
#pragma unroll
    for (int i = 0; i < N; ++i) {
        const uint32_t g = g0 + i;
        if (g >= lp.ptot) {
            cost[i] = 0;
            work[i] = 0;
            continue;
        }
        const uint32_t Ci = C[i] & 0x7FFFFFFFu, Ki = K[i] & 0x7FFFFFFFu;
        uint32_t cls, size;
        if (C[i] & 0x80000000u) {
            cls = Ci;  // start set {q0}
            size = 1;
        } else if (K[i] & 0x80000000u) {
            cls = Ci + 1;  // all of Q
            size = __ldg(&lp.dfas[test_at(lp, lo[i]).dfa].n_all);
        } else {
            const uint32_t v = __ldg(bp[i] + b[i]);
            if (v == kNone32) {  // a byte outside Sigma: the test fails, the chunk runs from {q0}
                atomicOr(&lp.test_err[lo[i]], 1u);
                cls = Ci;
                size = 1;
            } else if (dyn[i]) {
                cls = dyn_set(Ci);
                size = dyn[i] - 1;
            } else {
                cls = v >> 16;
                size = v & 0xFFFFu;
            }
        }
        if (!DFAM_OK(size <= 65535u && cls <= Ci + 2, &lp.test_err[lo[i]])) {
            size = 1;
            cls = Ci;
        }
        const uint32_t cnt = (size + Ki - 1) / Ki;
        cost[i] = cnt < 2 ? 2 : cnt;
        const DevTest t = test_at(lp, lo[i]);
        // a chunk opens a new DFA group when it is the first chunk of the launch,
        // or the first of a test whose group differs from the previous chunk's
        bool fresh = g == 0;
        if (!fresh && g == t.chunk_base) fresh = test_at(lp, find_test(lp, g - 1)).group != t.group;
        lp.chunk_test[g] = lo[i];
        lp.chunk_cls[g] = (uint16_t)cls;
        lp.cost[g] = cost[i] | (fresh ? kOpensTile : 0u);
        work[i] = (uint64_t)cost[i] * (en[i] - st[i]);
    }
}

// Per-chunk counts, scanned within each block of 1024 chunks: off[g] gets the
// block-local exclusive prefix of thread slots and wk[g] twice the
// block-local midpoint of the chunk's work; bsum/bsumw get the block totals.
__global__ void __launch_bounds__(kPlanThreads) k_count(LaunchPlan lp) {
    __shared__ uint32_t tmp[kPlanThreads / 32 + 1];
    __shared__ uint64_t tmpw[kPlanThreads / 32 + 1];
    const uint32_t g = blockIdx.x * kPlanThreads + threadIdx.x;
    uint32_t cost;
    uint64_t work;
    chunk_count_n<1>(lp, g, &cost, &work);
    uint32_t total;
    uint64_t totalw;
    const uint32_t ex = block_excl_scan<kPlanThreads>(cost, tmp, &total);
    const uint64_t exw = block_excl_scan<kPlanThreads>(work, tmpw, &totalw);
    if (g < lp.ptot) {
        lp.off[g] = ex;
        lp.wk[g] = 2 * exw + work;
    }
    if (threadIdx.x == 0) {
        lp.bsum[blockIdx.x] = total;
        lp.bsumw[blockIdx.x] = totalw;
    }
}

// Share boundaries: share c is chunks [share[c], share[c+1]); a chunk that
// starts a share is marked kOpensTile.  Shares that got no chunk are empty.
// sh_of(g) gives chunk g's share, for the chunks [0, ptot).
template <typename ShareOf>
__device__ __forceinline__ void share_bounds(uint32_t g, uint32_t ptot, uint32_t G, ShareOf sh_of,
                                             uint32_t* share, uint32_t* word) {
    const uint32_t c = sh_of(g);
    const int cp = g ? (int)sh_of(g - 1) : -1;
    if ((int)c != cp) {
        for (int x = cp + 1; x <= (int)c; ++x) share[x] = g;
        *word |= kOpensTile;
    }
    if (g + 1 == ptot)
        for (uint32_t x = c + 1; x <= G; ++x) share[x] = ptot;
}

// Sum of v[0..n) by all threads of a block of NTH threads (tmp: NTH/32+1 entries).
template <int NTH, typename T>
__device__ __forceinline__ T block_sum(const T* v, uint32_t n, T* tmp) {
    T acc = 0;
    for (uint32_t base = 0; base < n; base += NTH) {
        const uint32_t i = base + threadIdx.x;
        T total;
        block_excl_scan<NTH>(i < n ? v[i] : (T)0, tmp, &total);
        acc += total;
    }
    return acc;
}

// Launch-wide prefixes and CTA shares (multi-kernel path).  Every block adds
// the sums of the blocks before it (and needs the launch total W for the
// shares); chunk g gets its share, and a chunk that starts a share records
// the share boundaries and is marked kOpensTile.
__global__ void __launch_bounds__(kPlanThreads) k_offsets(LaunchPlan lp) {
    __shared__ uint32_t tmp[kPlanThreads / 32 + 1];
    __shared__ uint64_t tmpw[kPlanThreads / 32 + 1];
    __shared__ uint32_t cs[kPlanThreads];
    const uint32_t blk = blockIdx.x, g = blk * kPlanThreads + threadIdx.x;
    const uint32_t boff = block_sum<kPlanThreads>(lp.bsum, blk, tmp);
    const uint64_t bwoff = block_sum<kPlanThreads>(lp.bsumw, blk, tmpw);
    const uint32_t total = boff + block_sum<kPlanThreads>(lp.bsum + blk, lp.nblk - blk, tmp);
    const uint64_t W = bwoff + block_sum<kPlanThreads>(lp.bsumw + blk, lp.nblk - blk, tmpw);
    const uint64_t winv = share_recip(W);
    const uint32_t G = lp.grid;
    uint32_t c = 0;
    if (g < lp.ptot) {
        lp.off[g] += boff;
        c = cta_of_mid2(lp.wk[g] + 2 * bwoff, W, G, winv);
        cs[threadIdx.x] = c;
    }
    __syncthreads();
    if (g < lp.ptot) {
        uint32_t w = lp.cost[g];
        // the previous chunk's share: from this block, or recomputed for the first thread
        auto sh_of = [&](uint32_t x) -> uint32_t {
            if (x == g) return c;
            if (x >= blk * kPlanThreads) return cs[x - blk * kPlanThreads];
            return cta_of_mid2(lp.wk[x] + 2 * (bwoff - lp.bsumw[blk - 1]), W, G, winv);
        };
        share_bounds(g, lp.ptot, G, sh_of, lp.share, &w);
        lp.cost[g] = w;
    }
    if (g == 0) lp.off[lp.ptot] = total;
}

// Tile packing.  A tile is a run of consecutive chunks of one DFA group,
// inside one CTA share, whose thread slots fit one CTA (kThreads); each share
// is packed greedily in order by one warp: a chunk opens a new tile when it is
// marked kOpensTile (a new group or share) or would overflow the tile.  The
// CTA that owns a share runs its tiles one after the other, so tile starts
// come only from the shares' contents, never from how the work is split
// among warps.
struct Packer {
    uint32_t cur = 0, tiles = 0;
};

// Greedy pass over the packing words v[0..n) of chunks g0 .. g0+n-1 of a
// share starting at chunk f (every lane runs it; words are read 16 at a time
// with independent loads, then scanned in registers).  With out != nullptr,
// lane 0 writes each tile's first chunk to out[tile index].
__device__ __forceinline__ void pack_words(const uint32_t* v, uint32_t n, uint32_t g0, uint32_t f,
                                           Packer& pk, uint32_t* out) {
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t b = 0; b < n; b += 16) {
        uint32_t x[16];
#pragma unroll
        for (uint32_t i = 0; i < 16; ++i) x[i] = b + i < n ? v[b + i] : 0u;
#pragma unroll
        for (uint32_t i = 0; i < 16; ++i) {
            if (b + i >= n) break;
            const uint32_t g = g0 + b + i, c = word_cost(x[i]);
            if ((x[i] & kOpensTile) || g == f || pk.cur + c > (uint32_t)kThreads) {
                if (out && lane == 0) out[pk.tiles] = g;
                ++pk.tiles;
                pk.cur = 0;
            }
            pk.cur += c;
        }
    }
}

// The same greedy pass run by one thread over a whole share [f, e) of
// shared-memory words (the fused planner gives every share its own thread).
__device__ __forceinline__ uint32_t pack_share(const uint32_t* words, uint32_t f, uint32_t e,
                                               uint32_t* out) {
    uint32_t cur = 0, tiles = 0;
    for (uint32_t g = f; g < e; ++g) {
        const uint32_t x = words[g], c = word_cost(x);
        if ((x & kOpensTile) || g == f || cur + c > (uint32_t)kThreads) {
            if (out) out[tiles] = g;
            ++tiles;
            cur = 0;
        }
        cur += c;
    }
    return tiles;
}

constexpr uint32_t kPackWin = 512;  // packing words one warp stages at a time
constexpr int kPackWarps = 8;

// One warp per share.  Pass 0 packs the share from its words, staged through
// shared memory kPackWin at a time (one coalesced read each), and leaves its
// tile starts in the share's own slice of lp.cost (a tile start never
// overtakes the words still to be read); ntiles[c] gets the count.  Pass 1
// scans the counts (every block for itself), copies each slice to its place
// in tile_first and sets the CTA's tile range; the block of the last share
// also writes the tile count and closes the last tile.
__global__ void __launch_bounds__(kPackWarps * 32) k_pack(LaunchPlan lp, uint32_t pass) {
    __shared__ uint32_t win[kPackWarps][kPackWin];
    __shared__ uint32_t tmp[kPackWarps + 1];
    const uint32_t lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const uint32_t c = blockIdx.x * kPackWarps + wl;
    if (pass == 0) {
        if (c >= lp.grid) return;  // warp-uniform
        const uint32_t f = lp.share[c], e = lp.share[c + 1];
        Packer pk;
        for (uint32_t p0 = f; p0 < e; p0 += kPackWin) {
            const uint32_t p1 = min(p0 + kPackWin, e);
            __syncwarp();
            for (uint32_t i = lane; i < p1 - p0; i += 32) win[wl][i] = lp.cost[p0 + i];
            __syncwarp();
            pack_words(win[wl], p1 - p0, p0, f, pk, lp.cost + f);
        }
        if (lane == 0) lp.ntiles[c] = pk.tiles;
        return;
    }
    // pass 1: the first share of this block starts after the tiles of shares [0, c0)
    const uint32_t c0 = blockIdx.x * kPackWarps;
    const uint32_t before = block_sum<kPackWarps * 32>(lp.ntiles, c0, tmp);
    const uint32_t mine = c < lp.grid ? lp.ntiles[c] : 0;
    uint32_t blk_total;
    const uint32_t wex = block_excl_scan<kPackWarps * 32>(lane == 0 ? mine : 0u, tmp, &blk_total);
    if (c >= lp.grid) return;  // warp-uniform
    const uint32_t base = before + __shfl_sync(0xffffffffu, wex, 0);
    const uint32_t f = lp.share[c];
    for (uint32_t i = lane; i < mine; i += 32) lp.tile_first[base + i] = lp.cost[f + i];
    if (lane == 0) {
        lp.cta_range[2 * c] = base;
        lp.cta_range[2 * c + 1] = base + mine;
        if (c + 1 == lp.grid) {
            *lp.num_tiles = base + mine;
            lp.tile_first[base + mine] = lp.ptot;
        }
    }
}

// All planning steps in one CTA, for launches with at most kSmallPlan chunks
// and kSmallShares CTAs (one launch instead of four on latency-bound calls).
// The packing words, shares and per-share tile counts stay in shared memory;
// thread c packs share c.  Same tiles as the multi-kernel path.
constexpr uint32_t kSmallPlan = 2048;
constexpr uint32_t kSmallShares = 2048;
constexpr uint32_t kSmallPlanSmem = kSmallPlan * 4 + kSmallPlan * 2 + (2 * kSmallShares + 1) * 4;

__global__ void __launch_bounds__(kPlanThreads) k_plan_small(LaunchPlan lp) {
    extern __shared__ uint32_t pw[];                                       // [kSmallPlan] words
    uint16_t* cc = reinterpret_cast<uint16_t*>(pw + kSmallPlan);           // [kSmallPlan] shares
    uint32_t* share = reinterpret_cast<uint32_t*>(cc + kSmallPlan);        // [G + 1]
    uint32_t* cnt = share + kSmallShares + 1;                              // [G]
    __shared__ uint32_t tmp[kPlanThreads / 32 + 1];
    __shared__ uint64_t tmpw[kPlanThreads / 32 + 1];
    const uint32_t G = lp.grid;
    uint32_t carry = 0;
    uint64_t carryw = 0;
    // per-chunk counts and the exclusive scans, one chunk per thread and round;
    // wk[g] keeps twice the chunk's work midpoint until the total is known
    if (!lp.dyn) {  // otherwise k_lookahead ran first and the launch cleared them
        for (uint32_t i = threadIdx.x; i < 2 * lp.ntests; i += kPlanThreads) lp.test_err[i] = 0;
        __syncthreads();
    }
    for (uint32_t base = 0; base < lp.ptot; base += kPlanThreads) {
        const uint32_t g = base + threadIdx.x;
        uint32_t cost;
        uint64_t work;
        chunk_count_n<1>(lp, g, &cost, &work);
        uint32_t total;
        uint64_t totalw;
        const uint32_t ex = block_excl_scan<kPlanThreads>(cost, tmp, &total);
        const uint64_t exw = block_excl_scan<kPlanThreads>(work, tmpw, &totalw);
        if (g < lp.ptot) {
            pw[g] = lp.cost[g];
            lp.off[g] = carry + ex;
            lp.wk[g] = 2 * (carryw + exw) + work;
        }
        carry += total;
        carryw += totalw;
    }
    if (threadIdx.x == 0) lp.off[lp.ptot] = carry;
    __syncthreads();
    const uint64_t winv = share_recip(carryw);
    for (uint32_t g = threadIdx.x; g < lp.ptot; g += kPlanThreads)
        cc[g] = (uint16_t)cta_of_mid2(lp.wk[g], carryw, G, winv);
    __syncthreads();
    for (uint32_t g = threadIdx.x; g < lp.ptot; g += kPlanThreads)
        share_bounds(g, lp.ptot, G, [&](uint32_t x) { return (uint32_t)cc[x]; }, share, pw + g);
    __syncthreads();
    for (uint32_t c = threadIdx.x; c < G; c += kPlanThreads)
        cnt[c] = pack_share(pw, share[c], share[c + 1], nullptr);
    __syncthreads();
    uint32_t acc = 0;
    for (uint32_t base = 0; base < G; base += kPlanThreads) {
        const uint32_t i = base + threadIdx.x;
        const uint32_t v = i < G ? cnt[i] : 0;
        uint32_t total;
        const uint32_t ex = block_excl_scan<kPlanThreads>(v, tmp, &total);
        if (i < G) cnt[i] = acc + ex;
        acc += total;
    }
    if (threadIdx.x == 0) {
        *lp.num_tiles = acc;
        lp.tile_first[acc] = lp.ptot;
    }
    for (uint32_t c = threadIdx.x; c < G; c += kPlanThreads) {
        const uint32_t n = pack_share(pw, share[c], share[c + 1], lp.tile_first + cnt[c]);
        lp.cta_range[2 * c] = cnt[c];
        lp.cta_range[2 * c + 1] = cnt[c] + n;
    }
}

// ------------------------------------------------------------ matching

struct ChunkMeta {
    const uint8_t* ptr;     // first byte of the chunk
    const uint16_t* init;   // its initial-state set (ascending)
    uint32_t len;           // bytes
    uint32_t test;
    uint16_t toff;          // first thread (tile-local) of the chunk
    uint16_t cls;           // set index (class, start set, all of Q, or dyn_set)
    uint16_t cnt;           // threads actually used: ceil(|I|/K)
    uint16_t size;          // |I|
    uint8_t lo_slack;       // min(bytes of the string before the chunk, 255)
    uint8_t hi_slack;       // min(bytes of the string after the chunk, 255)
    uint8_t pad_[6];
};
static_assert(sizeof(ChunkMeta) == 40, "ChunkMeta layout");

// Shared-memory carve-up of k_match (byte offsets, all 16-byte aligned).
// Launches with sets larger than kSmemVcap keep the running map and its
// domain in global memory (LaunchPlan::big_maps) and hold here only one flag
// bit per map entry, used while a chunk's chains run in several passes.
struct SmemLayout {
    uint32_t table, boff, stage, lmap, linit, vmap, vdom, vflag, meta, misc, desc, total;
};

__host__ __device__ inline uint32_t align16(uint32_t x) { return (x + 15u) & ~15u; }

__host__ __device__ inline SmemLayout smem_layout(uint32_t table_cap, uint32_t kmax, uint32_t vcap,
                                                  uint32_t stage_bytes) {
    SmemLayout L;
    L.table = 0;
    L.boff = align16(table_cap);
    L.stage = L.boff + 1024;
    L.lmap = L.stage + 2 * stage_bytes;
    L.linit = L.lmap + align16(kThreads * kmax * 2);
    const bool big = vcap > kSmemVcap;
    L.vmap = L.linit + align16(kThreads * kmax * 2);
    L.vdom = L.vmap + (big ? 0u : align16(vcap * 2));
    L.vflag = L.vdom + (big ? 0u : align16(vcap * 2));
    L.meta = L.vflag + (big ? align16((vcap + 31) / 32 * 4) : 0u);
    L.misc = L.meta + kMaxChunksPerTile * sizeof(ChunkMeta);
    L.desc = L.misc + 64;
    L.total = L.desc + align16(sizeof(DevDfa));
    return L;
}

// misc words
enum { M_MAXLEN = 0, M_LAST = 1, M_DFA = 2, M_CELL = 3 };

// Advance K chains of one chunk over one staged segment of S positions.
// Shared-memory table, 16-bit row offsets, StBytes-sized entries.
template <int K, int SB>
__device__ __forceinline__ void run_smem(uint32_t (&s)[K], uint32_t tb, uint32_t stage_addr, int S) {
    for (int j = 0; j < S; j += 8) {
        const uint4 w = lds_v4(stage_addr + 2 * j);
        const uint32_t words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
#pragma unroll
            for (int half = 0; half < 2; ++half) {
                const uint32_t row = tb + (half ? (words[h] >> 16) : (words[h] & 0xFFFFu));
#pragma unroll
                for (int u = 0; u < K; ++u) s[u] = SB == 1 ? lds_u8(row + s[u]) : lds_u16(row + s[u]);
            }
        }
    }
}

// Shared-memory table with an 8-bit class stream: one 16-byte read covers 16
// steps; the row of class c starts at tb + c * rowbytes.
template <int K, int SB>
__device__ __forceinline__ void run_smem8(uint32_t (&s)[K], uint32_t tb, uint32_t rowbytes,
                                          uint32_t stage_addr, int S) {
    for (int j = 0; j < S; j += 16) {
        const uint4 w = lds_v4(stage_addr + j);
        const uint32_t words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const uint32_t row = tb + ((words[h] >> (8 * b)) & 0xFFu) * rowbytes;
#pragma unroll
                for (int u = 0; u < K; ++u) s[u] = SB == 1 ? lds_u8(row + s[u]) : lds_u16(row + s[u]);
            }
        }
    }
}

// Same with the table read through L2 (32-bit row offsets, 4 per 16 bytes).
template <int K, int SB>
__device__ __forceinline__ void run_global(uint32_t (&s)[K], const uint8_t* tbl, uint32_t stage_addr,
                                           int S) {
    for (int j = 0; j < S; j += 4) {
        const uint4 w = lds_v4(stage_addr + 4 * j);
        const uint32_t words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const uint8_t* row = tbl + words[h];
#pragma unroll
            for (int u = 0; u < K; ++u)
                s[u] = SB == 1 ? ldg_u8(row + s[u]) : (SB == 2 ? ldg_u16(row + s[u]) : ldg_u32(row + s[u]));
        }
    }
}

// One chain step on a byte row (DFAs with at most 16 live states): the row's
// 16 bytes hold the codes (nib_code) of the next states; the code's low
// nibble selects a byte of each 8-byte half, and its bit 7 picks the half.
// Only byte 0 of the result is meaningful, and it is the next code.  (A
// third permute in place of the select measured slower: permutes issue at
// half rate.)
__device__ __forceinline__ uint32_t nib_step(const uint4& row, uint32_t code) {
    const uint32_t lo = __byte_perm(row.x, row.y, code);
    const uint32_t hi = __byte_perm(row.z, row.w, code);
    // all ones when bit 7 of the code is set: a permute in sign-replicating mode
    // (selector nibbles 0x8: byte 0's sign bit in every byte), issued beside the
    // two row permutes, so no predicate sits on the chain's dependent path
    uint32_t half;
    asm("prmt.b32 %0, %1, 0, 0x8888;" : "=r"(half) : "r"(code));
    return (lo & ~half) | (hi & half);
}

// Advance K chains over one staged segment of S positions with byte rows in
// shared memory at tb.  The stage holds 8-bit class indices (CLS8; row =
// class * 16) or 16-bit row byte offsets.  The rows depend only on the
// input, so they are loaded two groups of four steps ahead of the chains that
// use them (the stage entry, then the row: two dependent loads per step).
template <int K, bool CLS8, bool DEEP>
__device__ __forceinline__ void run_nib(uint32_t (&s)[K], uint32_t tb, uint32_t stage_addr, int S) {
    auto row_addr = [&](int j) -> uint32_t {
        return CLS8 ? tb + lds_u8(stage_addr + (uint32_t)j) * 16u
                    : tb + lds_u16(stage_addr + 2u * (uint32_t)j);
    };
    if (K > 2 || !DEEP) {
        // more chains per thread hide the loads themselves (and the kernel
        // variant with 40 registers has no room for more rows): one group ahead
        uint4 cur[4], nxt[4];
#pragma unroll
        for (int g = 0; g < 4; ++g) cur[g] = lds_v4(row_addr(g));
        for (int j = 0; j < S; j += 4) {
            const int jn = j + 4 < S ? j + 4 : j;
#pragma unroll
            for (int g = 0; g < 4; ++g) nxt[g] = lds_v4(row_addr(jn + g));
#pragma unroll
            for (int g = 0; g < 4; ++g)
#pragma unroll
                for (int u = 0; u < K; ++u) s[u] = nib_step(cur[g], s[u]);
#pragma unroll
            for (int g = 0; g < 4; ++g) cur[g] = nxt[g];
        }
        return;
    }
    uint4 r0[4], r1[4], r2[4];
#pragma unroll
    for (int g = 0; g < 4; ++g) r0[g] = lds_v4(row_addr(g));
#pragma unroll
    for (int g = 0; g < 4; ++g) r1[g] = lds_v4(row_addr(4 + g));
    for (int j = 0; j < S; j += 4) {
        const int jn = j + 8 < S ? j + 8 : S - 4;  // past the end: reload the last group
#pragma unroll
        for (int g = 0; g < 4; ++g) r2[g] = lds_v4(row_addr(jn + g));
#pragma unroll
        for (int g = 0; g < 4; ++g)
#pragma unroll
            for (int u = 0; u < K; ++u) s[u] = nib_step(r0[g], s[u]);
#pragma unroll
        for (int g = 0; g < 4; ++g) {
            r0[g] = r1[g];
            r1[g] = r2[g];
        }
    }
}

// One tile's chains for a given K: load initial states, run all segments
// (staging is done by the caller through `stage_fn`), store the final states
// into the tile-local map (plain state ids).
struct TileCtx {
    uint32_t tb;          // shared address of the table (smem placement)
    const uint8_t* gtbl;  // global table (L2 placement)
    uint32_t stage0;      // shared address of stage buffer 0
    uint32_t lmap;        // shared address of the tile map (final states per chain)
    uint32_t linit;       // shared address of the chains' initial states
    int sb, placement;
    int ci, r, active;    // my chunk, rank within chunk, has work
    int S;                // staged positions per chunk per segment
    uint32_t stage_bytes; // bytes of one stage buffer
};

// ------------------------------------------------------------ staging

// Convert bytes [pos, pos+16) of a chunk to 16 stage entries (class indices
// or row offsets) and store them at dst.  The bytes come from two aligned
// 16-byte loads and a funnel shift (adjacent threads take adjacent groups of
// the same chunk, so the loads coalesce); near the ends of the string, where
// an aligned 16-byte read could leave it, they are read one by one.  Positions
// past the chunk end get the identity row; bytes outside Sigma flag the test
// and also get the identity row.
template <uint32_t FMT>
__device__ __forceinline__ uint32_t stage_entry(uint32_t b, bool valid, uint32_t boff, uint32_t id_off,
                                                bool& bad, bool& oob) {
    uint32_t x;
    if (FMT == kOff32) {
        asm volatile("ld.shared.u32 %0, [%1];" : "=r"(x) : "r"(boff + 4 * b));
        if (x == kNone32) { bad |= valid; x = id_off; }
    } else if (FMT == kCls8) {
        x = lds_u8(boff + b);
        if (x == 0xFFu) { bad |= valid; x = id_off; }
    } else {
        x = lds_u16(boff + 2 * b);
        if (x == kNone16) { bad |= valid; x = id_off; }
    }
#ifdef DFA_DEBUG_BOUNDS
    if (x > id_off) { oob = true; x = id_off; }  // a row past the identity row
#endif
    return valid ? x : id_off;
}

template <uint32_t FMT>
__device__ __forceinline__ void stage_group(const ChunkMeta& m, uint32_t pos, uint32_t dst,
                                            uint32_t boff, uint32_t id_off, uint32_t* test_err) {
    uint32_t v[4] = {0, 0, 0, 0};
    uint32_t nvalid = 0;
    if (pos < m.len) {
        nvalid = min(16u, m.len - pos);
        const uint8_t* a = m.ptr + pos;
        const uint32_t d = (uint32_t)((uintptr_t)a & 15u);
        // fast path: the two aligned 16-byte vectors around [a, a+16) lie inside the string
        const bool fast = (pos + m.lo_slack >= d) && (pos + 32u <= m.len + m.hi_slack + d);
        if (fast) {
            const uint4* al = reinterpret_cast<const uint4*>(a - d);
            const uint4 x0 = __ldg(al), x1 = __ldg(al + 1);
            const uint32_t q = d >> 2, r = (d & 3u) * 8u;
            uint32_t sel[5];
            sel[0] = q == 0 ? x0.x : (q == 1 ? x0.y : (q == 2 ? x0.z : x0.w));
            sel[1] = q == 0 ? x0.y : (q == 1 ? x0.z : (q == 2 ? x0.w : x1.x));
            sel[2] = q == 0 ? x0.z : (q == 1 ? x0.w : (q == 2 ? x1.x : x1.y));
            sel[3] = q == 0 ? x0.w : (q == 1 ? x1.x : (q == 2 ? x1.y : x1.z));
            sel[4] = q == 0 ? x1.x : (q == 1 ? x1.y : (q == 2 ? x1.z : x1.w));
#pragma unroll
            for (int i = 0; i < 4; ++i) v[i] = __funnelshift_r(sel[i], sel[i + 1], r);
        } else {
            uint64_t lo = 0, hi = 0;
            for (uint32_t j = 0; j < nvalid; ++j) {
                const uint64_t byte = __ldg(a + j);
                if (j < 8) lo |= byte << (8 * j); else hi |= byte << (8 * (j - 8));
            }
            v[0] = (uint32_t)lo; v[1] = (uint32_t)(lo >> 32);
            v[2] = (uint32_t)hi; v[3] = (uint32_t)(hi >> 32);
        }
    }
    bool bad = false, oob = false;
    if (FMT == kCls8) {
        uint32_t w[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            uint32_t word = 0;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint32_t j = 4 * i + k;
                word |= stage_entry<FMT>((v[i] >> (8 * k)) & 0xFFu, j < nvalid, boff, id_off, bad, oob) << (8 * k);
            }
            w[i] = word;
        }
        sts_v4(dst, make_uint4(w[0], w[1], w[2], w[3]));
    } else if (FMT == kOff16) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            uint32_t w[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const uint32_t j = 8 * h + 2 * i;
                const uint32_t src = v[j >> 2] >> (8 * (j & 3));
                w[i] = stage_entry<FMT>(src & 0xFFu, j < nvalid, boff, id_off, bad, oob) |
                       (stage_entry<FMT>((src >> 8) & 0xFFu, j + 1 < nvalid, boff, id_off, bad, oob) << 16);
            }
            sts_v4(dst + 16 * h, make_uint4(w[0], w[1], w[2], w[3]));
        }
    } else {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            uint32_t w[4];
#pragma unroll
            for (int k = 0; k < 4; ++k)
                w[k] = stage_entry<FMT>((v[i] >> (8 * k)) & 0xFFu, 4u * i + k < nvalid, boff, id_off, bad, oob);
            sts_v4(dst + 16 * i, make_uint4(w[0], w[1], w[2], w[3]));
        }
    }
    if (bad) atomicOr(test_err + m.test, 1u);
    if (oob) atomicOr(test_err + m.test, 2u);
}

template <uint32_t FMT>
__device__ void stage_segment(const ChunkMeta* meta, int nch, int S, int seg, uint32_t stage,
                              uint32_t boff, uint32_t id_off, uint32_t* test_err) {
    const int groups = S / 16;
    const int items = nch * groups;
    for (int it = threadIdx.x; it < items; it += kThreads) {
        const int ci = it / groups, q = it - ci * groups;
        const ChunkMeta m = meta[ci];
        const uint32_t pos = (uint32_t)seg * (uint32_t)S + 16u * (uint32_t)q;
        const uint32_t dst = stage + (uint32_t)(ci * S + 16 * q) * stage_esz(FMT);
        stage_group<FMT>(m, pos, dst, boff, id_off, test_err);
    }
}

// DEEP: the kernel variant has the registers to load byte rows two groups ahead.
template <int K, bool DEEP>
__device__ void tile_chains(const DevDfa& d, const ChunkMeta* meta, int nch, uint32_t maxlen,
                            const TileCtx& c, uint32_t boff, uint32_t* test_err,
                            uint16_t* dbg_maps, uint32_t dbg_stride, uint32_t g0) {
    uint32_t s[K];
    const uint32_t fmt = d.stage_fmt;
    const uint32_t sh = d.sb == 4 ? 2 : (d.sb == 2 ? 1 : 0);
    const bool nib = d.nib != 0;
    if (c.active) {
        const ChunkMeta m = meta[c.ci];
        const uint32_t size = m.size;
#pragma unroll
        for (int u = 0; u < K; ++u) {
            uint32_t slot = (uint32_t)c.r * K + u;
            if (slot >= size) slot = (uint32_t)c.r * K;  // padding chain: repeat the first
            uint32_t init = m.init[slot];
            if (!DFAM_OK(init < d.qe && (!nib || init < 16u), test_err + m.test)) init = 0;
            s[u] = nib ? nib_code(init) : init << sh;
            asm volatile("st.shared.u16 [%0], %1;" :: "r"(c.linit + 2u * ((uint32_t)(threadIdx.x) * K + u)),
                         "h"((uint16_t)init) : "memory");
        }
    } else {
#pragma unroll
        for (int u = 0; u < K; ++u) s[u] = 0;
    }
    const uint32_t rowbytes = nib ? 16u : d.qpad * d.sb;
    const uint32_t id_off = fmt == kCls8 ? d.C : d.C * rowbytes;  // the identity row
    const int nseg = (int)((maxlen + c.S - 1) / c.S);
    const uint32_t esz = stage_esz(fmt);
    for (int seg = 0; seg < nseg; ++seg) {
        const uint32_t stage = c.stage0 + (uint32_t)(seg & 1) * c.stage_bytes;
        if (fmt == kCls8) stage_segment<kCls8>(meta, nch, c.S, seg, stage, boff, id_off, test_err);
        else if (fmt == kOff16) stage_segment<kOff16>(meta, nch, c.S, seg, stage, boff, id_off, test_err);
        else stage_segment<kOff32>(meta, nch, c.S, seg, stage, boff, id_off, test_err);
        __syncthreads();
        if (c.active) {
            const uint32_t my = stage + (uint32_t)(c.ci * c.S) * esz;
            if (nib) {
                if (fmt == kCls8) run_nib<K, true, DEEP>(s, c.tb, my, c.S);
                else run_nib<K, false, DEEP>(s, c.tb, my, c.S);
            } else if (fmt == kCls8) {
                if (d.sb == 1) run_smem8<K, 1>(s, c.tb, rowbytes, my, c.S);
                else run_smem8<K, 2>(s, c.tb, rowbytes, my, c.S);
            } else if (fmt == kOff16) {
                if (d.sb == 1) run_smem<K, 1>(s, c.tb, my, c.S);
                else run_smem<K, 2>(s, c.tb, my, c.S);
            } else {
                if (d.sb == 1) run_global<K, 1>(s, c.gtbl, my, c.S);
                else if (d.sb == 2) run_global<K, 2>(s, c.gtbl, my, c.S);
                else run_global<K, 4>(s, c.gtbl, my, c.S);
            }
        }
        // the next segment stages into the other buffer, so one barrier per segment suffices
    }
    if (c.active) {
        const ChunkMeta m = meta[c.ci];
#pragma unroll
        for (int u = 0; u < K; ++u) {
            uint32_t v = nib ? nib_state(s[u] & 0xFFu) : s[u] >> sh;
            if (!DFAM_OK(v < d.qe, test_err + m.test)) v = 0;
            asm volatile("st.shared.u16 [%0], %1;" :: "r"(c.lmap + 2u * ((uint32_t)(threadIdx.x) * K + u)),
                         "h"((uint16_t)v) : "memory");
            // inspection output: L_k[j] = delta*(j, chunk k) for j in I_k (Sec. 4.1)
            const uint32_t slot = (uint32_t)c.r * K + u;
            if (dbg_maps && slot < m.size)
                dbg_maps[(size_t)(g0 + c.ci) * dbg_stride + m.init[slot]] = (uint16_t)v;
        }
    }
}

// Stages segment maps i0 .. i0+nb-1 of test t (CTAs b0 + i0 + j) into sm, vw
// 16-byte vectors each (a segment map is seg_stride entries, a multiple of 8);
// a CTA without a share contributes the identity.  `valid` (nb bytes of shared
// memory) first records which CTAs hold a part of the test; the maps are then
// copied with asynchronous 16-byte global-to-shared copies, so every thread
// has all of its copies in flight at once and holds none of the data in
// registers.  The caller's barrier after the call publishes the stage.
__device__ __forceinline__ void stage_seg_maps(const LaunchPlan& lp, uint32_t t, uint32_t b0,
                                               uint32_t i0, uint32_t nb, uint32_t vw, uint4* sm,
                                               uint8_t* valid) {
    for (uint32_t j = threadIdx.x; j < nb; j += kThreads) {
        // a CTA between the test's first and last CTA either holds a part
        // of it or got no share at all (then its map is the identity)
        const uint32_t cb = b0 + i0 + j;
        valid[j] = __ldcg(lp.cta_range + 2 * cb) != __ldcg(lp.cta_range + 2 * cb + 1) ? 1 : 0;
    }
    __syncthreads();
    const uint32_t total = nb * vw;
    for (uint32_t k = threadIdx.x; k < total; k += kThreads) {
        const uint32_t j = k / vw, w = k - j * vw;
        if (valid[j]) {
            const uint4* src = reinterpret_cast<const uint4*>(
                lp.seg_vals + (size_t)(b0 + i0 + j + t) * lp.seg_stride) + w;
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                         :: "r"(sa(sm + k)), "l"(src) : "memory");
        } else {
            const uint32_t e = 8 * w;  // entries e .. e+7 of the identity
            sm[k] = make_uint4(e | ((e + 1) << 16), (e + 2) | ((e + 3) << 16),
                               (e + 4) | ((e + 5) << 16), (e + 6) | ((e + 7) << 16));
        }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
}

// Shared memory a combine keeps for the valid flags of one batch of maps.
constexpr uint32_t kCombineBatchMax = 1024;

constexpr uint32_t kMapStatesPerThread = (kMaxSmallQe + kThreads - 1) / kThreads;

// Map test: compose the whole segment maps (Eq. 9) for every state at once;
// thread x follows states x, x + kThreads, ... through the maps in order.
__device__ void combine_test_map(const LaunchPlan& lp, uint32_t t, const DevTest& tt,
                                 const DevDfa& d, uint32_t b0, uint32_t nseg, uint4* sm,
                                 uint8_t* valid, uint32_t per, uint32_t vw) {
    const uint32_t qe = d.qe;
    if (qe > kMapStatesPerThread * kThreads) {  // the host never pipelines such DFAs
        if (threadIdx.x == 0) {
            dfa_result_t r{};
            r.status = DFA_EINVAL;
            lp.results[tt.out] = r;
        }
        __syncthreads();
        return;
    }
    uint32_t cur[kMapStatesPerThread];
#pragma unroll
    for (uint32_t i = 0; i < kMapStatesPerThread; ++i) cur[i] = threadIdx.x + i * kThreads;
    for (uint32_t i0 = 0; i0 < nseg; i0 += per) {
        const uint32_t nb = min(per, nseg - i0);
        __syncthreads();
        stage_seg_maps(lp, t, b0, i0, nb, vw, sm, valid);
        __syncthreads();
        const uint16_t* m = reinterpret_cast<const uint16_t*>(sm);
        for (uint32_t j = 0; j < nb; ++j) {
#pragma unroll
            for (uint32_t i = 0; i < kMapStatesPerThread; ++i)
                if (cur[i] < qe) cur[i] = m[(size_t)j * 8 * vw + cur[i]];
        }
    }
    uint16_t* out = lp.maps + (size_t)tt.out * lp.map_stride;
#pragma unroll
    for (uint32_t i = 0; i < kMapStatesPerThread; ++i) {
        const uint32_t x = threadIdx.x + i * kThreads;
        if (x < qe) out[x] = (uint16_t)cur[i];
    }
    if (threadIdx.x == 0) {
        dfa_result_t r;
        r.final_state = 0;
        r.accept = 0;
        r.reserved[0] = r.reserved[1] = r.reserved[2] = 0;
        r.status = status_of(atomicOr(lp.test_err + t, 0u));
        lp.results[tt.out] = r;
    }
    __syncthreads();
}

// Final state of test t from its segment maps (slots b + t for b in
// [first_cta, last_cta]), applied in order to q0: Eq. (8) segment by segment.
// Each segment map is dense over Q (identity outside its domain), so one
// step is one lookup; the maps are staged through shared memory (`buf`,
// buf_bytes) in batches so the dependent chain runs at shared-memory latency.
// Called by all threads of the CTA.
__device__ void combine_test(const LaunchPlan& lp, uint32_t t, uint8_t* buf, uint32_t buf_bytes,
                             uint32_t* cell) {
    const DevTest tt = test_at(lp, t);
    const DevDfa& d = lp.dfas[tt.dfa];
    const uint32_t b0 = __ldcg(lp.first_cta + t), b1 = __ldcg(lp.last_cta + t);
    const uint32_t nseg = b1 - b0 + 1;
    [[maybe_unused]] const uint32_t qe = d.qe;  // (read by the debug build's checks)
    const uint32_t vw = lp.seg_stride / 8;  // 16-byte vectors per map
    // maps per batch; the last kCombineBatchMax bytes of buf hold the batch's valid flags
    const uint32_t per = buf_bytes > kCombineBatchMax
                             ? min(kCombineBatchMax, (buf_bytes - kCombineBatchMax) / (16 * vw)) : 0u;
    uint4* sm = reinterpret_cast<uint4*>(buf);
    uint8_t* valid = buf + buf_bytes - kCombineBatchMax;
    // a continuation segment starts from the previous segment's final state;
    // that launch ran earlier on the same stream, so its result is complete
    const bool cont = (tt.flags & kTestCont) != 0;
    if (tt.flags & kTestMap) {
        combine_test_map(lp, t, tt, d, b0, nseg, sm, valid, per, vw);
        return;
    }
    if (threadIdx.x == 0) *cell = cont ? lp.results[tt.out].final_state : d.q0;
    if (per == 0 && threadIdx.x == 0) {
        // maps larger than the staging buffer: thread 0 reads them in place
        uint32_t s = *cell;
        for (uint32_t j = 0; j < nseg; ++j) {
            const uint32_t cb = b0 + j;
            if (__ldcg(lp.cta_range + 2 * cb) == __ldcg(lp.cta_range + 2 * cb + 1)) continue;
            s = __ldcg(lp.seg_vals + (size_t)(cb + t) * lp.seg_stride + s);
            if (!DFAM_OK(s < qe, lp.test_err + t)) s = 0;
        }
        *cell = s;
    }
    for (uint32_t i0 = 0; i0 < nseg && per; i0 += per) {
        const uint32_t nb = min(per, nseg - i0);
        __syncthreads();
        stage_seg_maps(lp, t, b0, i0, nb, vw, sm, valid);
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t s = *cell;
            const uint16_t* m = reinterpret_cast<const uint16_t*>(sm);
            for (uint32_t j = 0; j < nb; ++j) {
                s = m[(size_t)j * 8 * vw + s];
                if (!DFAM_OK(s < qe, lp.test_err + t)) s = 0;
            }
            *cell = s;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t s = *cell;
        dfa_result_t r;
        const uint32_t err = atomicOr(lp.test_err + t, 0u) | (cont ? err_of(lp.results[tt.out].status) : 0u);
        r.final_state = final_of(err, s);
        r.accept = err ? 0 : d.accept[s];
        r.reserved[0] = r.reserved[1] = r.reserved[2] = 0;
        r.status = status_of(err);
        lp.results[tt.out] = r;
    }
    __syncthreads();
}

// KMAX: largest chains-per-thread of the launch; MINB: CTAs per SM the
// register budget is sized for (3 for K <= 4: more warps hide the shared-
// memory load latency when each thread carries few chains).
template <int KMAX, int MINB>
__global__ void __launch_bounds__(kThreads, MINB) k_match(LaunchPlan lp, uint32_t kmax) {
    extern __shared__ __align__(16) uint8_t sm[];
    const SmemLayout L = smem_layout(lp.smem_table_cap, kmax, lp.vcap, lp.stage_bytes);
    ChunkMeta* meta = reinterpret_cast<ChunkMeta*>(sm + L.meta);
    uint32_t* misc = reinterpret_cast<uint32_t*>(sm + L.misc);
    // the running map and its domain: shared memory, or this CTA's slice of
    // big_maps when the launch's sets are larger than kSmemVcap
    uint16_t* vmap = lp.vmap_stride ? lp.big_maps + (size_t)blockIdx.x * 2 * lp.vmap_stride
                                    : reinterpret_cast<uint16_t*>(sm + L.vmap);
    uint16_t* vdom = lp.vmap_stride ? vmap + lp.vmap_stride : reinterpret_cast<uint16_t*>(sm + L.vdom);
    uint32_t* vflag = reinterpret_cast<uint32_t*>(sm + L.vflag);
    const uint16_t* lmap = reinterpret_cast<const uint16_t*>(sm + L.lmap);
    const uint16_t* linit = reinterpret_cast<const uint16_t*>(sm + L.linit);
    const int tid = threadIdx.x;

    const uint32_t b = blockIdx.x;
    // CTA b owns tiles [t0, t1): its share of the launch's work (chunk_cta);
    // a CTA without a share returns at once
    const uint32_t t0 = lp.cta_range[2 * b], t1 = lp.cta_range[2 * b + 1];
    if (t0 >= t1) return;
    // the done-flags of multi-pass composition start cleared (shared memory
    // holds whatever an earlier kernel left there); each multi-pass chunk
    // clears the flags it set
    if (lp.vmap_stride)
        for (uint32_t w = tid; w < (lp.vcap + 31) / 32; w += kThreads) vflag[w] = 0;
    const uint32_t c_lo = lp.tile_first[t0], c_hi = lp.tile_first[t1];

    int cur_dfa = -1;
    DevDfa& d = *reinterpret_cast<DevDfa*>(sm + L.desc);  // the current tile's DFA
    // running segment (CTA-uniform)
    int cur_test = -1;
    uint32_t seg_first = 0, seg_n = 0, seg_cls = 0, nD = 0;

    // Finishes the running segment of cur_test.  It runs when the next chunk
    // belongs to another test, which may already be in a tile of another DFA,
    // so it reads the test's own DFA descriptor, never the shared-memory copy.
    auto end_segment = [&]() {
        const DevTest tt = test_at(lp, (uint32_t)cur_test);
        const DevDfa& td = lp.dfas[tt.dfa];
        const bool covered = tt.chunk_base >= c_lo && tt.chunk_base + tt.P <= c_hi &&
                             !(tt.flags & kTestCont);
        if (covered) {
            // the segment is the whole test, started at chunk 0 from {q0}: V[0] is the answer
            if (tid == 0) {
                const uint32_t s = vmap[0];
                const uint32_t err = atomicOr(lp.test_err + cur_test, 0u);
                dfa_result_t r;
                r.final_state = final_of(err, s);
                r.accept = err ? 0 : td.accept[s];
                r.reserved[0] = r.reserved[1] = r.reserved[2] = 0;
                r.status = status_of(err);
                lp.results[tt.out] = r;
            }
            return;
        }
        // publish this CTA's part of the test as a dense map over Q: identity
        // outside the segment's domain (those states are excluded, hence fixed)
        const size_t slot = (size_t)b + (size_t)cur_test;
        uint16_t* dense = lp.seg_vals + slot * lp.seg_stride;
        const uint32_t tqe = td.qe;
        for (uint32_t s = tid; s < tqe; s += kThreads) dense[s] = (uint16_t)s;
        __syncthreads();
        for (uint32_t x = tid; x < nD; x += kThreads)
            if (DFAM_OK(vdom[x] < tqe && vmap[x] < tqe, lp.test_err + cur_test)) dense[vdom[x]] = vmap[x];
        if (tid == 0) {
            lp.seg_hdr[slot * 4 + 0] = seg_first;
            lp.seg_hdr[slot * 4 + 1] = seg_n;
            lp.seg_hdr[slot * 4 + 2] = seg_cls;
            lp.seg_hdr[slot * 4 + 3] = nD;
            if (seg_first == tt.chunk_base) lp.first_cta[cur_test] = b;
            if (seg_first + seg_n == tt.chunk_base + tt.P) lp.last_cta[cur_test] = b;
        }
        __syncthreads();
        if (tid == 0) {
            __threadfence();
            const uint32_t old = atomicAdd(lp.arrived + cur_test, seg_n);
            misc[M_LAST] = (old + seg_n == tt.P) ? 1u : 0u;
        }
        __syncthreads();
        if (misc[M_LAST]) {
            __threadfence();
            // the stage buffers are free during the composition phase
            combine_test(lp, (uint32_t)cur_test, sm + L.stage, 2 * lp.stage_bytes, misc + M_CELL);
        }
        __syncthreads();
    };

    for (uint32_t t = t0; t < t1; ++t) {
        const uint32_t gA = lp.tile_first[t], gB = lp.tile_first[t + 1];
        const int nch = (int)(gB - gA);
        const uint32_t test0 = lp.chunk_test[gA];
        const int di = (int)test_at(lp, test0).dfa;
        if (di != cur_dfa) {
            __syncthreads();
            if (tid < (int)(sizeof(DevDfa) / 4))
                reinterpret_cast<uint32_t*>(&d)[tid] = reinterpret_cast<const uint32_t*>(lp.dfas + di)[tid];
            __syncthreads();
            if (lp.no_nib) {  // this launch matches byte-row DFAs from their tables
                if (tid == 0) d.nib = 0;
                __syncthreads();
            }
            if (d.placement == kSmem) {
                const uint4* src = reinterpret_cast<const uint4*>(d.nib ? d.nib_rows : d.table);
                uint4* dst = reinterpret_cast<uint4*>(sm + L.table);
                const uint32_t n16 = d.nib ? d.C + 1 : (d.table_bytes + 15) / 16;
                for (uint32_t i = tid; i < n16; i += kThreads) dst[i] = __ldg(src + i);
                if (d.stage_fmt == kCls8) {
                    uint8_t* bc = sm + L.boff;
                    for (int i = tid; i < 256; i += kThreads) {
                        const uint32_t c = __ldg(d.byte_class + i);
                        bc[i] = c == kNone16 ? (uint8_t)0xFF : (uint8_t)c;
                    }
                } else {
                    uint16_t* bo = reinterpret_cast<uint16_t*>(sm + L.boff);
                    const uint16_t* src16 = d.nib ? d.nib_off16 : d.byte_off16;
                    for (int i = tid; i < 256; i += kThreads) bo[i] = __ldg(src16 + i);
                }
            } else {
                uint32_t* bo = reinterpret_cast<uint32_t*>(sm + L.boff);
                for (int i = tid; i < 256; i += kThreads) bo[i] = __ldg(d.byte_off32 + i);
            }
            cur_dfa = di;
        }
        // chunk metadata
        if (tid == 0) misc[M_MAXLEN] = 0;
        __syncthreads();
        const uint32_t off0 = lp.off[gA];
        for (int i = tid; i < nch; i += kThreads) {
            const uint32_t g = gA + (uint32_t)i;
            const uint32_t te = lp.chunk_test[g];
            const DevTest tt = test_at(lp, te);
            const uint32_t k = g - tt.chunk_base;
            uint64_t st = cstart(lp, tt, k), en = cstart(lp, tt, k + 1);
            uint32_t cls = lp.chunk_cls[g];
            if (!DFAM_OK(st <= en && en <= tt.n && en - st < (1ull << 31), lp.test_err + te)) en = st;
            if (!DFAM_OK(cls <= d.C + 2 && (cls < d.C + 2 || lp.dyn), lp.test_err + te)) cls = d.C;
            ChunkMeta m;
            uint32_t size;
            if (cls == dyn_set(d.C)) {
                const DevGroup gr = group_at(lp, tt.group);
                size = lp.set_size[g];
                m.init = lp.sets + gr.set_base + (uint64_t)(g - gr.first_chunk) * gr.set_stride;
            } else {
                size = d.iset_off[cls + 1] - d.iset_off[cls];
                m.init = d.iset + d.iset_off[cls];
            }
            if (!DFAM_OK(size <= lp.vcap, lp.test_err + te)) size = 1;
            m.size = (uint16_t)size;
            m.ptr = tt.str + st;
            m.len = (uint32_t)(en - st);
            m.test = te;
            m.toff = (uint16_t)(lp.off[g] - off0);
            m.cls = (uint16_t)cls;
            m.cnt = (uint16_t)((size + d.K - 1) / d.K);
            const uint64_t avail = bytes_before(tt, st);
            m.lo_slack = (uint8_t)(avail < 255 ? avail : 255);
            m.hi_slack = (uint8_t)(tt.n - en < 255 ? tt.n - en : 255);
            meta[i] = m;
            atomicMax(misc + M_MAXLEN, m.len);
        }
        __syncthreads();
        const uint32_t maxlen = misc[M_MAXLEN];

        // A tile is either a run of chunks whose chains fit its threads, or one
        // chunk with more chains than that (large DFAs): the chunk's chains then
        // run in passes of kThreads threads, each pass re-staging the chunk.
        const uint32_t cnt0 = meta[0].cnt;
        const uint32_t passes = (nch == 1 && cnt0 > (uint32_t)kThreads)
                                    ? (cnt0 + kThreads - 1) / kThreads : 1u;
        bool fresh = false;  // the multi-pass chunk opened a new segment (CTA-uniform)
        for (uint32_t pass = 0; pass < passes; ++pass) {
        TileCtx c;
        if (passes > 1) {
            c.ci = 0;
            c.r = tid + (int)(pass * kThreads);
            c.active = c.r < (int)cnt0;
        } else {
            // my chunk: last ci with toff <= tid
            int lo = 0, hi = nch - 1;
            while (lo < hi) {
                int mid = (lo + hi + 1) >> 1;
                if (meta[mid].toff <= tid) lo = mid; else hi = mid - 1;
            }
            c.ci = lo;
            c.r = tid - meta[lo].toff;
            c.active = c.r < (int)meta[lo].cnt;
        }
        const uint32_t esz = stage_esz(d.stage_fmt);
        // positions per chunk per segment: a multiple of 16, at most what the
        // stage buffer holds for this tile's chunks; the segments then share the
        // longest chunk evenly, so the last one is not mostly identity padding
        const int quant = 16;
        int S = (int)(lp.stage_bytes / ((uint32_t)nch * esz)) / quant * quant;
        S = S < quant ? quant : (S > kMaxSegLen ? kMaxSegLen : S);
        if (maxlen > 0) {
            const uint32_t nseg = (maxlen + (uint32_t)S - 1) / (uint32_t)S;
            S = (int)(((maxlen + nseg - 1) / nseg + quant - 1) / quant * quant);
        }
        c.S = S;
        c.stage_bytes = lp.stage_bytes;
        c.tb = sa(sm + L.table);
        c.gtbl = d.table;
        c.stage0 = sa(sm + L.stage);
        c.lmap = sa(sm + L.lmap);
        c.linit = sa(sm + L.linit);
        c.sb = (int)d.sb;
        c.placement = (int)d.placement;
        const uint32_t boff = sa(sm + L.boff);
        uint16_t* dbg = lp.dbg_maps;
        const uint32_t dst_ = lp.qe_max;
        constexpr bool kDeep = KMAX >= 8;
        if (d.K == 1) tile_chains<1, kDeep>(d, meta, nch, maxlen, c, boff, lp.test_err, dbg, dst_, gA);
        else if (d.K == 2) tile_chains<2, kDeep>(d, meta, nch, maxlen, c, boff, lp.test_err, dbg, dst_, gA);
        else if (KMAX >= 8 && d.K == 4)
            tile_chains<(KMAX >= 8 ? 4 : 2), kDeep>(d, meta, nch, maxlen, c, boff, lp.test_err, dbg, dst_, gA);
        else if (KMAX >= 16 && d.K == 8)
            tile_chains<(KMAX >= 16 ? 8 : 2), kDeep>(d, meta, nch, maxlen, c, boff, lp.test_err, dbg, dst_, gA);
        else tile_chains<KMAX, kDeep>(d, meta, nch, maxlen, c, boff, lp.test_err, dbg, dst_, gA);
        __syncthreads();

        if (passes > 1) {
            // Eq. (9) for one pass of a multi-pass chunk: the pass holds the chains
            // of I_k[lo, hi) (tile-local slot x - lo).  Every entry of the running
            // map is composed with the chunk exactly once, by the pass that holds
            // its entering state's slot (vflag marks it done); excluded states
            // (no slot) stay fixed.
            const ChunkMeta m = meta[0];
            const uint32_t lo = pass * (uint32_t)kThreads * d.K;
            const uint32_t hi = min((uint32_t)m.size, lo + (uint32_t)kThreads * d.K);
            if (pass == 0 && (int)m.test != cur_test) {
                if (cur_test >= 0) end_segment();
                cur_test = (int)m.test;
                seg_first = gA;
                seg_n = 0;
                seg_cls = m.cls;
                nD = m.size;
                fresh = true;
            }
            if (fresh) {
                for (uint32_t x = lo + tid; x < hi; x += kThreads) {
                    vmap[x] = lmap[x - lo];
                    vdom[x] = linit[x - lo];
                }
            } else {
                const uint16_t* pos = d.pos + (size_t)m.cls * d.qe;
                for (uint32_t x = tid; x < nD; x += kThreads) {
                    if ((vflag[x >> 5] >> (x & 31)) & 1u) continue;
                    if (!DFAM_OK(vmap[x] < d.qe, lp.test_err + m.test)) continue;
                    const uint32_t p = __ldg(pos + vmap[x]);
                    if (p != kNone16 && p >= lo && p < hi) {
                        vmap[x] = lmap[p - lo];
                        atomicOr(vflag + (x >> 5), 1u << (x & 31));
                    }
                }
            }
            __syncthreads();
            if (pass + 1 == passes) {
                ++seg_n;
                for (uint32_t w = tid; w < (nD + 31) / 32; w += kThreads) vflag[w] = 0;
            }
            __syncthreads();
            continue;
        }

        // Compose the tile's chunk maps, in order, into the running map of each
        // test (Eq. 9).  Thread x owns entries x, x+kThreads, ... of the running map.
        for (int i = 0; i < nch; ++i) {
            const ChunkMeta m = meta[i];
            const uint32_t base = (uint32_t)m.toff * d.K;
            if ((int)m.test != cur_test) {
                if (cur_test >= 0) end_segment();
                cur_test = (int)m.test;
                seg_first = gA + (uint32_t)i;
                seg_n = 0;
                seg_cls = m.cls;
                nD = m.size;
                for (uint32_t x = tid; x < nD; x += kThreads) {
                    vmap[x] = lmap[base + x];
                    vdom[x] = linit[base + x];
                }
            } else if (m.cls == dyn_set(d.C)) {
                // the chunk's set came from r >= 2 lookahead symbols: find the
                // entering state's slot by binary search in its initial states
                const uint16_t* keys = linit + base;
                for (uint32_t x = tid; x < nD; x += kThreads) {
                    const uint32_t v = vmap[x];
                    uint32_t lo = 0, hi = m.size;
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi) >> 1;
                        if (keys[mid] < v) lo = mid + 1; else hi = mid;
                    }
                    if (lo < m.size && keys[lo] == v) vmap[x] = lmap[base + lo];
                }
            } else {
                const uint16_t* pos = d.pos + (size_t)m.cls * d.qe;
                for (uint32_t x = tid; x < nD; x += kThreads) {
                    const uint32_t v = vmap[x];
                    if (!DFAM_OK(v < d.qe, lp.test_err + m.test)) continue;
                    const uint32_t p = __ldg(pos + v);
                    if (p != kNone16 &&
                        DFAM_OK(p < m.size && base + p < (uint32_t)kThreads * kmax, lp.test_err + m.test))
                        vmap[x] = lmap[base + p];
                }
            }
            ++seg_n;
        }
        __syncthreads();
        }  // passes
    }
    if (cur_test >= 0) end_segment();
}

// ------------------------------------------------------------ host side

// CTAs per SM the match kernel aims for: 3 when every DFA of the launch
// uses K <= 4 (the kernel variant then fits 3 x 512 threads in registers),
// else 2; `want` overrides it (1-3).
uint32_t match_target_ctas(uint32_t kmax, uint32_t want) {
    uint32_t t = kmax <= 4 ? 3u : 2u;
    if (want >= 1 && want <= t) t = want;
    return t;
}

// Smallest stage buffer for stage entries of esz bytes: a tile's
// kMaxChunksPerTile chunks each stage at least 16 positions (and at least
// 8 KB, below which segments get too short).  32-bit row offsets need 16 KB.
__host__ __device__ constexpr uint32_t min_stage_bytes(uint32_t esz) {
    return kMaxChunksPerTile * 16u * esz > 8192u ? kMaxChunksPerTile * 16u * esz : 8192u;
}
static_assert(min_stage_bytes(4) == 16u * 1024u && min_stage_bytes(1) == 8192u, "stage floor");

// Shared memory of k_match and the stage-buffer size: the largest stage
// (min_stage_bytes(esz_max) to 64 KB per buffer) that lets `target` CTAs
// share an SM, else fewer CTAs.  esz_max is the widest stage entry of the
// launch's DFAs.  A launch whose tables are all read through L2 takes the
// smallest stage instead: the shared memory it leaves to L1 caches the hot
// table rows.
uint32_t match_smem_bytes(uint32_t table_cap, uint32_t kmax, uint32_t vcap, uint32_t esz_max,
                          uint32_t* stage_bytes, uint32_t target) {
    const uint32_t per_sm = 228u * 1024u, reserved = 1024u, min_stage = min_stage_bytes(esz_max);
    if (table_cap == 0) {
        *stage_bytes = min_stage;
        return smem_layout(table_cap, kmax, vcap, min_stage).total;
    }
    for (uint32_t ctas = target; ctas >= 1; --ctas) {
        for (uint32_t sb = 64u * 1024u; sb >= min_stage; sb -= 2048u) {
            if (ctas * (smem_layout(table_cap, kmax, vcap, sb).total + reserved) <= per_sm) {
                *stage_bytes = sb;
                return smem_layout(table_cap, kmax, vcap, sb).total;
            }
        }
    }
    *stage_bytes = min_stage;
    return smem_layout(table_cap, kmax, vcap, min_stage).total;
}

// Per-device properties the launches need; the kernel attributes are set once
// per device when they are first read (thread-safe).
struct DevProps {
    bool ready = false;
    uint32_t sms = 0;          // streaming multiprocessors
    uint32_t smem_optin = 0;   // largest dynamic shared memory per CTA
    uint32_t smem_per_sm = 0;  // shared memory per SM
};
constexpr int kMaxDevices = 64;
static DevProps g_props[kMaxDevices];
static std::mutex g_props_mu;

static const DevProps* dev_props() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> g(g_props_mu);
    DevProps& p = g_props[dev];
    if (p.ready) return &p;
    int sms = 0, optin = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) !=
            cudaSuccess ||
        sms < 1 || optin < 1 || per_sm < 1)
        return nullptr;
    // k_lookahead's per-warp bitmap and set buffer for the largest DFA (4096 states)
    const int la_max = kLaWarps * (4096 / 32 + 4096 / 2) * 4;
    // The match kernels may take up to the opt-in maximum per launch: set once,
    // so plans prepared in any order (batch parts, concurrent server batches)
    // launch with whatever shared memory each needs.  The split between shared
    // memory and L1 is chosen per launch (carveout_pct).
    if (cudaFuncSetAttribute(k_lookahead, cudaFuncAttributeMaxDynamicSharedMemorySize, la_max) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_plan_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             kSmallPlanSmem) != cudaSuccess ||
        cudaFuncSetAttribute(k_match<16, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_match<8, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) !=
            cudaSuccess ||
        cudaFuncSetAttribute(k_match<4, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin) !=
            cudaSuccess)
        return nullptr;
    p.sms = (uint32_t)sms;
    p.smem_optin = (uint32_t)optin;
    p.smem_per_sm = (uint32_t)per_sm;
    p.ready = true;
    return &p;
}

template <int KMAX, int MINB>
static int grid_for(const DevProps& p, uint32_t smem, uint32_t* grid) {
    if (smem > p.smem_optin) return DFA_ECUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_match<KMAX, MINB>, kThreads,
                                                      smem) != cudaSuccess ||
        per_sm < 1)
        return DFA_ECUDA;
    *grid = p.sms * (uint32_t)per_sm;
    return DFA_OK;
}

uint32_t device_sms() {
    const DevProps* p = dev_props();
    return p ? p->sms : 0u;
}

int match_grid(uint32_t smem, uint32_t kmax, uint32_t* grid) {
    const DevProps* p = dev_props();
    if (!p) return DFA_ECUDA;
    if (kmax > 8) return grid_for<16, 2>(*p, smem, grid);
    if (kmax > 4) return grid_for<8, 2>(*p, smem, grid);
    return grid_for<4, 3>(*p, smem, grid);
}

// Eq. (8) over the segments of one string: seg_res[0] is the first
// segment's result, segments 1 .. nseg-1 are map tests.
__global__ void k_compose_segments(const dfa_result_t* seg_res, const uint16_t* maps,
                                   uint32_t stride, uint32_t nseg, const uint8_t* accept,
                                   dfa_result_t* out) {
    if (threadIdx.x != 0) return;
    uint32_t s = seg_res[0].final_state;
    uint32_t err = err_of(seg_res[0].status);
    for (uint32_t i = 1; i < nseg; ++i) {
        err |= err_of(seg_res[i].status);
        if (!err) s = maps[(size_t)i * stride + s];
    }
    dfa_result_t r;
    r.final_state = final_of(err, s);
    r.accept = err ? 0 : accept[s];
    r.reserved[0] = r.reserved[1] = r.reserved[2] = 0;
    r.status = status_of(err);
    *out = r;
}

int launch_compose_segments(const dfa_result_t* seg_res, const uint16_t* maps, uint32_t stride,
                            uint32_t nseg, const uint8_t* accept, dfa_result_t* out, void* st) {
    k_compose_segments<<<1, 32, 0, static_cast<cudaStream_t>(st)>>>(seg_res, maps, stride, nseg,
                                                                    accept, out);
    return cudaPeekAtLastError() == cudaSuccess ? DFA_OK : DFA_ECUDA;
}

// Every kernel of a launch runs with one shared-memory carve-out: what the
// match kernel's CTAs per SM need (a per-launch hint).  The rest of the SM's
// unified L1/shared storage stays L1, which caches input sectors, descriptors
// and L2-placed tables; without the hint the split would follow the kernel's
// dynamic shared memory limit.  One value for all kernels of the launch
// spares the SMs a reconfiguration between them.
static uint32_t carveout_pct(const LaunchPlan& lp, uint32_t smem) {
    const DevProps* p = dev_props();
    if (!p) return 100u;
    const uint32_t resident = lp.waves > 1 ? lp.grid / lp.waves : lp.grid;
    const uint32_t per_sm = (resident + p->sms - 1) / p->sms;
    const uint32_t need = std::max(per_sm * (smem + 1024u), kSmallPlanSmem + 1024u);
    return std::min(100u, (need * 100u + p->smem_per_sm - 1) / p->smem_per_sm);
}

template <typename... Params, typename... Args>
static cudaError_t launch_ex(void (*kernel)(Params...), uint32_t grid, uint32_t block, uint32_t smem,
                             cudaStream_t st, uint32_t pct, Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributePreferredSharedMemoryCarveout;
    attr[0].val.sharedMemCarveout = pct;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

uint32_t launch_kernel_count(uint32_t ptot, uint32_t grid, bool dyn, bool bnd) {
    return (ptot <= kSmallPlan && grid <= kSmallShares ? 2u : 5u) + (dyn ? 1u : 0u) +
           (bnd ? 1u : 0u);
}

// Issue the whole launch on `st`: memsets of the per-test counters, the
// planning kernels (k_boundaries only for tests with a placement window,
// k_lookahead only for r >= 2) and the match kernel.
// With plan_only the match kernel is skipped.
int launch_plan(const LaunchPlan& lp, uint32_t kmax, uint32_t smem, cudaStream_t st,
                uint32_t* kernels, void* ev_begin, void* ev_end, bool plan_only) {
    const uint32_t nb = lp.nblk;
    const bool small = lp.ptot <= kSmallPlan && lp.grid <= kSmallShares;
    // test_err and arrived (adjacent) start at zero; k_plan_small clears them
    // itself unless k_lookahead, which may flag a test, runs first
    if ((!small || lp.dyn) &&
        cudaMemsetAsync(lp.test_err, 0, sizeof(uint32_t) * lp.ntests * 2, st) != cudaSuccess)
        return DFA_ECUDA;
    uint32_t nk = launch_kernel_count(lp.ptot, lp.grid, lp.dyn != 0, lp.bnd != 0);
    const uint32_t pct = carveout_pct(lp, smem);
    int e = 0;  // launch errors (cudaError_t values OR-ed: nonzero = failed)
    if (lp.bnd)
        e |= launch_ex(k_boundaries, (lp.ptot + kBndWarps - 1) / kBndWarps, kBndWarps * 32, 0, st,
                       pct, lp);
    if (lp.dyn) {
        const uint32_t qe_words = (lp.qe_max + 31) / 32, set_words = (lp.vcap + 1) / 2;
        const uint32_t la_smem = kLaWarps * (qe_words + set_words) * 4;
        e |= launch_ex(k_lookahead, (lp.ptot + kLaWarps - 1) / kLaWarps, kLaWarps * 32, la_smem, st, pct,
                  lp, qe_words, set_words);
    }
    if (small) {
        e |= launch_ex(k_plan_small, 1, kPlanThreads, kSmallPlanSmem, st, pct, lp);
    } else {
        const uint32_t pblocks = (lp.grid + kPackWarps - 1) / kPackWarps;
        e |= launch_ex(k_count, nb, kPlanThreads, 0, st, pct, lp);
        e |= launch_ex(k_offsets, nb, kPlanThreads, 0, st, pct, lp);
        e |= launch_ex(k_pack, pblocks, kPackWarps * 32, 0, st, pct, lp, 0u);
        e |= launch_ex(k_pack, pblocks, kPackWarps * 32, 0, st, pct, lp, 1u);
    }
    if (plan_only) {
        if (kernels) *kernels = nk - 1;
        return e == 0 && cudaPeekAtLastError() == cudaSuccess ? DFA_OK : DFA_ECUDA;
    }
    if (ev_begin) cudaEventRecord(static_cast<cudaEvent_t>(ev_begin), st);
    if (kmax > 8) e |= launch_ex(k_match<16, 2>, lp.grid, kThreads, smem, st, pct, lp, kmax);
    else if (kmax > 4) e |= launch_ex(k_match<8, 2>, lp.grid, kThreads, smem, st, pct, lp, kmax);
    else e |= launch_ex(k_match<4, 3>, lp.grid, kThreads, smem, st, pct, lp, kmax);
    if (ev_end) cudaEventRecord(static_cast<cudaEvent_t>(ev_end), st);
    if (kernels) *kernels = nk;
    return e == 0 && cudaPeekAtLastError() == cudaSuccess ? DFA_OK : DFA_ECUDA;
}

}  // namespace dfam
