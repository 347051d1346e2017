// Several DFAs on one input string, with the input staged once for all of
// them.  Sec. 5 of the paper stores the tables of several DFAs side by side
// in one array (SBase) and converts the input once to symbol indices (IBase)
// that every DFA reads; this file is the GPU form of that arrangement.
//
// Each DFA of a group is matched by Algorithm 3 with one reverse-lookahead
// symbol, on chunk starts shared by the whole group (Eqs. 6-7 with unit
// weights and m = 1), and its chunk maps are combined by Eqs. 8-9, so its
// answer is the one dfa_match gives for it alone.
//
// Joint classes.  The group re-encodes every table over the common refinement
// of the DFAs' byte classes: bytes b and b' share a joint class iff they share
// a class in every DFA (or are outside Sigma in the same DFAs).  The input is
// then staged once, as 8-bit joint-class indices, and every DFA's table has
// one row per joint class (plus the identity row that pads chunk tails).
//
// Kernels (one stream):
//   k_group_plan   one CTA: per chunk the thread slots of its G items (one per
//                  DFA: ceil(|I|/K) threads), the launch's work prefix and the
//                  CTA share of each chunk (equal shares of slots x length)
//   k_group_match  persistent: each CTA takes its share of chunks in tiles
//                  whose items fit 512 threads; stages a tile's chunks once,
//                  runs every item's chains from the shared stage, composes
//                  each DFA's chunk maps in order (Eq. 9), publishes one map
//                  per DFA; the last CTA to finish applies them (Eq. 8).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "dfa_internal.h"

namespace dfam {
namespace grp {

constexpr uint32_t kMaxDfas = 16;            // DFAs per group
constexpr uint32_t kMaxQe = 4096;            // |Q|+1 per DFA (16-bit entries hold 2 x state)
constexpr uint32_t kMaxJoint = 255;          // joint classes; the identity row is index J <= 255
constexpr uint32_t kTableMax = 160u * 1024u; // all joint tables (each CTA holds them all)
constexpr uint32_t kVcapMax = 8192;          // sum over the DFAs of their largest set
constexpr uint32_t kMaxChunks = 1u << 18;    // P per launch
constexpr uint32_t kGThreads = 512;           // threads per CTA of k_group_match
constexpr uint32_t kMaxTileChunks = 256;     // chunks per tile
constexpr uint32_t kPlanThreads = 1024;
constexpr uint32_t kMinChunk = 512;          // shortest default chunk (bytes)
constexpr uint32_t kTilesPerCta = 8;         // default P aims for about this many tiles per CTA
constexpr uint32_t kMaxSeg = 2048;           // longest staged segment per chunk (positions)
constexpr uint32_t kMinStage = kMaxTileChunks * 16;  // 256 chunks x 16 positions x 1 byte
constexpr uint32_t kStartSet = 256;          // item class marker: chunk entered in q0 ({q0})
constexpr uint64_t kMaxLen = 1ull << 46;     // n * k of Eq. (6) stays below 2^64

// One DFA of a group as the kernels see it (64 bytes).
struct GDfa {
    const uint32_t* iset_off;  // the DFA's own CSR of initial-state sets (set C = {q0})
    const uint16_t* iset;
    const uint16_t* pos;       // [(C+2) * qe]: index of state s in set c, kNone16 if absent
    const uint8_t* accept;     // [qe]
    uint32_t qe, q0, C;
    uint32_t qpad;             // entries per joint-table row
    uint32_t tbl_off;          // byte offset of its joint table in the group's table image
    uint32_t vcap;             // largest set (incl. the start set)
    uint32_t pad_[2];
};
static_assert(sizeof(GDfa) == 64, "GDfa layout");

// Per launch (kernel parameter).
struct GPlan {
    const GDfa* gd;
    const uint32_t* jinfo;    // [G * 256]: (class << 16) | |I_class| of DFA g for joint class j
    const uint16_t* jmap;     // [256]: byte -> joint class, bit 15 set if some DFA has it outside Sigma
    const uint16_t* jbad;     // [256]: joint class -> mask of the DFAs that have it outside Sigma
    const uint8_t* tables;    // joint tables, tbytes in all
    const uint8_t* str;
    uint64_t n;
    uint32_t G, J, P, K, grid, tbytes, stage_bytes, vcap_sum, seg_stride, qe_max;
    uint32_t* share;          // [grid + 1]: first chunk of each CTA share
    uint32_t* cshare;         // [P]: CTA share of each chunk (planner scratch)
    uint32_t* err;            // [G]: error word of each DFA's test (bit 0: byte outside Sigma)
    uint32_t* arrived;        // [1]
    uint16_t* seg_maps;       // [grid * G * seg_stride]: each CTA's map of each DFA, dense over Q
    dfa_result_t* results;    // [G]
    unsigned long long* work; // optional [1]: lookups of the launch
    uint16_t* dbg;            // optional [G * P * qe_max]: chunk maps L_k
    // continuation of a longer string whose earlier bytes precede str on the
    // device (chunk 0 takes the set of its lookahead byte str[-1], not {q0});
    // with out_maps the launch publishes, per DFA g, the state map of its
    // whole string, out_maps[g * seg_stride + x] = delta*(x, str), instead of
    // a final state (results get only the status)
    uint32_t cont;
    uint16_t* out_maps;
};

// ------------------------------------------------------------ device helpers

#ifdef DFA_DEBUG_BOUNDS
// as in the match kernel of the single-DFA path: the error word keeps the
// largest source line of a failed check above bit 8, bit 1 marks the failure
#define GRP_OK(cond, err_word) \
    ((cond) ? true : (atomicMax((err_word), ((uint32_t)__LINE__ << 8) | 2u), false))
#else
#define GRP_OK(cond, err_word) true
#endif

__device__ __forceinline__ uint32_t g_sa(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t g_lds_u8(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u8 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint32_t g_lds_u16(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}
__device__ __forceinline__ uint4 g_lds_v4(uint32_t a) {
    uint4 v;
    asm volatile("ld.shared.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(a));
    return v;
}
__device__ __forceinline__ void g_sts_v4(uint32_t a, uint4 v) {
    asm volatile("st.shared.v4.u32 [%0], {%1,%2,%3,%4};"
                 :: "r"(a), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w) : "memory");
}

// Status and final state of a test from its error word (bit 0: a byte
// outside Sigma, bit 1: a failed debug check whose line sits above bit 8).
__device__ __forceinline__ int32_t g_status(uint32_t err) {
    return (err & 2u) ? DFA_EBOUNDS : (err ? DFA_ESYMBOL : DFA_OK);
}
__device__ __forceinline__ uint32_t g_final(uint32_t err, uint32_t s) {
    return err ? ((err & 2u) ? err >> 8 : 0u) : s;
}

// Start of chunk k of n bytes in P chunks: Eq. (6) with unit weights and
// m = 1, floor(n k / P) (n k < 2^64 because n < 2^46 and k <= 2^18).
__device__ __forceinline__ uint64_t g_start(uint64_t n, uint32_t P, uint32_t k) {
    return k >= P ? n : (n * (uint64_t)k) / P;
}

// Set of DFA g for a chunk whose lookahead class is jc (kStartSet: {q0}):
// (set index << 16) | |I|.
__device__ __forceinline__ uint32_t g_set(const GPlan& p, const GDfa& d, uint32_t g, uint32_t jc) {
    if (jc == kStartSet) return (d.C << 16) | 1u;
    return __ldg(p.jinfo + g * 256u + jc);
}

__device__ __forceinline__ uint32_t g_slots(uint32_t size, uint32_t K) {
    const uint32_t c = (size + K - 1) / K;
    return c ? c : 1u;
}

// Lookahead class of chunk k: the joint class of the byte before it, or
// kStartSet for a chunk that starts the string (a continuation's string
// starts after the bytes of the earlier segments).
__device__ __forceinline__ uint32_t g_lookahead(const GPlan& p, const uint16_t* jmap, uint32_t k,
                                                uint64_t st) {
    if (k == 0 || st == 0) return p.cont ? (jmap[__ldg(p.str - 1)] & 0xFFu) : kStartSet;
    return jmap[__ldg(p.str + st - 1)] & 0xFFu;
}

// ------------------------------------------------------------ planner

// One CTA.  Thread t takes chunks [P t / 1024, P (t+1) / 1024): their thread
// slots (sum over the DFAs of ceil(|I|/K), at least 1 each) times their
// length is their work; a block scan gives each chunk's work prefix, and
// chunk k goes to CTA share floor(mid2 * grid / (2 W)), mid2 being twice its
// work midpoint, so every CTA gets W / grid +- one chunk.  The shares are
// monotone in k (the rounding of the product is monotone too), hence
// contiguous; share[b] is the first chunk of share b.
__global__ void __launch_bounds__(kPlanThreads) k_group_plan(GPlan p) {
    __shared__ uint16_t s_jmap[256];
    __shared__ unsigned long long s_w[kPlanThreads / 32], s_l[kPlanThreads / 32];
    __shared__ unsigned long long s_total[2];
    const uint32_t t = threadIdx.x, lane = t & 31u, warp = t >> 5;
    for (uint32_t i = t; i < 256; i += kPlanThreads) s_jmap[i] = p.jmap[i];
    __syncthreads();
    const uint32_t k0 = (uint32_t)((uint64_t)p.P * t / kPlanThreads);
    const uint32_t k1 = (uint32_t)((uint64_t)p.P * (t + 1) / kPlanThreads);
    auto chunk_cost = [&](uint32_t k, unsigned long long* lookups) -> unsigned long long {
        const uint64_t st = g_start(p.n, p.P, k), en = g_start(p.n, p.P, k + 1);
        const uint32_t jc = g_lookahead(p, s_jmap, k, st);
        uint32_t slots = 0;
        unsigned long long sz = 0;
        for (uint32_t g = 0; g < p.G; ++g) {
            const uint32_t info = g_set(p, p.gd[g], g, jc);
            slots += g_slots(info & 0xFFFFu, p.K);
            sz += info & 0xFFFFu;
        }
        if (lookups) *lookups += sz * (en - st);
        return (unsigned long long)slots * (en - st);
    };
    unsigned long long w = 0, l = 0;
    for (uint32_t k = k0; k < k1; ++k) w += chunk_cost(k, &l);
    // block exclusive scan of w, block sum of l
    unsigned long long incl = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= (uint32_t)o) incl += v;
    }
    unsigned long long lsum = l;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_down_sync(0xFFFFFFFFu, lsum, o);
    if (lane == 31) s_w[warp] = incl;
    if (lane == 0) s_l[warp] = lsum;
    __syncthreads();
    if (warp == 0) {
        unsigned long long v = s_w[lane], x = v, lv = s_l[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= (uint32_t)o) x += y;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lv += __shfl_down_sync(0xFFFFFFFFu, lv, o);
        s_w[lane] = x - v;  // exclusive prefix of the warp totals
        if (lane == 31) s_total[0] = x;
        if (lane == 0) s_total[1] = lv;
    }
    __syncthreads();
    const unsigned long long W = s_total[0];
    unsigned long long base = s_w[warp] + incl - w;
    const double scale = W ? (double)p.grid / (2.0 * (double)W) : 0.0;
    for (uint32_t k = k0; k < k1; ++k) {
        const unsigned long long c = chunk_cost(k, nullptr);
        const double x = (double)(2 * base + c) * scale;
        uint32_t sh = (uint32_t)x;
        if (sh >= p.grid) sh = p.grid - 1;
        p.cshare[k] = sh;
        base += c;
    }
    __syncthreads();  // cshare of every chunk is visible to the block
    for (uint32_t k = k0; k < k1; ++k) {
        const uint32_t cur = p.cshare[k];
        const uint32_t prev_end = k ? p.cshare[k - 1] + 1 : 0u;
        for (uint32_t s = prev_end; s <= cur; ++s) p.share[s] = k;
        if (k + 1 == p.P)
            for (uint32_t s = cur + 1; s <= p.grid; ++s) p.share[s] = p.P;
    }
    if (t == 0 && p.work) *p.work = s_total[1];
}

// ------------------------------------------------------------ match kernel

struct GItem {                // one (chunk, DFA) pair of a tile: 16 bytes
    const uint16_t* init;     // its initial-state set
    uint16_t toff;            // first thread (tile-local)
    uint16_t cnt;             // threads with chains: ceil(|I| / K)
    uint16_t size;            // |I|
    uint16_t cls;             // set index in the DFA (for pos)
};
static_assert(sizeof(GItem) == 16, "GItem layout");

struct GChunk {               // one chunk of a tile: 16 bytes
    uint64_t start;
    uint32_t len;
    uint32_t jc_cost;         // lookahead joint class (9 bits) | thread slots << 9
};
static_assert(sizeof(GChunk) == 16, "GChunk layout");

// Shared-memory carve-up of k_group_match (byte offsets, 16-byte aligned).
struct GSmem {
    uint32_t table, jmap, stage, lmap, linit, vmap, vdom, vdfa, items, chunks, misc, gd, total;
};

__host__ __device__ inline uint32_t g_align16(uint32_t x) { return (x + 15u) & ~15u; }

__host__ __device__ inline GSmem g_layout(uint32_t tbytes, uint32_t K, uint32_t vcap_sum,
                                          uint32_t stage_bytes) {
    GSmem L;
    L.table = 0;
    L.jmap = g_align16(tbytes);
    L.stage = L.jmap + 1024;  // byte -> joint class, joint class -> outside-Sigma mask (u16 x 256 each)
    L.lmap = L.stage + 2 * stage_bytes;
    L.linit = L.lmap + kGThreads * K * 2;
    L.vmap = L.linit + kGThreads * K * 2;
    L.vdom = L.vmap + g_align16(2 * vcap_sum);
    L.vdfa = L.vdom + g_align16(2 * vcap_sum);
    L.items = L.vdfa + g_align16(vcap_sum);
    L.chunks = L.items + kGThreads * (uint32_t)sizeof(GItem);
    L.misc = L.chunks + kMaxTileChunks * (uint32_t)sizeof(GChunk);
    // last: the descriptors and misc words outlive the tiles (the combine uses
    // everything below misc as its buffer)
    L.gd = L.misc + 64 * 4;
    L.total = L.gd + kMaxDfas * (uint32_t)sizeof(GDfa);
    return L;
}

// misc words
enum { GM_NCH = 0, GM_LAST = 1, GM_MAXLEN = 2, GM_DOM = 4 /* G+1 words */, GM_CUR = 24 /* G */,
       GM_SCAN = 40 /* kGThreads / 32 */ };

// Advance K chains over S staged positions: 8-bit joint classes, the DFA's
// joint table at tb (rows of rowbytes), entries of SB bytes holding
// next_state * SB.  One 16-byte stage read covers 16 steps.
template <int K, int SB>
__device__ __forceinline__ void g_run(uint32_t (&s)[K], uint32_t tb, uint32_t rowbytes,
                                      uint32_t stage_addr, int S) {
    for (int j = 0; j < S; j += 16) {
        const uint4 w = g_lds_v4(stage_addr + (uint32_t)j);
        const uint32_t words[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t row = tb + ((words[h] >> (8 * q)) & 0xFFu) * rowbytes;
#pragma unroll
                for (int u = 0; u < K; ++u)
                    s[u] = SB == 1 ? g_lds_u8(row + s[u]) : g_lds_u16(row + s[u]);
            }
        }
    }
}

// Stage positions [pos, pos + 16) of a chunk as joint classes at dst (shared
// address): two aligned 16-byte loads and a funnel shift where both vectors
// lie inside the string, else byte loads.  Positions past the chunk end get
// the identity row J.  Returns the mask of DFAs that see a byte outside
// their Sigma among the valid positions.
__device__ __forceinline__ uint32_t g_stage16(const GPlan& p, const GChunk& c, uint32_t pos,
                                              uint32_t dst, const uint16_t* jmap,
                                              const uint16_t* jbad) {
    uint32_t v[4] = {0, 0, 0, 0};
    uint32_t nvalid = 0;
    if (pos < c.len) {
        nvalid = min(16u, c.len - pos);
        const uint64_t at = c.start + pos;
        const uint8_t* a = p.str + at;
        const uint32_t d = (uint32_t)((uintptr_t)a & 15u);
        if (at >= d && at + 32u <= p.n + d) {
            const uint4* al = reinterpret_cast<const uint4*>(a - d);
            const uint4 x0 = __ldg(al), x1 = __ldg(al + 1);
            const uint32_t q = d >> 2, r = (d & 3u) * 8u;
            const uint32_t w8[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
            uint32_t sel[5];
#pragma unroll
            for (int i = 0; i < 5; ++i)  // w8[q + i], with constant indices (registers)
                sel[i] = q == 0 ? w8[i] : (q == 1 ? w8[i + 1] : (q == 2 ? w8[i + 2] : w8[i + 3]));
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
    uint32_t w[4], flagged = 0;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        uint32_t word = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t j = 4 * i + k;
            uint32_t e = jmap[(v[i] >> (8 * k)) & 0xFFu];
            if (j >= nvalid) e = p.J;
            flagged |= e;
            word |= (e & 0xFFu) << (8 * k);
        }
        w[i] = word;
    }
    g_sts_v4(dst, make_uint4(w[0], w[1], w[2], w[3]));
    uint32_t bad = 0;
    if (flagged & 0x8000u) {  // rare: some DFA sees a byte outside its Sigma
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if ((uint32_t)(4 * i + k) < nvalid) bad |= jbad[(w[i] >> (8 * k)) & 0xFFu];
    }
    return bad;
}

// Block-wide exclusive scan of one value per thread (kGThreads threads);
// tmp holds kGThreads / 32 words.
__device__ __forceinline__ uint32_t g_block_scan(uint32_t v, uint32_t* tmp) {
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= (uint32_t)o) x += y;
    }
    if (lane == 31) tmp[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const uint32_t n = kGThreads / 32;
        uint32_t t = lane < n ? tmp[lane] : 0u, z = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, z, o);
            if (lane >= (uint32_t)o) z += y;
        }
        if (lane < n) tmp[lane] = z - t;
    }
    __syncthreads();
    const uint32_t r = tmp[warp] + x - v;
    __syncthreads();
    return r;
}

// Eq. (8) for every DFA of the group, by the last CTA to finish: each DFA's
// final state is q0 pushed through the CTA maps in CTA order (CTAs without a
// share published nothing and are skipped).  The maps (rows b * G + g of
// seg_stride entries, b-major) are staged through shared memory (buf,
// buf_bytes: at least one row and 1 KB of flags) in batches of consecutive
// rows, so the dependent walks run at shared-memory latency; thread g walks
// DFA g through the rows of each batch that belong to it, in order of b.
__device__ void g_combine(const GPlan& p, const GDfa* gd, uint8_t* buf, uint32_t buf_bytes,
                          uint32_t* cur) {
    const uint32_t tid = threadIdx.x;
    const bool maps = p.out_maps != nullptr;
    // map mode: every state of every DFA is walked; their current values sit
    // at the start of buf, the staged rows after them
    uint16_t* walk = reinterpret_cast<uint16_t*>(buf);
    const uint32_t nwalk = maps ? p.G * p.seg_stride : 0u;
    if (maps) {
        const uint32_t skip = g_align16(2u * nwalk);
        buf += skip;
        buf_bytes -= skip;
        for (uint32_t f = tid; f < nwalk; f += kGThreads) walk[f] = (uint16_t)(f % p.seg_stride);
    } else if (tid < p.G) {
        cur[tid] = gd[tid].q0;
    }
    const uint32_t row_bytes = p.seg_stride * 2u;   // a multiple of 16
    const uint32_t rows = p.grid * p.G;
    // rows per batch; the last kBatchMax bytes of buf hold the batch's valid flags
    constexpr uint32_t kBatchMax = 1024;
    uint32_t per = (buf_bytes - kBatchMax) / row_bytes;
    per = per < 1 ? 1 : (per > kBatchMax ? kBatchMax : per);  // the host guarantees room for one row
    uint8_t* valid = buf + buf_bytes - kBatchMax;
    const uint32_t vec_row = row_bytes / 16u;
    __syncthreads();
    for (uint32_t r0 = 0; r0 < rows; r0 += per) {
        const uint32_t r1 = min(rows, r0 + per), total = (r1 - r0) * vec_row;
        for (uint32_t r = r0 + tid; r < r1; r += kGThreads) {
            const uint32_t b = r / p.G;
            valid[r - r0] = p.share[b] < p.share[b + 1] ? 1 : 0;
        }
        __syncthreads();
        const uint4* src = reinterpret_cast<const uint4*>(p.seg_maps + (size_t)r0 * p.seg_stride);
        const uint32_t dst = g_sa(buf);
        // asynchronous 16-byte global-to-shared copies: all of a thread's
        // copies in flight at once, none of the data in registers
        for (uint32_t i = tid; i < total; i += kGThreads)
            if (valid[i / vec_row])
                asm volatile("cp.async.cg.shared.global [%0], [%1], 16;"
                             :: "r"(dst + 16u * i), "l"(src + i) : "memory");
        asm volatile("cp.async.wait_all;" ::: "memory");
        __syncthreads();
        const uint16_t* m = reinterpret_cast<const uint16_t*>(buf);
        if (maps) {
            // thread f walks state x of DFA g (f = g * seg_stride + x) through
            // this batch's rows of DFA g, in order of b
            for (uint32_t f = tid; f < nwalk; f += kGThreads) {
                const uint32_t g = f / p.seg_stride;
                if (f - g * p.seg_stride >= gd[g].qe) continue;
                uint32_t s = walk[f];
                for (uint32_t r = r0 + (g + p.G - r0 % p.G) % p.G; r < r1; r += p.G) {
                    if (!valid[r - r0]) continue;
                    const uint32_t nx = m[(size_t)(r - r0) * p.seg_stride + s];
                    if (GRP_OK(nx < gd[g].qe, p.err + g)) s = nx;
                }
                walk[f] = (uint16_t)s;
            }
        } else if (tid < p.G) {
            uint32_t s = cur[tid];
            // rows r of this batch with r % G == tid, in increasing r (hence b)
            uint32_t r = r0 + (tid + p.G - r0 % p.G) % p.G;
            for (; r < r1; r += p.G) {
                if (!valid[r - r0]) continue;  // a CTA without a share published nothing
                const uint32_t nx = m[(size_t)(r - r0) * p.seg_stride + s];
                if (GRP_OK(nx < gd[tid].qe, p.err + tid)) s = nx;
            }
            cur[tid] = s;
        }
        __syncthreads();
    }
    if (maps)
        for (uint32_t f = tid; f < nwalk; f += kGThreads) p.out_maps[f] = walk[f];
    if (tid < p.G) {
        const uint32_t err = atomicOr(p.err + tid, 0u);
        dfa_result_t r;
        const uint32_t s = maps ? 0u : cur[tid];
        r.final_state = g_final(err, s);
        r.accept = (err || maps) ? 0 : gd[tid].accept[s];
        r.reserved[0] = r.reserved[1] = r.reserved[2] = 0;
        r.status = g_status(err);
        p.results[tid] = r;
    }
}

// Eq. (8) over the segments of one string, for every DFA of a group (thread g,
// DFA g): the first segment's final state pushed through the state maps of the
// later segments (maps + (s - 1) * G * seg_stride), their statuses combined.
__global__ void k_group_compose(const dfa_result_t* seg_res, const uint16_t* maps, uint32_t nseg,
                                uint32_t G, uint32_t seg_stride, const GDfa* gd, dfa_result_t* out) {
    const uint32_t g = threadIdx.x;
    if (g >= G) return;
    uint32_t err = 0;
    for (uint32_t s = 0; s < nseg; ++s) {
        const int32_t st = seg_res[(size_t)s * G + g].status;
        err |= st == DFA_OK ? 0u : (st == DFA_EBOUNDS ? 2u : 1u);
    }
    uint32_t q = seg_res[g].final_state;
    const uint32_t qe = gd[g].qe;
    if (err || q >= qe) q = 0;
    for (uint32_t s = 1; s < nseg && !err; ++s) {
        const uint32_t nx = maps[((size_t)(s - 1) * G + g) * seg_stride + q];
        q = nx < qe ? nx : 0u;
    }
    dfa_result_t r;
    r.final_state = err ? 0u : q;
    r.accept = err ? 0 : gd[g].accept[q];
    r.reserved[0] = r.reserved[1] = r.reserved[2] = 0;
    r.status = err ? ((err & 2u) ? DFA_EBOUNDS : DFA_ESYMBOL) : DFA_OK;
    out[g] = r;
}

template <int K, int SB>
__global__ void __launch_bounds__(kGThreads, 2) k_group_match(GPlan p) {
    extern __shared__ __align__(16) uint8_t sm[];
    const GSmem L = g_layout(p.tbytes, K, p.vcap_sum, p.stage_bytes);
    uint16_t* jmap = reinterpret_cast<uint16_t*>(sm + L.jmap);
    GDfa* gd = reinterpret_cast<GDfa*>(sm + L.gd);
    uint16_t* lmap = reinterpret_cast<uint16_t*>(sm + L.lmap);
    uint16_t* linit = reinterpret_cast<uint16_t*>(sm + L.linit);
    uint16_t* vmap = reinterpret_cast<uint16_t*>(sm + L.vmap);
    uint16_t* vdom = reinterpret_cast<uint16_t*>(sm + L.vdom);
    uint8_t* vdfa = sm + L.vdfa;
    GItem* items = reinterpret_cast<GItem*>(sm + L.items);
    GChunk* chunks = reinterpret_cast<GChunk*>(sm + L.chunks);
    uint32_t* misc = reinterpret_cast<uint32_t*>(sm + L.misc);
    const uint32_t tid = threadIdx.x, b = blockIdx.x, G = p.G;

    // the group descriptors are needed by every CTA (also by the combine)
    for (uint32_t i = tid; i < G * (uint32_t)sizeof(GDfa) / 4; i += kGThreads)
        reinterpret_cast<uint32_t*>(gd)[i] = reinterpret_cast<const uint32_t*>(p.gd)[i];
    const uint32_t c0 = p.share[b], c1 = p.share[b + 1];
    if (c0 < c1) {
        {
            const uint4* src = reinterpret_cast<const uint4*>(p.tables);
            uint4* dst = reinterpret_cast<uint4*>(sm + L.table);
            for (uint32_t i = tid; i < p.tbytes / 16; i += kGThreads) dst[i] = __ldg(src + i);
            for (uint32_t i = tid; i < 256; i += kGThreads) {
                jmap[i] = p.jmap[i];
                jmap[256 + i] = p.jbad[i];
            }
        }
        __syncthreads();
        const uint16_t* jbad = jmap + 256;
        const uint32_t tbase = g_sa(sm + L.table);
        bool first = true;
        for (uint32_t cursor = c0; cursor < c1;) {
            // ---- tile: the longest run of chunks from cursor whose slots fit kGThreads
            const uint32_t navail = min(kMaxTileChunks, c1 - cursor);
            if (tid < navail) {
                const uint32_t k = cursor + tid;
                const uint64_t st = g_start(p.n, p.P, k), en = g_start(p.n, p.P, k + 1);
                const uint32_t jc = g_lookahead(p, jmap, k, st);
                uint32_t slots = 0;
                for (uint32_t g = 0; g < G; ++g) slots += g_slots(g_set(p, gd[g], g, jc) & 0xFFFFu, K);
                GChunk c;
                c.start = st;
                c.len = (uint32_t)(en - st);
                c.jc_cost = jc | (slots << 9);
                chunks[tid] = c;
            }
            __syncthreads();
            if (tid < 32) {
                uint32_t cost[8], tot = 0;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const uint32_t i = tid * 8 + e;
                    cost[e] = i < navail ? (chunks[i].jc_cost >> 9) : kGThreads + 1;
                    tot += cost[e];
                }
                uint32_t x = tot;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
                    if (tid >= (uint32_t)o) x += y;
                }
                uint32_t run = x - tot, cnt = 0;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    run += cost[e];
                    if (run <= kGThreads) cnt = tid * 8 + e + 1;
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) cnt = max(cnt, __shfl_xor_sync(0xFFFFFFFFu, cnt, o));
                uint32_t ml = 0;
#pragma unroll
                for (int e = 0; e < 8; ++e) {
                    const uint32_t i = tid * 8 + e;
                    if (i < cnt) ml = max(ml, chunks[i].len);
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) ml = max(ml, __shfl_xor_sync(0xFFFFFFFFu, ml, o));
                if (tid == 0) {
                    if (!GRP_OK(cnt >= 1, p.err)) cnt = 1;
                    misc[GM_NCH] = cnt;
                    misc[GM_MAXLEN] = ml;
                }
            }
            __syncthreads();
            const uint32_t nch = misc[GM_NCH], maxlen = misc[GM_MAXLEN];
            const uint32_t nitems = nch * G;  // <= kGThreads: every item takes >= 1 slot

            // ---- items (chunk-major, DFA-minor) and their thread offsets
            uint32_t my_slots = 0;
            GItem it;
            it.init = nullptr;
            it.toff = it.cnt = it.size = it.cls = 0;
            if (tid < nitems) {
                const uint32_t i = tid / G, g = tid - i * G;
                const uint32_t jc = chunks[i].jc_cost & 0x1FFu;
                const uint32_t info = g_set(p, gd[g], g, jc);
                uint32_t cls = info >> 16, size = info & 0xFFFFu;
                if (!GRP_OK(cls <= gd[g].C && size <= gd[g].vcap, p.err + g)) { cls = gd[g].C; size = 1; }
                it.init = gd[g].iset + gd[g].iset_off[cls];
                it.cnt = (uint16_t)((size + K - 1) / K);
                it.size = (uint16_t)size;
                it.cls = (uint16_t)cls;
                my_slots = g_slots(size, K);
            }
            const uint32_t toff = g_block_scan(my_slots, misc + GM_SCAN);
            if (tid < nitems) {
                it.toff = (uint16_t)toff;
                items[tid] = it;
            }
            __syncthreads();

            // ---- my item: the last one whose first thread is at or before mine
            int lo = 0, hi = (int)nitems - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (items[mid].toff <= tid) lo = mid; else hi = mid - 1;
            }
            const GItem mine = items[lo];
            const uint32_t mi = (uint32_t)lo / G, mg = (uint32_t)lo - mi * G;
            const uint32_t r = tid - mine.toff;
            const bool active = r < mine.cnt;
            const uint32_t tb = tbase + gd[mg].tbl_off;
            const uint32_t rowbytes = gd[mg].qpad * SB;
            uint32_t s[K];
#pragma unroll
            for (int u = 0; u < K; ++u) {
                uint32_t init = 0;
                if (active) {
                    uint32_t slot = r * K + u;
                    if (slot >= mine.size) slot = r * K;  // padding chain: repeat the first
                    init = mine.init[slot];
                    if (!GRP_OK(init < gd[mg].qe, p.err + mg)) init = 0;
                }
                s[u] = init * SB;
                linit[tid * K + u] = (uint16_t)init;
            }

            // ---- segments: stage each chunk once, run every item's chains on it
            const int quant = 16;
            int S = (int)(p.stage_bytes / nch) / quant * quant;
            S = S < quant ? quant : (S > (int)kMaxSeg ? (int)kMaxSeg : S);
            if (maxlen > 0) {
                const uint32_t nseg = (maxlen + (uint32_t)S - 1) / (uint32_t)S;
                S = (int)(((maxlen + nseg - 1) / nseg + quant - 1) / quant * quant);
            }
            const uint32_t nseg = maxlen ? (maxlen + (uint32_t)S - 1) / (uint32_t)S : 0u;
            const uint32_t stage0 = g_sa(sm + L.stage);
            const uint32_t groups = (uint32_t)S / 16u;
            uint32_t bad = 0;
            for (uint32_t seg = 0; seg < nseg; ++seg) {
                const uint32_t stage = stage0 + (seg & 1u) * p.stage_bytes;
                for (uint32_t w = tid; w < nch * groups; w += kGThreads) {
                    const uint32_t i = w / groups, q = w - i * groups;
                    bad |= g_stage16(p, chunks[i], seg * (uint32_t)S + 16u * q,
                                     stage + i * (uint32_t)S + 16u * q, jmap, jbad);
                }
                __syncthreads();
                if (active) g_run<K, SB>(s, tb, rowbytes, stage + mi * (uint32_t)S, S);
                // the next segment stages into the other buffer: one barrier per segment
            }
            if (bad)
                for (uint32_t g = 0; g < G; ++g)
                    if ((bad >> g) & 1u) atomicOr(p.err + g, 1u);
#pragma unroll
            for (int u = 0; u < K; ++u) {
                uint32_t v = s[u] / SB;
                if (active && !GRP_OK(v < gd[mg].qe, p.err + mg)) v = 0;
                lmap[tid * K + u] = (uint16_t)v;
                // inspection output: L_k[j] = delta*(j, chunk k) for j in I_k (Sec. 4.1)
                const uint32_t slot = r * K + u;
                if (p.dbg && active && slot < mine.size)
                    p.dbg[((size_t)mg * p.P + cursor + mi) * p.qe_max + linit[tid * K + u]] = (uint16_t)v;
            }
            __syncthreads();

            // ---- Eq. (9): compose each DFA's chunk maps, in order, into its running map
            uint32_t i0 = 0;
            if (first) {
                // the share's first chunk starts every DFA's running map: its
                // domain is that chunk's initial-state set
                if (tid == 0) {
                    uint32_t o = 0;
                    for (uint32_t g = 0; g < G; ++g) {
                        misc[GM_DOM + g] = o;
                        o += items[g].size;
                    }
                    misc[GM_DOM + G] = o;
                }
                __syncthreads();
                for (uint32_t g = 0; g < G; ++g) {
                    const uint32_t o = misc[GM_DOM + g], base = (uint32_t)items[g].toff * K;
                    for (uint32_t x = tid; x < items[g].size; x += kGThreads) {
                        vmap[o + x] = lmap[base + x];
                        vdom[o + x] = linit[base + x];
                        vdfa[o + x] = (uint8_t)g;
                    }
                }
                __syncthreads();
                i0 = 1;
                first = false;
            }
            const uint32_t nD = misc[GM_DOM + G];
            for (uint32_t x = tid; x < nD; x += kGThreads) {
                const uint32_t g = vdfa[x];
                const GDfa& d = gd[g];
                uint32_t v = vmap[x];
                for (uint32_t i = i0; i < nch; ++i) {
                    const GItem& e = items[i * G + g];
                    if (!GRP_OK(v < d.qe, p.err + g)) break;
                    const uint32_t q = __ldg(d.pos + (size_t)e.cls * d.qe + v);
                    if (q != kNone16 && GRP_OK(q < e.size, p.err + g)) v = lmap[(uint32_t)e.toff * K + q];
                }
                vmap[x] = (uint16_t)v;
            }
            __syncthreads();
            cursor += nch;
        }
        // ---- publish this CTA's map of each DFA, dense over Q (identity
        // outside the domain: those states are excluded, hence fixed)
        uint16_t* mine = p.seg_maps + (size_t)b * G * p.seg_stride;
        for (uint32_t i = tid; i < G * p.seg_stride; i += kGThreads) {
            const uint32_t g = i / p.seg_stride, s = i - g * p.seg_stride;
            mine[i] = (uint16_t)(s < gd[g].qe ? s : 0u);
        }
        __syncthreads();
        const uint32_t nD = misc[GM_DOM + G];
        for (uint32_t x = tid; x < nD; x += kGThreads) {
            const uint32_t g = vdfa[x];
            if (GRP_OK(vdom[x] < gd[g].qe && vmap[x] < gd[g].qe, p.err + g))
                mine[(size_t)g * p.seg_stride + vdom[x]] = vmap[x];
        }
    }
    __syncthreads();
    if (tid == 0) {
        __threadfence();
        const uint32_t old = atomicAdd(p.arrived, 1u);
        misc[GM_LAST] = old + 1 == gridDim.x ? 1u : 0u;
    }
    __syncthreads();
    if (misc[GM_LAST]) {
        __threadfence();
        // everything below the misc words is free now
        g_combine(p, gd, sm, L.misc, misc + GM_CUR);
    }
}

// ------------------------------------------------------------ host side

using MatchFn = void (*)(GPlan);

template <int K, int SB>
MatchFn match_fn() { return k_group_match<K, SB>; }

MatchFn pick(uint32_t K, uint32_t sb) {
    switch (K * 4 + sb) {
        case 1 * 4 + 1: return match_fn<1, 1>();
        case 1 * 4 + 2: return match_fn<1, 2>();
        case 2 * 4 + 1: return match_fn<2, 1>();
        case 2 * 4 + 2: return match_fn<2, 2>();
        case 4 * 4 + 1: return match_fn<4, 1>();
        case 4 * 4 + 2: return match_fn<4, 2>();
        case 8 * 4 + 1: return match_fn<8, 1>();
        case 8 * 4 + 2: return match_fn<8, 2>();
        case 16 * 4 + 1: return match_fn<16, 1>();
        case 16 * 4 + 2: return match_fn<16, 2>();
        default: return nullptr;
    }
}

// Kernel attributes, set once per device (thread-safe).
struct Props {
    bool ready = false;
    uint32_t sms = 0, optin = 0, per_sm = 0;
};
constexpr int kMaxDevices = 64;
Props g_props[kMaxDevices];
std::mutex g_mu;

const Props* props() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    std::lock_guard<std::mutex> lk(g_mu);
    Props& p = g_props[dev];
    if (p.ready) return &p;
    int sms = 0, optin = 0, per_sm = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev) != cudaSuccess ||
        sms < 1 || optin < 1 || per_sm < 1)
        return nullptr;
    for (uint32_t K : {1u, 2u, 4u, 8u, 16u})
        for (uint32_t sb : {1u, 2u})
            if (cudaFuncSetAttribute(pick(K, sb), cudaFuncAttributeMaxDynamicSharedMemorySize, optin) !=
                cudaSuccess)
                return nullptr;
    p.sms = (uint32_t)sms;
    p.optin = (uint32_t)optin;
    p.per_sm = (uint32_t)per_sm;
    p.ready = true;
    return &p;
}

}  // namespace grp
}  // namespace dfam

using namespace dfam;
using namespace dfam::grp;

// The opaque group handle of the C ABI.
struct dfa_group_s {
    std::vector<const dfa_s*> dfas;
    uint32_t G = 0, J = 0, sb = 1, tbytes = 0, vcap_sum = 0, qe_max = 0, K0 = 4, seg_stride = 0;
    uint32_t ctas0 = 0;            // default thread blocks per SM (0: 2 where they fit)
    std::vector<uint16_t> jmap;    // 256: joint class | 0x8000 if some DFA has it outside Sigma
    std::vector<uint16_t> jbad;    // 256: joint class -> mask of DFAs with it outside Sigma
    std::vector<uint32_t> jinfo;   // G * 256
    std::vector<uint8_t> tables;   // tbytes
    std::vector<GDfa> gd;          // device pointers (on_device groups)
    std::vector<double> mean_slots_by_k;  // per K in {1,2,4,8,16}: sum over DFAs of the mean slots
    bool on_device = false;
    int device = -1;
    void* dev_block = nullptr;
    uint64_t dev_bytes = 0;
    GDfa* d_gd = nullptr;
    uint32_t* d_jinfo = nullptr;
    uint16_t* d_jmap = nullptr;
    uint16_t* d_jbad = nullptr;
    uint8_t* d_tables = nullptr;
    // dfa_group_match's device buffers (input copy, workspace and results),
    // grown as needed and reused; the mutex serialises those calls
    std::mutex mu;
    uint8_t* d_str = nullptr;
    uint64_t str_cap = 0;
    uint8_t* d_ws = nullptr;
    uint64_t ws_cap = 0;
    cudaStream_t copy_stream = nullptr;   // host input copies of the pipelined path
    cudaStream_t match_stream = nullptr;  // its launches
};

namespace {

uint32_t k_index(uint32_t K) {
    return K == 1 ? 0u : K == 2 ? 1u : K == 4 ? 2u : K == 8 ? 3u : K == 16 ? 4u : 5u;
}

// Thread slots one chunk can need at most for chains-per-thread K.
uint32_t max_chunk_slots(const dfa_group_s* g, uint32_t K) {
    uint32_t s = 0;
    for (const dfa_s* d : g->dfas) s += std::max(1u, (std::max(d->h.imax, 1u) + K - 1) / K);
    return s;
}

struct GLaunch {
    GPlan p;
    uint32_t smem = 0, K = 0;
    uint64_t ws_share = 0, ws_cshare = 0, ws_err = 0, ws_maps = 0, ws_total = 0;
};

uint64_t al256(uint64_t x) { return (x + 255) & ~255ull; }

int plan_launch(const dfa_group_s* g, uint64_t n, const dfa_group_opts_t* o, GLaunch* out) {
    if (!g) return DFA_EINVAL;
    if (!g->on_device) return DFA_EHOSTONLY;
    if (n >= kMaxLen) return DFA_EINVAL;
    const uint32_t K = (o && o->states_per_thread) ? o->states_per_thread : g->K0;
    if (k_index(K) > 4 || max_chunk_slots(g, K) > kGThreads) return DFA_EINVAL;
    const uint32_t want = (o && o->ctas_per_sm) ? o->ctas_per_sm : (g->ctas0 ? g->ctas0 : 2u);
    if (want > 2) return DFA_EINVAL;
    const Props* pr = props();
    if (!pr) return DFA_ECUDA;
    // the largest stage (up to 32 KB per buffer) that lets `want` CTAs share an
    // SM, else fewer CTAs; the combine needs room for one CTA's maps below the
    // descriptors
    uint32_t stage = 0, ctas = 0;
    for (uint32_t c = want; c >= 1 && !ctas; --c)
        for (uint32_t sbts = 32u * 1024u; sbts >= kMinStage; sbts -= 2048u) {
            const GSmem L = g_layout(g->tbytes, K, g->vcap_sum, sbts);
            if (L.total <= pr->optin && c * (L.total + 1024u) <= pr->per_sm) {
                stage = sbts;
                ctas = c;
                break;
            }
        }
    if (!ctas) return DFA_EINVAL;
    const GSmem L = g_layout(g->tbytes, K, g->vcap_sum, stage);
    if (L.misc < g->seg_stride * 2u + 1024u) return DFA_EINVAL;  // the combine stages one map row at least
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pick(K, g->sb), kGThreads, L.total) !=
            cudaSuccess ||
        per_sm < 1)
        return DFA_ECUDA;
    const uint32_t grid = pr->sms * std::min<uint32_t>((uint32_t)per_sm, ctas);
    uint64_t P;
    if (o && o->num_chunks) {
        P = o->num_chunks;
    } else {
        // enough slots for kTilesPerCta tiles on every CTA, chunks >= kMinChunk
        const double mean = std::max(1.0, g->mean_slots_by_k[k_index(K)]);
        const double want_p = (double)grid * kGThreads * kTilesPerCta * 0.9 / mean;
        P = std::min<uint64_t>((uint64_t)want_p, n / kMinChunk);
        P = std::min<uint64_t>(P, kMaxChunks);
        P = std::max<uint64_t>(P, (n + 0x7FFFFFFFull - 1) / 0x7FFFFFFFull);
        P = std::max<uint64_t>(P, 1);
    }
    if (P > kMaxChunks || (n + P - 1) / P >= (1ull << 31)) return DFA_EINVAL;
    std::memset(out, 0, sizeof *out);
    GPlan& p = out->p;
    p.gd = g->d_gd;
    p.jinfo = g->d_jinfo;
    p.jmap = g->d_jmap;
    p.jbad = g->d_jbad;
    p.tables = g->d_tables;
    p.n = n;
    p.G = g->G;
    p.J = g->J;
    p.P = (uint32_t)P;
    p.K = K;
    p.grid = grid;
    p.tbytes = g->tbytes;
    p.stage_bytes = stage;
    p.vcap_sum = g->vcap_sum;
    p.seg_stride = g->seg_stride;
    p.qe_max = g->qe_max;
    out->smem = L.total;
    out->K = K;
    out->ws_share = 0;
    out->ws_cshare = al256(out->ws_share + 4ull * (grid + 1));
    out->ws_err = al256(out->ws_cshare + 4ull * P);
    out->ws_maps = al256(out->ws_err + 4ull * (g->G + 1));
    out->ws_total = al256(out->ws_maps + 2ull * grid * g->G * g->seg_stride);
    return DFA_OK;
}

void bind_ws(GLaunch& l, uint8_t* ws) {
    l.p.share = reinterpret_cast<uint32_t*>(ws + l.ws_share);
    l.p.cshare = reinterpret_cast<uint32_t*>(ws + l.ws_cshare);
    l.p.err = reinterpret_cast<uint32_t*>(ws + l.ws_err);
    l.p.arrived = l.p.err + l.p.G;
    l.p.seg_maps = reinterpret_cast<uint16_t*>(ws + l.ws_maps);
}

int issue(const GLaunch& l, uint32_t sb, const dfa_group_opts_t* o, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(l.p.err, 0, 4ull * (l.p.G + 1), st) != cudaSuccess) return DFA_ECUDA;
    k_group_plan<<<1, kPlanThreads, 0, st>>>(l.p);
    if (cudaGetLastError() != cudaSuccess) return DFA_ECUDA;
    if (o && o->match_begin_event &&
        cudaEventRecord(static_cast<cudaEvent_t>(o->match_begin_event), st) != cudaSuccess)
        return DFA_ECUDA;
    GPlan p = l.p;
    void* args[] = {&p};
    if (cudaLaunchKernel(reinterpret_cast<const void*>(pick(l.K, sb)), dim3(l.p.grid), dim3(kGThreads),
                         args, l.smem, st) != cudaSuccess)
        return DFA_ECUDA;
    if (o && o->match_end_event &&
        cudaEventRecord(static_cast<cudaEvent_t>(o->match_end_event), st) != cudaSuccess)
        return DFA_ECUDA;
    return DFA_OK;
}

// Next state of s on class c in a compiled DFA's class-major host table
// (entries of h.sb bytes holding next * h.sb, little-endian).
uint32_t host_next(const HostDfa& h, uint32_t c, uint32_t s) {
    const uint8_t* e = h.table.data() + ((size_t)c * h.qpad + s) * h.sb;
    uint32_t v = 0;
    for (uint32_t i = 0; i < h.sb; ++i) v |= (uint32_t)e[i] << (8 * i);
    return v / h.sb;
}

uint32_t set_size(const HostDfa& h, uint32_t c) { return h.iset_off[c + 1] - h.iset_off[c]; }

// Host input of a group is copied in segments on a copy stream while the
// earlier segments are matched: segment lengths double from len/32 (clamped
// to [16 MiB, 256 MiB]) up to a quarter of the string.  Every segment after
// the first is a continuation launch (its chunk 0 looks back into the bytes
// before it) that publishes each DFA's state map of the segment; one thread
// per DFA then applies those maps to the first segment's final state (Eq. 8).
// Returns false (copy the string whole) when the string is too short or a
// map-mode combine does not fit.
bool group_segments(const dfa_group_s* g, uint64_t len, std::vector<uint64_t>* seg) {
    const uint64_t MiB = 1ull << 20;
    const uint64_t first = std::min<uint64_t>(std::max<uint64_t>(len / 32, 16 * MiB), 256 * MiB);
    if (len < 2 * first || (uint64_t)g->G * g->seg_stride > 8192) return false;
    const uint64_t cap = std::max<uint64_t>(first, len / 4);
    seg->clear();
    uint64_t at = 0, next = first;
    while (at < len) {
        uint64_t l = std::min<uint64_t>(next, len - at);
        if (len - at - l < first / 2) l = len - at;  // no short last segment
        seg->push_back(l);
        at += l;
        next = std::min<uint64_t>(2 * next, cap);
    }
    return seg->size() >= 2;
}

int grow_buf(uint8_t** p, uint64_t* cap, uint64_t need) {
    if (*cap >= need) return DFA_OK;
    cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (cudaMalloc(p, need) != cudaSuccess) {
        cudaGetLastError();
        return DFA_ENOMEM;
    }
    *cap = need;
    return DFA_OK;
}

// The pipelined path of dfa_group_match (caller holds g->mu).
int group_match_pipelined(dfa_group_s* g, const uint8_t* str, const std::vector<uint64_t>& seg,
                          const dfa_group_opts_t* opts, dfa_result_t* out) {
    const uint32_t nseg = (uint32_t)seg.size();
    uint64_t len = 0;
    for (uint64_t l : seg) len += l;
    std::vector<GLaunch> ls(nseg);
    uint64_t ws_need = 0;
    for (uint32_t i = 0; i < nseg; ++i) {
        int rc = plan_launch(g, seg[i], opts, &ls[i]);
        if (rc != DFA_OK) return rc;
        const GSmem L = g_layout(g->tbytes, ls[i].K, g->vcap_sum, ls[i].p.stage_bytes);
        if (L.misc < g_align16(2u * g->G * g->seg_stride) + g->seg_stride * 2u + 1024u) return DFA_EINVAL;
        ws_need = std::max(ws_need, ls[i].ws_total);
    }
    // workspace | results of every segment (nseg * G) | final results (G) | maps
    const uint64_t res_off = ws_need;
    const uint64_t fin_off = al256(res_off + sizeof(dfa_result_t) * nseg * g->G);
    const uint64_t map_off = al256(fin_off + sizeof(dfa_result_t) * g->G);
    const uint64_t total = map_off + 2ull * (nseg - 1) * g->G * g->seg_stride;
    int rc;
    if ((rc = grow_buf(&g->d_str, &g->str_cap, len)) != DFA_OK) return rc;
    if ((rc = grow_buf(&g->d_ws, &g->ws_cap, total)) != DFA_OK) return rc;
    if (!g->copy_stream &&
        cudaStreamCreateWithFlags(&g->copy_stream, cudaStreamNonBlocking) != cudaSuccess)
        return DFA_ECUDA;
    if (!g->match_stream &&
        cudaStreamCreateWithFlags(&g->match_stream, cudaStreamNonBlocking) != cudaSuccess)
        return DFA_ECUDA;
    std::vector<cudaEvent_t> ev(nseg, nullptr);
    rc = DFA_OK;
    for (uint32_t i = 0; i < nseg && rc == DFA_OK; ++i)
        if (cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming) != cudaSuccess) rc = DFA_ECUDA;
    dfa_result_t* res = reinterpret_cast<dfa_result_t*>(g->d_ws + res_off);
    dfa_result_t* fin = reinterpret_cast<dfa_result_t*>(g->d_ws + fin_off);
    uint16_t* maps = reinterpret_cast<uint16_t*>(g->d_ws + map_off);
    uint64_t at = 0;
    for (uint32_t i = 0; i < nseg && rc == DFA_OK; ++i) {
        if (cudaMemcpyAsync(g->d_str + at, str + at, seg[i], cudaMemcpyHostToDevice, g->copy_stream) !=
                cudaSuccess ||
            cudaEventRecord(ev[i], g->copy_stream) != cudaSuccess)
            rc = DFA_ECUDA;
        at += seg[i];
    }
    at = 0;
    for (uint32_t i = 0; i < nseg && rc == DFA_OK; ++i) {
        if (cudaStreamWaitEvent(g->match_stream, ev[i], 0) != cudaSuccess) {
            rc = DFA_ECUDA;
            break;
        }
        GLaunch& l = ls[i];
        bind_ws(l, g->d_ws);  // launches on one stream run one after the other
        l.p.str = g->d_str + at;
        l.p.results = res + (size_t)i * g->G;
        l.p.work = nullptr;
        l.p.dbg = nullptr;
        l.p.cont = i > 0 ? 1u : 0u;
        l.p.out_maps = i > 0 ? maps + (size_t)(i - 1) * g->G * g->seg_stride : nullptr;
        rc = issue(l, g->sb, nullptr, g->match_stream);
        at += seg[i];
    }
    if (rc == DFA_OK) {
        k_group_compose<<<1, 32, 0, g->match_stream>>>(res, maps, nseg, g->G, g->seg_stride, g->d_gd, fin);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(out, fin, sizeof(dfa_result_t) * g->G, cudaMemcpyDeviceToHost,
                            g->match_stream) != cudaSuccess)
            rc = DFA_ECUDA;
    }
    // wait for everything issued, whatever happened
    if (cudaStreamSynchronize(g->copy_stream) != cudaSuccess) rc = DFA_ECUDA;
    if (cudaStreamSynchronize(g->match_stream) != cudaSuccess) rc = DFA_ECUDA;
    for (cudaEvent_t e : ev)
        if (e) cudaEventDestroy(e);
    return rc;
}

}  // namespace

extern "C" {

int dfa_group_create(const dfa_t* const* dfas, uint32_t count, dfa_group_t** out) {
    return dfam::no_throw([&]() -> int {
        if (!out) return DFA_EINVAL;
        *out = nullptr;
        if (!dfas || count == 0 || count > kMaxDfas) return DFA_EINVAL;
        uint32_t on_dev = 0;
        for (uint32_t i = 0; i < count; ++i) {
            if (!dfas[i] || dfas[i]->h.qe > kMaxQe) return DFA_EINVAL;
            on_dev += dfas[i]->on_device ? 1u : 0u;
            if (dfas[i]->on_device && dfas[i]->device != dfas[0]->device) return DFA_EINVAL;
        }
        if (on_dev != 0 && on_dev != count) return DFA_EINVAL;  // all on one device, or all host-only
        dfa_group_s* g = new (std::nothrow) dfa_group_s;
        if (!g) return DFA_ENOMEM;
        g->G = count;
        g->dfas.assign(dfas, dfas + count);
        // joint classes: distinct tuples (class in DFA 0, ..., class in DFA G-1) over the bytes
        std::map<std::vector<uint16_t>, uint32_t> ids;
        std::vector<uint32_t> rep;  // a byte of each joint class
        g->jmap.assign(256, 0);
        for (uint32_t b = 0; b < 256; ++b) {
            std::vector<uint16_t> key(count);
            for (uint32_t i = 0; i < count; ++i) key[i] = dfas[i]->h.byte_class[b];
            auto it = ids.find(key);
            if (it == ids.end()) {
                it = ids.emplace(key, (uint32_t)rep.size()).first;
                rep.push_back(b);
            }
            g->jmap[b] = (uint16_t)it->second;
        }
        g->J = (uint32_t)rep.size();
        if (g->J > kMaxJoint) {
            delete g;
            return DFA_EINVAL;
        }
        g->jbad.assign(256, 0);
        for (uint32_t j = 0; j < g->J; ++j)
            for (uint32_t i = 0; i < count; ++i)
                if (dfas[i]->h.byte_class[rep[j]] == kNone16) g->jbad[j] |= (uint16_t)(1u << i);
        for (uint32_t b = 0; b < 256; ++b)
            if (g->jbad[g->jmap[b]]) g->jmap[b] |= 0x8000u;
        // joint tables: per DFA, J rows (one per joint class) and the identity row
        g->sb = 1;
        for (uint32_t i = 0; i < count; ++i) {
            g->qe_max = std::max(g->qe_max, dfas[i]->h.qe);
            if (dfas[i]->h.qe > 256) g->sb = 2;
        }
        g->seg_stride = (g->qe_max + 7) & ~7u;
        std::vector<uint32_t> qpad(count), toff(count), vcap(count);
        uint64_t tb = 0;
        for (uint32_t i = 0; i < count; ++i) {
            const uint32_t per16 = 16 / g->sb;
            qpad[i] = (dfas[i]->h.qe + per16 - 1) / per16 * per16;
            toff[i] = (uint32_t)tb;
            tb += (uint64_t)(g->J + 1) * qpad[i] * g->sb;
        }
        if (tb > kTableMax) {
            delete g;
            return DFA_EINVAL;
        }
        g->tbytes = (uint32_t)tb;
        g->tables.assign(tb, 0);
        g->jinfo.assign((size_t)count * 256, 0);
        g->mean_slots_by_k.assign(5, 0.0);
        for (uint32_t i = 0; i < count; ++i) {
            const HostDfa& h = dfas[i]->h;
            uint8_t* t = g->tables.data() + toff[i];
            for (uint32_t j = 0; j <= g->J; ++j) {
                const uint32_t c = j < g->J ? h.byte_class[rep[j]] : kNone16;
                for (uint32_t s = 0; s < h.qe; ++s) {
                    const uint32_t nx = c == kNone16 ? s : host_next(h, c, s);  // identity row or outside Sigma
                    const uint32_t v = nx * g->sb;
                    uint8_t* e = t + ((size_t)j * qpad[i] + s) * g->sb;
                    e[0] = (uint8_t)v;
                    if (g->sb == 2) e[1] = (uint8_t)(v >> 8);
                }
                if (j < g->J) {
                    // a lookahead byte outside Sigma fails the test; its chunk takes the start set
                    const uint32_t cls = c == kNone16 ? h.C : c;
                    g->jinfo[(size_t)i * 256 + j] = (cls << 16) | set_size(h, cls);
                }
            }
            vcap[i] = 0;
            for (uint32_t c = 0; c <= h.C; ++c) vcap[i] = std::max(vcap[i], set_size(h, c));
            g->vcap_sum += vcap[i];
            for (uint32_t ki = 0; ki < 5; ++ki) {
                const uint32_t K = 1u << ki;
                double m = 0;
                for (uint32_t c = 0; c < h.C; ++c) m += std::max(1u, (set_size(h, c) + K - 1) / K);
                g->mean_slots_by_k[ki] += h.C ? m / h.C : 1.0;
            }
        }
        if (g->vcap_sum > kVcapMax) {
            delete g;
            return DFA_EINVAL;
        }
        // default chains per thread: for one DFA the compiler's rule on its mean set
        // size; for several, 2 (a warp then spans the fewest (chunk, DFA) items, whose
        // rows differ: K = 2 ran 15% faster than K = 4 on the 8 protein-shaped DFAs
        // of the bench), raised until one chunk's items fit a CTA
        double mean_set = 0;
        for (uint32_t i = 0; i < count; ++i) mean_set += dfas[i]->h.mean_iset;
        g->K0 = count == 1 ? k_for_set_size(mean_set) : std::min(2u, k_for_set_size(mean_set / count));
        while (g->K0 <= 16 && max_chunk_slots(g, g->K0) > kGThreads) g->K0 *= 2;
        if (g->K0 > 16) {
            delete g;
            return DFA_EINVAL;
        }
        if (on_dev) {
            int cur = -1;
            if (cudaGetDevice(&cur) != cudaSuccess || cur != dfas[0]->device) {
                delete g;
                return DFA_EINVAL;
            }
            const uint64_t o_gd = 0, o_ji = al256(o_gd + sizeof(GDfa) * count),
                           o_jm = al256(o_ji + 4ull * count * 256), o_jb = al256(o_jm + 512),
                           o_tb = al256(o_jb + 512), total = al256(o_tb + tb);
            void* blk = nullptr;
            if (cudaMalloc(&blk, total) != cudaSuccess) {
                cudaGetLastError();
                delete g;
                return DFA_ENOMEM;
            }
            uint8_t* base = static_cast<uint8_t*>(blk);
            g->dev_block = blk;
            g->dev_bytes = total;
            g->device = cur;
            g->d_gd = reinterpret_cast<GDfa*>(base + o_gd);
            g->d_jinfo = reinterpret_cast<uint32_t*>(base + o_ji);
            g->d_jmap = reinterpret_cast<uint16_t*>(base + o_jm);
            g->d_jbad = reinterpret_cast<uint16_t*>(base + o_jb);
            g->d_tables = base + o_tb;
            g->gd.resize(count);
            for (uint32_t i = 0; i < count; ++i) {
                const DevDfa& x = dfas[i]->dev;
                GDfa& d = g->gd[i];
                std::memset(&d, 0, sizeof d);
                d.iset_off = x.iset_off;
                d.iset = x.iset;
                d.pos = x.pos;
                d.accept = x.accept;
                d.qe = x.qe;
                d.q0 = x.q0;
                d.C = x.C;
                d.qpad = qpad[i];
                d.tbl_off = toff[i];
                d.vcap = vcap[i];
            }
            if (cudaMemcpy(g->d_gd, g->gd.data(), sizeof(GDfa) * count, cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(g->d_jinfo, g->jinfo.data(), 4ull * count * 256, cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(g->d_jmap, g->jmap.data(), 512, cudaMemcpyHostToDevice) != cudaSuccess ||
                cudaMemcpy(g->d_jbad, g->jbad.data(), 512, cudaMemcpyHostToDevice) != cudaSuccess ||
                (tb && cudaMemcpy(g->d_tables, g->tables.data(), tb, cudaMemcpyHostToDevice) != cudaSuccess)) {
                cudaFree(blk);
                delete g;
                return DFA_ECUDA;
            }
            g->on_device = true;
        }
        *out = g;
        return DFA_OK;
    });
}

void dfa_group_destroy(dfa_group_t* g) {
    if (!g) return;
    if (g->dev_block) {
        int cur = -1;
        const bool other = cudaGetDevice(&cur) == cudaSuccess && cur != g->device;
        if (other) cudaSetDevice(g->device);
        cudaFree(g->dev_block);
        cudaFree(g->d_str);
        cudaFree(g->d_ws);
        if (g->copy_stream) cudaStreamDestroy(g->copy_stream);
        if (g->match_stream) cudaStreamDestroy(g->match_stream);
        if (other) cudaSetDevice(cur);
    }
    delete g;
}

int dfa_group_info(const dfa_group_t* g, dfa_group_info_t* out) {
    if (!g || !out) return DFA_EINVAL;
    std::memset(out, 0, sizeof *out);
    out->num_dfas = g->G;
    out->joint_classes = g->J;
    out->state_bytes = g->sb;
    out->states_per_thread = g->K0;
    out->ctas_per_sm = g->ctas0;
    out->max_states_ext = g->qe_max;
    out->sum_max_set = g->vcap_sum;
    out->table_bytes = g->tbytes;
    out->device_bytes = g->dev_bytes;
    return DFA_OK;
}

int dfa_group_joint_classes(const dfa_group_t* g, uint16_t* out) {
    if (!g || !out) return DFA_EINVAL;
    for (uint32_t b = 0; b < 256; ++b) out[b] = g->jmap[b] & 0xFFu;
    return DFA_OK;
}

int dfa_group_autotune(dfa_group_t* g, const uint8_t* dev_sample, uint64_t len, void* stream,
                       uint32_t* states_per_thread, uint32_t* ctas_per_sm, double* best_ms) {
    return dfam::no_throw([&]() -> int {
        if (!g || (len && !dev_sample)) return DFA_EINVAL;
        if (!g->on_device) return DFA_EHOSTONLY;
        struct Cand {
            uint32_t K, ctas;
            GLaunch l;
        };
        std::vector<Cand> cands;
        uint64_t ws_need = 0;
        for (uint32_t K : {1u, 2u, 4u, 8u, 16u})
            for (uint32_t c : {1u, 2u}) {
                dfa_group_opts_t o;
                std::memset(&o, 0, sizeof o);
                o.states_per_thread = K;
                o.ctas_per_sm = c;
                Cand x;
                x.K = K;
                x.ctas = c;
                if (plan_launch(g, len, &o, &x.l) != DFA_OK) continue;
                ws_need = std::max(ws_need, x.l.ws_total);
                cands.push_back(x);
            }
        if (cands.empty()) return DFA_EINVAL;
        void *ws = nullptr, *res = nullptr;
        if (cudaMalloc(&ws, ws_need) != cudaSuccess || cudaMalloc(&res, sizeof(dfa_result_t) * g->G) != cudaSuccess) {
            cudaGetLastError();
            cudaFree(ws);
            return DFA_ENOMEM;
        }
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        int rc = (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) ? DFA_OK
                                                                                              : DFA_ECUDA;
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        double best = 1e30;
        const Cand* win = nullptr;
        for (Cand& x : cands) {
            if (rc != DFA_OK) break;
            bind_ws(x.l, static_cast<uint8_t*>(ws));
            x.l.p.str = dev_sample;
            x.l.p.results = static_cast<dfa_result_t*>(res);
            float t = 1e30f;
            for (int rep = 0; rep < 3 && rc == DFA_OK; ++rep) {  // the first launch warms up
                if (cudaEventRecord(e0, st) != cudaSuccess) rc = DFA_ECUDA;
                if (rc == DFA_OK) rc = issue(x.l, g->sb, nullptr, stream);
                if (rc == DFA_OK && (cudaEventRecord(e1, st) != cudaSuccess ||
                                     cudaEventSynchronize(e1) != cudaSuccess))
                    rc = DFA_ECUDA;
                float ms = 0;
                if (rc == DFA_OK && rep > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess)
                    t = std::min(t, ms);
            }
            if (rc == DFA_OK && t < best) {
                best = t;
                win = &x;
            }
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFree(ws);
        cudaFree(res);
        if (rc != DFA_OK) return rc;
        if (!win) return DFA_ECUDA;
        g->K0 = win->K;
        g->ctas0 = win->ctas;
        if (states_per_thread) *states_per_thread = win->K;
        if (ctas_per_sm) *ctas_per_sm = win->ctas;
        if (best_ms) *best_ms = best;
        return DFA_OK;
    });
}

int dfa_group_plan_chunks(const dfa_group_t* g, uint64_t len, const dfa_group_opts_t* opts,
                          uint32_t* P) {
    return dfam::no_throw([&]() -> int {
        if (!P) return DFA_EINVAL;
        GLaunch l;
        const int rc = plan_launch(g, len, opts, &l);
        if (rc != DFA_OK) return rc;
        *P = l.p.P;
        return DFA_OK;
    });
}

int dfa_group_workspace_size(const dfa_group_t* g, uint64_t len, const dfa_group_opts_t* opts,
                             uint64_t* bytes) {
    return dfam::no_throw([&]() -> int {
        if (!bytes) return DFA_EINVAL;
        GLaunch l;
        const int rc = plan_launch(g, len, opts, &l);
        if (rc != DFA_OK) return rc;
        *bytes = l.ws_total;
        return DFA_OK;
    });
}

int dfa_group_match_async(const dfa_group_t* g, const uint8_t* dev_str, uint64_t len,
                          const dfa_group_opts_t* opts, dfa_result_t* dev_out, void* dev_workspace,
                          uint64_t workspace_bytes, void* stream) {
    return dfam::no_throw([&]() -> int {
        if (!g || !dev_out || !dev_workspace || (len && !dev_str)) return DFA_EINVAL;
        if (((uintptr_t)dev_out & 3u) || ((uintptr_t)dev_workspace & 255u)) return DFA_EINVAL;
        if (opts && opts->dev_work && ((uintptr_t)opts->dev_work & 7u)) return DFA_EINVAL;
        GLaunch l;
        const int rc = plan_launch(g, len, opts, &l);
        if (rc != DFA_OK) return rc;
        if (workspace_bytes < l.ws_total) return DFA_ENOSPACE;
        bind_ws(l, static_cast<uint8_t*>(dev_workspace));
        l.p.str = dev_str;
        l.p.results = dev_out;
        l.p.work = opts ? reinterpret_cast<unsigned long long*>(opts->dev_work) : nullptr;
        l.p.dbg = nullptr;
        return issue(l, g->sb, opts, stream);
    });
}

int dfa_group_match(dfa_group_t* g, const uint8_t* str, uint64_t len, const dfa_group_opts_t* opts,
                    dfa_result_t* out) {
    return dfam::no_throw([&]() -> int {
        if (!g || !out || (len && !str)) return DFA_EINVAL;
        if (!g->on_device) return DFA_EHOSTONLY;
        bool on_dev = false;
        if (len) {
            cudaPointerAttributes at;
            if (cudaPointerGetAttributes(&at, str) == cudaSuccess)
                on_dev = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
            cudaGetLastError();
        }
        GLaunch l;
        int rc = plan_launch(g, len, opts, &l);
        if (rc != DFA_OK) return rc;
        std::lock_guard<std::mutex> lock(g->mu);
        std::vector<uint64_t> seg;
        if (len && !on_dev && !(opts && (opts->num_chunks || opts->dev_work ||
                                          opts->match_begin_event || opts->match_end_event)) &&
            group_segments(g, len, &seg))
            return group_match_pipelined(g, str, seg, opts, out);
        const uint8_t* use = str;
        if (len && !on_dev) {
            if ((rc = grow_buf(&g->d_str, &g->str_cap, len)) != DFA_OK) return rc;
            if (cudaMemcpyAsync(g->d_str, str, len, cudaMemcpyHostToDevice, 0) != cudaSuccess)
                return DFA_ECUDA;
            use = g->d_str;
        }
        const uint64_t res_off = l.ws_total;
        if ((rc = grow_buf(&g->d_ws, &g->ws_cap, res_off + sizeof(dfa_result_t) * g->G)) != DFA_OK)
            return rc;
        bind_ws(l, g->d_ws);
        l.p.str = use;
        l.p.results = reinterpret_cast<dfa_result_t*>(g->d_ws + res_off);
        l.p.work = opts ? reinterpret_cast<unsigned long long*>(opts->dev_work) : nullptr;
        l.p.dbg = nullptr;
        if ((rc = issue(l, g->sb, opts, nullptr)) != DFA_OK) return rc;
        if (cudaMemcpy(out, l.p.results, sizeof(dfa_result_t) * g->G, cudaMemcpyDeviceToHost) != cudaSuccess)
            return DFA_ECUDA;
        return DFA_OK;
    });
}

int dfa_group_debug_chunk_maps(const dfa_group_t* g, const uint8_t* dev_str, uint64_t len,
                               const dfa_group_opts_t* opts, uint16_t* maps, uint32_t cap,
                               uint32_t* P, uint32_t* final_states) {
    return dfam::no_throw([&]() -> int {
        if (!g || !P || (len && !dev_str)) return DFA_EINVAL;
        GLaunch l;
        int rc = plan_launch(g, len, opts, &l);
        if (rc != DFA_OK) return rc;
        *P = l.p.P;
        if (!maps && !final_states) return DFA_OK;
        const uint64_t per = (uint64_t)g->G * l.p.P * g->qe_max;
        std::vector<uint16_t> host(per);
        for (uint64_t i = 0; i < per; ++i) host[i] = (uint16_t)(i % g->qe_max);  // identity outside I_k
        void *ws = nullptr, *dbg = nullptr, *res = nullptr;
        rc = DFA_OK;
        if (cudaMalloc(&ws, l.ws_total) != cudaSuccess || cudaMalloc(&dbg, per * 2) != cudaSuccess ||
            cudaMalloc(&res, sizeof(dfa_result_t) * g->G) != cudaSuccess) {
            cudaGetLastError();
            rc = DFA_ENOMEM;
        }
        if (rc == DFA_OK && cudaMemcpy(dbg, host.data(), per * 2, cudaMemcpyHostToDevice) != cudaSuccess)
            rc = DFA_ECUDA;
        if (rc == DFA_OK) {
            bind_ws(l, static_cast<uint8_t*>(ws));
            l.p.str = dev_str;
            l.p.results = static_cast<dfa_result_t*>(res);
            l.p.work = nullptr;
            l.p.dbg = static_cast<uint16_t*>(dbg);
            rc = issue(l, g->sb, opts, nullptr);
            if (rc == DFA_OK && cudaStreamSynchronize(nullptr) != cudaSuccess) rc = DFA_ECUDA;
        }
        std::vector<dfa_result_t> r(g->G);
        if (rc == DFA_OK &&
            (cudaMemcpy(host.data(), dbg, per * 2, cudaMemcpyDeviceToHost) != cudaSuccess ||
             cudaMemcpy(r.data(), res, sizeof(dfa_result_t) * g->G, cudaMemcpyDeviceToHost) != cudaSuccess))
            rc = DFA_ECUDA;
        cudaFree(ws);
        cudaFree(dbg);
        cudaFree(res);
        if (rc != DFA_OK) return rc;
        if (maps) {
            const uint32_t np = std::min(cap, l.p.P);
            for (uint32_t i = 0; i < g->G; ++i)
                std::memcpy(maps + (uint64_t)i * np * g->qe_max, host.data() + (uint64_t)i * l.p.P * g->qe_max,
                            2ull * np * g->qe_max);
        }
        if (final_states)
            for (uint32_t i = 0; i < g->G; ++i) final_states[i] = r[i].status ? 0xFFFFFFFFu : r[i].final_state;
        return DFA_OK;
    });
}

}  // extern "C"
