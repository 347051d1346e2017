// Internal structures of libdfamatch: the compiled DFA (host and device
// images), per-launch plans and the kernel launchers.
#pragma once

#include <cstddef>
#include <cstdint>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/dfamatch.h"

namespace dfam {

// ------------------------------------------------------------------ tuning
constexpr int kThreads = 512;            // threads per CTA of the match kernel
constexpr int kMaxChunksPerTile = kThreads / 2;  // every chunk is charged >= 2 thread slots
constexpr int kMaxSegLen = 2048;         // longest staged segment per chunk (positions)
constexpr uint16_t kNone16 = 0xFFFF;     // "not a member" in pos tables / invalid byte
constexpr uint32_t kNone32 = 0xFFFFFFFFu;
constexpr uint32_t kSmemTableMax = 112 * 1024;  // tables larger than this are read through L2
constexpr uint32_t kMaxStates = 65534;      // |Q| limit: states and q_e are 16-bit ids, 0xFFFF reserved
// Launches whose largest set (the capacity of a running state map) exceeds
// this keep each CTA's running map in global memory instead of shared memory.
constexpr uint32_t kSmemVcap = 4096;
// Largest |Q|+1 for the sets of Eq. (13) computed per chunk (k_lookahead keeps a
// bitmap over Q and a set buffer per warp in shared memory) and for the map
// tests of the pipelined host path (one register per state per thread).
constexpr uint32_t kMaxSmallQe = 4096;
constexpr uint32_t kMaxLookahead = 8;    // reverse-lookahead symbols r of Eq. (13)
constexpr uint32_t kMaxBoundaryWindow = 65536;  // largest Sec. 4.2 placement window (bytes)

// Tuning records and launch descriptors exist per lookahead depth r, once for
// the chunk starts of Eqs. (6)-(7) and once for starts placed by Sec. 4.2
// (the placed sets are far smaller, so the best K and tiles differ).
constexpr uint32_t kTuningSlots = 2 * (kMaxLookahead + 1);
inline uint32_t tuning_slot(uint32_t lookahead, bool placed) {
    return lookahead + (placed ? kMaxLookahead + 1 : 0u);
}
inline uint32_t slot_lookahead(uint32_t slot) { return slot % (kMaxLookahead + 1); }

enum Placement : uint32_t { kSmem = 0, kGlobal = 1 };

// Chains per thread the compiler picks for chunks whose sets have about
// `size` states (before the tile-fit rule raises it for I_max).
inline uint32_t k_for_set_size(double size) { return size >= 48 ? 8u : (size >= 12 ? 4u : 2u); }

// ------------------------------------------------------- device DFA image
// Everything the kernels read about one DFA.  Pointers are device pointers.
struct DevDfa {
    const uint8_t* table;        // (C+1) rows x qpad entries of sb bytes (1, 2 or 4); entry = next_state*sb;
                                 // row C is the identity row used to pad chunk tails
    const uint16_t* byte_off16;  // [256] byte -> row byte offset c*qpad*sb (kNone16: not in Sigma)
    const uint32_t* byte_off32;  // [256] same, 32-bit (global placement)
    const uint16_t* byte_class;  // [256] byte -> class (kNone16: not in Sigma)
    const uint32_t* iset_off;    // [C+3] CSR offsets; set C = start set {q0}, set C+1 = all of Q
    const uint16_t* iset;        // CSR members (ascending)
    const uint16_t* pos;         // [(C+2)*qe] index of state s in set c, kNone16 if absent
    const uint8_t* accept;       // [qe] 1 iff accepting
    const uint8_t* excluded;     // [qe] 1 iff left out of every initial-state set
    const uint32_t* byte_plan;   // [256] (class << 16) | |I_class|; kNone32 for bytes outside Sigma
    uint32_t qe;                 // states incl. q_e
    uint32_t qpad;               // row stride (entries)
    uint32_t C;                  // classes (without the start set)
    uint32_t sb;                 // bytes per table entry (1, 2, or 4 when |Q|+1 > 32768)
    uint32_t placement;          // Placement
    uint32_t table_bytes;        // (C+1)*qpad*sb
    uint32_t q0;
    uint32_t imax;               // Eq. (12) over real classes
    uint32_t K;                  // states per thread
    uint32_t vcap;               // largest set size (incl. start set) = capacity of a state map
    uint32_t stage_fmt;          // StageFmt of the staged input stream
    uint32_t n_all;              // |Q| minus the excluded states: the set Algorithm 2 matches
    uint32_t nib;                // 1: at most 16 live states, byte rows available (nib_rows)
    const uint8_t* nib_rows;     // nib: (C+1) rows of 16 bytes, byte s = nib_code(delta(s, c))
    const uint16_t* nib_off16;   // nib: [256] byte -> byte-row offset class * 16 (kNone16: not in Sigma)
};

// Byte rows for DFAs whose chains only ever visit 16 states or fewer (every
// state, or every state but an unreachable q_e): row c holds, in byte s,
// the code of delta(s, c), so one step of a chain is a byte permute of the
// row (two 8-byte halves, picked by bit 7 of the code) instead of a
// dependent table load.  Code of state s: the low 3 bits of s, and bit 3 of
// s moved to bit 7, so the code's low nibble is a clean permute selector.
#ifdef __CUDACC__
__host__ __device__
#endif
inline uint32_t nib_code(uint32_t s) { return (s & 7u) | ((s & 8u) << 4); }
#ifdef __CUDACC__
__host__ __device__
#endif
inline uint32_t nib_state(uint32_t code) { return (code & 7u) | ((code >> 4) & 8u); }

// How a chunk's input is staged in shared memory: 8-bit class indices
// (16 positions per 16-byte read; shared-memory tables with at most 254
// classes), 16-bit row byte offsets (other shared-memory tables) or 32-bit
// row byte offsets (tables read through L2).
enum StageFmt : uint32_t { kCls8 = 0, kOff16 = 1, kOff32 = 2 };

// Bytes per staged position of a stage format.
#ifdef __CUDACC__
__host__ __device__
#endif
constexpr uint32_t stage_esz(uint32_t fmt) {
    return fmt == kOff32 ? 4u : (fmt == kOff16 ? 2u : 1u);
}

// One membership test of a launch.
struct DevTest {
    const uint8_t* str;
    uint64_t n;
    uint64_t qinv;        // floor((2^64 - 1) / (m + P - 1)): Eq. (6)'s divisor, inverted once
    uint32_t dfa;         // index into the launch's DevDfa array
    uint32_t P;           // chunks
    uint32_t m;           // multiplicity of Eq. (10) used in the partition
    uint32_t chunk_base;  // global index of its chunk 0
    uint32_t group;       // run of consecutive tests sharing one DFA
    uint32_t lookahead;   // 1: Algorithm 3, 0: Algorithm 2 (all states)
    uint32_t out;         // index of its result in the caller's output array
    uint32_t flags;       // kTestCont, kTestMap
    uint32_t window;      // Sec. 4.2 placement window actually searched (0: Eqs. 6-7 starts)
    uint32_t pad_;
};
static_assert(sizeof(DevTest) == 64, "DevTest layout");

// floor((2^64 - 1) / q) for q >= 1: the reciprocal the device uses to divide
// by q with one 64-bit multiply-high and at most two corrections.
inline uint64_t recip64(uint64_t q) { return ~0ull / q; }

// A continuation test is one segment of a longer string whose earlier
// segments were matched by earlier launches on the same stream: the bytes
// before `str` are readable, its chunk 0 is speculative like any other chunk
// (reverse lookahead into the previous segment), and Eq. (8) starts from the
// final state (and status) already in its result slot instead of q0.
constexpr uint32_t kTestCont = 1;
// A map test (always also a continuation) publishes the state map of its
// whole string instead of a final state: map[s] = delta*(s, str) for every s
// that can enter it (the reverse-lookahead set of its first chunk and the
// excluded states; other entries are the identity), written to
// LaunchPlan::maps + out * map_stride.  Its result slot gets only the status.
constexpr uint32_t kTestMap = 2;

struct DevGroup {
    uint32_t first_chunk, end_chunk, dfa, first_test;
    uint32_t set_stride;  // entries per chunk in the lookahead-set arena (r >= 2)
    uint32_t pad_;
    uint64_t set_base;    // offset (entries) of the group's first chunk in that arena
};
static_assert(sizeof(DevGroup) == 32, "DevGroup layout");

// Set index of a chunk whose initial-state set was computed from r >= 2
// lookahead symbols (Eq. 13) and stored in the launch's set arena.
#ifdef __CUDACC__
__host__ __device__
#endif
inline uint32_t dyn_set(uint32_t C) { return C + 2; }

// Device-side result (layout identical to dfa_result_t).
static_assert(sizeof(dfa_result_t) == 12, "dfa_result_t layout");

// Per-launch device workspace (all pointers into one caller-provided block).
struct LaunchPlan {
    const DevDfa* dfas;
    const DevTest* tests;
    const DevGroup* groups;
    uint32_t ntests, ngroups, ptot, nblk;
    uint32_t grid;              // CTAs of the match kernel
    uint32_t waves;             // grid / CTAs that fit the GPU at once (0 or 1: one wave)
    uint32_t seg_stride;        // entries per segment map
    uint32_t smem_table_cap;    // bytes reserved for a shared-memory table
    uint32_t vcap;              // entries reserved for the running map
    uint32_t stage_bytes;       // bytes of one of the two stage buffers
    uint32_t* chunk_test;       // [ptot]
    uint16_t* chunk_cls;        // [ptot]
    uint32_t* cost;             // [ptot] packing word (thread slots, opens-a-tile flag);
                                // then scratch for the tile starts of each CTA share
    uint32_t* off;              // [ptot+1] exclusive prefix of cost (within the launch)
    uint64_t* wk;               // [ptot+1] scratch: chunk work (slots x length) or its midpoint
    uint32_t* bsum;             // [nblk+1]
    uint64_t* bsumw;            // [nblk+1] block sums of wk
    uint32_t* tile_first;       // [ptot+1]
    uint32_t* ccta;             // [ptot] CTA share of each chunk
    uint32_t* share;            // [grid+1] first chunk of each CTA share
    uint32_t* ntiles;           // [grid+1] tiles per share, then their bases
    uint32_t* num_tiles;        // [1]
    uint32_t* test_err;         // [ntests]
    uint32_t* arrived;          // [ntests]
    uint32_t* cta_range;        // [2*grid] tiles [first, end) of each CTA (cleared: empty)
    uint32_t* first_cta;        // [ntests]
    uint32_t* last_cta;         // [ntests]
    uint32_t* seg_hdr;          // [(grid+ntests)*4]: first chunk, nchunks, -, -
    uint16_t* seg_vals;         // [(grid+ntests)*seg_stride]: dense maps over Q
    uint16_t* sets;             // lookahead-set arena (r >= 2), see DevGroup
    uint32_t* set_size;         // [ptot] |I| of each chunk computed by k_lookahead
    uint32_t dyn;               // 1 if some test uses r >= 2 lookahead symbols
    uint32_t no_nib;            // 1: match byte-row DFAs from their class-major tables instead
    uint32_t bnd;               // 1 if some test places its chunk starts (Sec. 4.2)
    uint64_t* starts;           // [ptot] start of every chunk k >= 1 of a placing test
    uint16_t* dbg_maps;         // optional [ptot * qe_max]: chunk maps L_k (identity pre-filled)
    uint16_t* big_maps;         // vcap > kSmemVcap: [grid][2][vmap_stride] running map and its domain
    uint32_t vmap_stride;       // entries per running-map array in big_maps
    uint32_t qe_max;            // largest |Q|+1 of the launch's DFAs
    dfa_result_t* results;      // [ntests] in the caller's order (DevTest::out)
    uint16_t* maps;             // map tests: their state maps, map_stride entries each
    uint32_t map_stride;
    // single-test launches carry their descriptors by value (tests/groups == nullptr)
    DevTest test1;
    DevGroup group1;
};

// Workspace carve-up of one launch (byte offsets into the device workspace).
struct WsLayout {
    uint64_t dfas, tests, groups, chunk_test, chunk_cls, cost, off, wk, bsum, bsumw, tile_first,
        ccta, share, ntiles, num_tiles, test_err, first_cta, last_cta, seg_hdr, seg_vals, set_size, sets,
        starts, big_maps, total;
};

// A batch planned on the host: descriptors, sizes and the workspace layout.
struct Prepared {
    std::vector<DevDfa> dfas;
    std::vector<DevTest> tests;
    std::vector<DevGroup> groups;
    uint32_t ptot = 0, nblk = 0, grid = 0, kmax = 2, vcap = 1, table_cap = 0, smem = 0, stage = 0;
    uint32_t qe_max = 1, dyn = 0, bnd = 0;
    uint64_t set_entries = 0;
    WsLayout ws{};
};

// ------------------------------------------------------------ host image
struct HostDfa {
    uint32_t Q = 0, S = 0, qe = 0, q0 = 0, C = 0, qpad = 0, sb = 0;
    uint32_t imax = 0, num_excluded = 0, placement = kSmem, K = 4;
    uint32_t K0 = 4;  // the compiler's K (from the mean set size), kept when tuning changes K
    double gamma = 0, mean_iset = 0;
    std::vector<uint16_t> byte_class;   // 256, kNone16 = not in Sigma
    std::vector<uint8_t> accept;        // qe
    std::vector<uint8_t> excluded;      // qe
    std::vector<uint32_t> iset_off;     // C+3
    std::vector<uint16_t> iset;
    std::vector<uint16_t> pos;          // (C+2)*qe
    std::vector<uint8_t> table;         // (C+1)*qpad*sb
    std::vector<uint16_t> byte_off16;   // 256
    std::vector<uint32_t> byte_off32;   // 256
    std::vector<uint8_t> nib_rows;      // (C+1) x 16 when at most 16 states are live, else empty
};

// Runs an entry point's body; a failed host allocation becomes DFA_ENOMEM (and
// any other C++ exception DFA_EINVAL), so no exception crosses the C ABI.
template <typename F>
inline int no_throw(F&& f) {
    try {
        return f();
    } catch (const std::bad_alloc&) {
        return DFA_ENOMEM;
    } catch (...) {
        return DFA_EINVAL;
    }
}

// Compile (validation, classes, excluded states, I sets, table image).
int compile_dfa(uint32_t num_states, uint32_t num_symbols, const int32_t* delta, uint32_t q0,
                const uint32_t* finals, uint32_t num_finals, const uint8_t* byte_to_symbol,
                HostDfa* out);

uint64_t chunk_start(uint64_t n, uint32_t P, uint32_t m, uint32_t k);

}  // namespace dfam

struct dfa_s;
namespace dfam {
// Batch planning and launching (dfa_api.cu), shared with the serving loop.
// out_ids (optional): the result index of each test (default: its position).
int prepare(uint32_t count, const dfa_s* const* dfas, const uint8_t* const* strs,
            const uint64_t* lens, const dfa_match_opts_t* opts, bool batched, Prepared* out,
            const uint32_t* out_ids = nullptr);
int prepare_parts(uint32_t count, const dfa_s* const* dfas, const uint8_t* const* strs,
                  const uint64_t* lens, const dfa_match_opts_t* opts, std::vector<Prepared>* parts,
                  std::vector<uint64_t>* ws_off, uint64_t* ws_total);
void fill_plan(const Prepared& p, LaunchPlan& lp, uint8_t* ws, dfa_result_t* out);
int upload_desc_async(const Prepared& p, uint8_t* ws, uint8_t* pinned, void* stream);
uint64_t desc_span(const Prepared& p);
int launch_prepared(const Prepared& p, uint8_t* ws, dfa_result_t* out, void* stream);

// Single-test launch: plan (descriptors by value), workspace layout, binding.
struct Single {
    LaunchPlan lp;
    WsLayout ws;
    uint32_t smem, kmax;
};
int plan_single(const dfa_s* d, uint64_t len, const dfa_match_opts_t* opts, Single* s);
void bind(LaunchPlan& lp, uint8_t* base, const WsLayout& w);
int launch_single(const Single& s, void* stream, void* ev_begin, void* ev_end);
// Eq. (8) over the segments of one string: the first segment's result, then
// the state maps of the map tests that follow it (one thread, on `st`).
int launch_compose_segments(const dfa_result_t* seg_res, const uint16_t* maps, uint32_t stride,
                            uint32_t nseg, const uint8_t* accept, dfa_result_t* out, void* st);
}  // namespace dfam

// The opaque handle of the C ABI.
struct dfa_s {
    dfam::HostDfa h;
    bool on_device = false;
    int device = -1;
    void* dev_block = nullptr;       // one allocation holding every device array
    uint64_t dev_bytes = 0;
    dfam::DevDfa dev;                // pointers into dev_block
    // device descriptors for launches of every tuning slot (lookahead r = 0 ..
    // kMaxLookahead, with and without Sec. 4.2 placement; dfam::tuning_slot),
    // each with the K of that slot's tuning
    dfam::DevDfa* dev_desc = nullptr;
    const dfam::DevDfa* dev_desc_for(uint32_t slot) const;
    dfa_tuning_t tuning{};           // base tuning record (dfa_set_tuning / dfa_autotune)
    // records of one slot (dfa_set_tuning_opts / dfa_autotune_opts); a placed
    // slot without its own record uses its depth's record, a depth without
    // its own record the base record
    dfa_tuning_t tuning_r[dfam::kTuningSlots]{};
    bool has_tuning_r[dfam::kTuningSlots]{};
    // device-only rate (GB/s) the autotuner measured for each slot's chosen
    // tuning on its sample (0: not autotuned); sizes the host pipeline's segments
    double tuned_gbs[dfam::kTuningSlots]{};
    const dfa_tuning_t& tuning_for(uint32_t slot) const {
        if (slot < dfam::kTuningSlots && has_tuning_r[slot]) return tuning_r[slot];
        if (slot > dfam::kMaxLookahead && slot < dfam::kTuningSlots)
            return tuning_for(slot - (dfam::kMaxLookahead + 1));
        return tuning;
    }
};
