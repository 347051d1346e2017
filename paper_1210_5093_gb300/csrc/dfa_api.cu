// C ABI of libdfamatch (declared in include/dfamatch.h): DFA creation and
// upload, the planner (partition of Eqs. 6-7/10 and launch layout), and the
// synchronous, asynchronous and batched match calls.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "dfa_internal.h"

namespace dfam {
uint32_t match_smem_bytes(uint32_t table_cap, uint32_t kmax, uint32_t vcap, uint32_t esz_max,
                          uint32_t* stage_bytes, uint32_t target);
uint32_t match_target_ctas(uint32_t kmax, uint32_t want);
int match_grid(uint32_t smem, uint32_t kmax, uint32_t* grid);
uint32_t launch_kernel_count(uint32_t ptot, uint32_t grid, bool dyn, bool bnd);
uint32_t device_sms();
int launch_plan(const LaunchPlan& lp, uint32_t kmax, uint32_t smem, cudaStream_t st,
                uint32_t* kernels, void* ev_begin = nullptr, void* ev_end = nullptr,
                bool plan_only = false);

constexpr uint32_t kTilesPerCta = 8;       // persistent CTAs each get about this many tiles
constexpr uint64_t kMinChunk = 512;        // bytes; shorter chunks cost more in tile overhead
constexpr uint32_t kBatchSmemTable = 64 * 1024;  // largest shared-memory table in a multi-DFA launch
constexpr uint32_t kBatchKMax = 8;                // largest K in a multi-DFA launch, unless needed
constexpr uint64_t kBatchChunk = 8192;     // default chunk length for batched tests
constexpr uint64_t kBatchChunksTarget = 65536;  // chunks a batched launch aims for at least
constexpr uint64_t kBatchChunkMin = 2048;       // shortest batched chunk
constexpr uint64_t kMaxChunk = 1ull << 31; // chunk lengths are 32-bit on the device
constexpr uint32_t kMaxWaves = 4;          // largest dfa_tuning_t.grid_waves

inline uint64_t up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

// Entries per running-map array of one CTA when a launch's maps live in global
// memory (vcap > kSmemVcap), else 0.
inline uint32_t vmap_stride_for(uint32_t vcap) { return vcap > kSmemVcap ? (vcap + 7u) & ~7u : 0u; }

WsLayout ws_layout(uint32_t ndfa, uint32_t ntests, uint32_t ngroups, uint32_t ptot, uint32_t nblk,
                   uint32_t grid, uint32_t stride, bool inline_desc, bool dyn = false,
                   uint64_t set_entries = 0, bool bnd = false, uint32_t vcap = 0) {
    WsLayout w;
    uint64_t o = 0;
    auto take = [&](uint64_t bytes) { uint64_t r = o; o = up(o + bytes, 256); return r; };
    w.dfas = take(inline_desc ? 0 : sizeof(DevDfa) * ndfa);
    w.tests = take(inline_desc ? 0 : sizeof(DevTest) * ntests);
    w.groups = take(inline_desc ? 0 : sizeof(DevGroup) * ngroups);
    w.chunk_test = take(4ull * ptot);
    w.chunk_cls = take(2ull * ptot);
    w.cost = take(4ull * ptot);
    w.off = take(4ull * (ptot + 1));
    w.wk = take(8ull * (ptot + 1));
    w.bsum = take(4ull * (nblk + 1));
    w.bsumw = take(8ull * (nblk + 1));
    w.tile_first = take(4ull * (ptot + 1));
    w.ccta = take(4ull * ptot);
    w.share = take(4ull * (grid + 1));
    w.ntiles = take(4ull * (grid + 1));
    w.num_tiles = take(4);
    w.test_err = take(8ull * ntests + 8ull * grid);  // test_err, arrived, cta_range
    w.first_cta = take(4ull * ntests);
    w.last_cta = take(4ull * ntests);
    w.seg_hdr = take(16ull * (grid + ntests));
    w.seg_vals = take(2ull * stride * (grid + ntests));
    w.set_size = take(dyn ? 4ull * ptot : 0);
    w.sets = take(dyn ? 2ull * set_entries : 0);
    w.starts = take(bnd ? 8ull * ptot : 0);
    w.big_maps = take(2ull * 2 * vmap_stride_for(vcap) * grid);
    w.total = o;
    return w;
}

void bind(LaunchPlan& lp, uint8_t* base, const WsLayout& w) {
    lp.chunk_test = reinterpret_cast<uint32_t*>(base + w.chunk_test);
    lp.chunk_cls = reinterpret_cast<uint16_t*>(base + w.chunk_cls);
    lp.cost = reinterpret_cast<uint32_t*>(base + w.cost);
    lp.off = reinterpret_cast<uint32_t*>(base + w.off);
    lp.wk = reinterpret_cast<uint64_t*>(base + w.wk);
    lp.bsum = reinterpret_cast<uint32_t*>(base + w.bsum);
    lp.bsumw = reinterpret_cast<uint64_t*>(base + w.bsumw);
    lp.tile_first = reinterpret_cast<uint32_t*>(base + w.tile_first);
    lp.ccta = reinterpret_cast<uint32_t*>(base + w.ccta);
    lp.share = reinterpret_cast<uint32_t*>(base + w.share);
    lp.ntiles = reinterpret_cast<uint32_t*>(base + w.ntiles);
    lp.num_tiles = reinterpret_cast<uint32_t*>(base + w.num_tiles);
    lp.test_err = reinterpret_cast<uint32_t*>(base + w.test_err);
    lp.arrived = lp.test_err + lp.ntests;
    lp.cta_range = lp.arrived + lp.ntests;
    lp.first_cta = reinterpret_cast<uint32_t*>(base + w.first_cta);
    lp.last_cta = reinterpret_cast<uint32_t*>(base + w.last_cta);
    lp.seg_hdr = reinterpret_cast<uint32_t*>(base + w.seg_hdr);
    lp.seg_vals = reinterpret_cast<uint16_t*>(base + w.seg_vals);
    lp.set_size = reinterpret_cast<uint32_t*>(base + w.set_size);
    lp.sets = reinterpret_cast<uint16_t*>(base + w.sets);
    lp.starts = reinterpret_cast<uint64_t*>(base + w.starts);
    lp.big_maps = reinterpret_cast<uint16_t*>(base + w.big_maps);
}

// Reverse-lookahead symbols requested by opts: 1 (Algorithm 3) by default,
// 0 for Algorithm 2, up to kMaxLookahead for Eq. (13).
inline uint32_t opts_lookahead(const dfa_match_opts_t* o) { return o ? o->lookahead : 1u; }
// Sec. 4.2 placement window requested by opts (0: the starts of Eqs. 6-7).
inline uint32_t opts_window(const dfa_match_opts_t* o) { return o ? o->boundary_window : 0u; }
// The tuning slot of a call: its lookahead depth, placed or not.  Algorithm 2
// has no lookahead symbol to place by, so it always takes the unplaced slot.
inline uint32_t opts_slot(const dfa_match_opts_t* o) {
    const uint32_t r = opts_lookahead(o);
    return tuning_slot(r, r != 0 && opts_window(o) != 0);
}
inline bool opts_valid(const dfa_match_opts_t* o) {
    return opts_lookahead(o) <= kMaxLookahead && opts_window(o) <= kMaxBoundaryWindow;
}
// The sets of Eq. (13) (r >= 2) are computed per chunk for DFAs of at most
// kMaxSmallQe states (q_e included).
inline bool lookahead_ok(const dfa_t* d, const dfa_match_opts_t* o) {
    return opts_lookahead(o) < 2 || d->h.qe <= kMaxSmallQe;
}
// Chains per thread a tuning may use: every chunk's chains fit one tile at K,
// or K = 16 (larger sets then run in several passes over their chunk).
inline bool k_allowed(const dfa_t* d, uint32_t K) {
    return K == 16 || (std::max(d->h.imax, 1u) + K - 1) / K <= (uint32_t)kThreads / 2;
}

// The window a test of n bytes in P chunks (multiplicity m) actually searches:
// at most a quarter of floor(n / (m + P - 1)), the shortest chunk after the
// first, so the window lies inside the string and placed starts stay strictly
// increasing; none for Algorithm 2 or a single chunk.
uint32_t test_window(const dfa_match_opts_t* o, uint64_t n, uint32_t P, uint32_t m) {
    const uint32_t w = opts_window(o);
    if (w == 0 || opts_lookahead(o) == 0 || P <= 1) return 0;
    const uint64_t quarter = n / ((uint64_t)m + P - 1) / 4;
    return (uint32_t)std::min<uint64_t>(w, quarter);
}
// Entries per segment map: |Q|+1 rounded up to 8, so every map starts on a
// 16-byte boundary (the combine stages them with 16-byte loads).
inline uint32_t seg_stride_for(uint32_t qe_max) { return (qe_max + 7) & ~7u; }

// Bytes of a shared-memory DFA's table image in k_match's shared memory: its
// byte rows when it has them, else its class-major table.
inline uint32_t smem_table_bytes(const DevDfa& x) {
    return (uint32_t)up(x.nib ? (x.C + 1) * 16u : x.table_bytes, 16);
}

// Launch-specific copy of a DFA's device descriptor for a tuning slot.  K is
// raised when the largest set the launch matches would not fit one tile.
DevDfa launch_desc(const dfa_t* d, uint32_t slot) {
    DevDfa x = d->dev;
    const uint32_t lookahead = slot_lookahead(slot);
    const uint32_t tk = d->tuning_for(slot).states_per_thread;
    x.K = tk ? tk : d->h.K;
    const uint32_t vmax = lookahead ? std::max(d->h.imax, 1u) : d->h.qe;
    while ((vmax + x.K - 1) / x.K > (uint32_t)kThreads / 2 && x.K < 16) x.K *= 2;
    x.vcap = vmax;
    return x;
}

// Chunk count for one test (Sec. 4.1's partition is applied per test with P
// chunks).  Batched tests use the DFA's batched chunk length, at most
// batch_cap bytes (the launch's bytes spread over kBatchChunksTarget chunks):
// a launch holding little input gets shorter chunks and so more parallelism.
uint32_t plan_chunks(const dfa_t* d, uint64_t n, uint32_t grid, const dfa_match_opts_t* o,
                     bool batched, uint64_t batch_cap) {
    const dfa_tuning_t& tu = d->tuning_for(opts_slot(o));
    uint64_t P;
    if (o && o->num_chunks) {
        P = o->num_chunks;
    } else if (batched) {
        uint64_t L = tu.batch_chunk_bytes ? tu.batch_chunk_bytes : kBatchChunk;
        if (batch_cap) L = std::min(L, batch_cap);
        P = (n + L - 1) / L;
    } else {
        // enough lane tasks for kTilesPerCta tiles on every CTA, chunks >= kMinChunk;
        // a chunk costs its set's thread slots: the mean over the classes, or with
        // Sec. 4.2 placement the smallest set (the one the placement looks for)
        double mean_cost = 0, min_cost = 1e30;
        const HostDfa& h = d->h;
        for (uint32_t c = 0; c < h.C; ++c) {
            uint32_t sz = h.iset_off[c + 1] - h.iset_off[c];
            const uint32_t K = tu.states_per_thread ? tu.states_per_thread : h.K;
            const double cost = std::max((sz + K - 1) / K, 2u);
            mean_cost += cost;
            min_cost = std::min(min_cost, cost);
        }
        mean_cost = h.C ? mean_cost / h.C : 2.0;
        if (h.C && opts_slot(o) > kMaxLookahead) mean_cost = min_cost;
        const uint32_t tpc = tu.tiles_per_cta ? tu.tiles_per_cta : kTilesPerCta;
        double want = (double)grid * kThreads * tpc * 0.9 / mean_cost;
        uint64_t by_len = n / (tu.min_chunk_bytes ? tu.min_chunk_bytes : kMinChunk);
        P = std::min<uint64_t>((uint64_t)want, by_len);
    }
    P = std::max<uint64_t>(P, (n + kMaxChunk - 1) / kMaxChunk);
    P = std::max<uint64_t>(P, 1);
    P = std::min<uint64_t>(P, 1ull << 30);
    return (uint32_t)P;
}

int prepare(uint32_t count, const dfa_t* const* dfas, const uint8_t* const* strs,
            const uint64_t* lens, const dfa_match_opts_t* opts, bool batched, Prepared* out,
            const uint32_t* out_ids) {
    if (count == 0 || !dfas || !strs || !lens) return DFA_EINVAL;
    if (!opts_valid(opts)) return DFA_EINVAL;
    const uint32_t lookahead = opts_lookahead(opts), slot = opts_slot(opts);
    const uint32_t m = (opts && opts->multiplicity) ? opts->multiplicity : 1u;
    Prepared p;
    // group tests by DFA (stable), unique DFAs in first-seen order
    std::map<const dfa_t*, uint32_t> idx;
    std::vector<const dfa_t*> uniq;
    for (uint32_t i = 0; i < count; ++i) {
        const dfa_t* d = dfas[i];
        if (!d) return DFA_EINVAL;
        if (!d->on_device) return DFA_EHOSTONLY;
        if (lens[i] && !strs[i]) return DFA_EINVAL;
        if (!lookahead_ok(d, opts)) return DFA_EINVAL;
        if (!idx.count(d)) {
            idx[d] = (uint32_t)uniq.size();
            uniq.push_back(d);
        }
    }
    for (const dfa_t* d : uniq) {
        DevDfa x = launch_desc(d, slot);
        // batched launches are bound by the shared-memory pipe, where a byte
        // row (a 16-byte read per step) costs more than a table lookup
        x.nib = 0;
        if (uniq.size() > 1) {
            // One launch has one kernel variant and one shared-memory layout,
            // sized for its largest K and largest shared-memory table.  In a
            // launch of several DFAs each DFA takes the compiler's K (from its
            // mean set size; a single-test tuning says little about a mixed
            // launch), capped at kBatchKMax unless a chunk's chains need more
            // to fit a tile, and a table above kBatchSmemTable is read through
            // L2, so that one DFA does not cut the occupancy of every other test.
            if (x.placement == kSmem && smem_table_bytes(x) > kBatchSmemTable) {
                x.placement = kGlobal;
                x.stage_fmt = kOff32;
                x.nib = 0;
            }
            // With Sec. 4.2 placement the chunks start after the symbols of the
            // smallest sets, so K follows the smallest set instead of the mean.
            uint32_t K0 = d->h.K0;
            if (slot > kMaxLookahead && d->h.C) {
                uint32_t smallest = ~0u;
                for (uint32_t c = 0; c < d->h.C; ++c)
                    smallest = std::min(smallest, d->h.iset_off[c + 1] - d->h.iset_off[c]);
                K0 = k_for_set_size(std::max(1u, smallest));
            }
            uint32_t K = std::min(K0, kBatchKMax);
            while ((x.vcap + K - 1) / K > (uint32_t)kThreads / 2 && K < 16) K *= 2;
            x.K = K;
        }
        p.dfas.push_back(x);
        p.kmax = std::max(p.kmax, x.K);
        p.vcap = std::max(p.vcap, x.vcap);
        p.qe_max = std::max(p.qe_max, x.qe);
        if (x.placement == kSmem) p.table_cap = std::max(p.table_cap, smem_table_bytes(x));
    }
    uint32_t esz_max = 1;
    for (const DevDfa& x : p.dfas) esz_max = std::max(esz_max, stage_esz(x.stage_fmt));
    p.smem = match_smem_bytes(p.table_cap, p.kmax, p.vcap, esz_max, &p.stage,
                              match_target_ctas(p.kmax, 0));
    int rc = match_grid(p.smem, p.kmax, &p.grid);
    if (rc != DFA_OK) return rc;
    uint64_t total = 0;
    for (uint32_t i = 0; i < count; ++i) total += lens[i];
    const uint64_t batch_cap = std::max<uint64_t>(kBatchChunkMin, total / kBatchChunksTarget);
    std::vector<uint32_t> order(count);
    for (uint32_t i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](uint32_t a, uint32_t b) { return idx[dfas[a]] < idx[dfas[b]]; });
    uint64_t chunks = 0;
    for (uint32_t j = 0; j < count; ++j) {
        const uint32_t i = order[j];
        const dfa_t* d = dfas[i];
        DevTest t{};
        t.str = strs[i];
        t.n = lens[i];
        t.dfa = idx[d];
        t.P = plan_chunks(d, lens[i], p.grid, opts, batched, batch_cap);
        t.m = m;
        t.qinv = recip64((uint64_t)m + t.P - 1);
        t.chunk_base = (uint32_t)chunks;
        t.lookahead = lookahead;
        t.window = test_window(opts, t.n, t.P, m);
        p.bnd |= t.window ? 1u : 0u;
        t.out = out_ids ? out_ids[i] : i;
        if (p.groups.empty() || p.groups.back().dfa != t.dfa) {
            if (!p.groups.empty()) {
                const DevGroup& pg = p.groups.back();
                p.set_entries += (uint64_t)(pg.end_chunk - pg.first_chunk) * pg.set_stride;
            }
            DevGroup g{};
            g.first_chunk = (uint32_t)chunks;
            g.dfa = t.dfa;
            g.first_test = j;
            g.set_stride = std::max(d->h.imax, 1u);
            g.set_base = p.set_entries;
            p.groups.push_back(g);
        }
        t.group = (uint32_t)p.groups.size() - 1;
        chunks += t.P;
        p.groups.back().end_chunk = (uint32_t)chunks;
        if (chunks > 0xF0000000ull) return DFA_EINVAL;
        p.tests.push_back(t);
    }
    p.ptot = (uint32_t)chunks;
    p.nblk = (p.ptot + 1023) / 1024;
    {
        const DevGroup& pg = p.groups.back();
        p.set_entries += (uint64_t)(pg.end_chunk - pg.first_chunk) * pg.set_stride;
    }
    p.dyn = lookahead >= 2 ? 1u : 0u;
    p.ws = ws_layout((uint32_t)p.dfas.size(), count, (uint32_t)p.groups.size(), p.ptot, p.nblk,
                     p.grid, seg_stride_for(p.qe_max), false, p.dyn != 0, p.set_entries,
                     p.bnd != 0, p.vcap);
    *out = std::move(p);
    return DFA_OK;
}

void fill_plan(const Prepared& p, LaunchPlan& lp, uint8_t* ws, dfa_result_t* out) {
    std::memset(&lp, 0, sizeof lp);
    lp.ntests = (uint32_t)p.tests.size();
    lp.ngroups = (uint32_t)p.groups.size();
    lp.ptot = p.ptot;
    lp.nblk = p.nblk;
    lp.grid = p.grid;
    lp.seg_stride = seg_stride_for(p.qe_max);
    lp.smem_table_cap = p.table_cap;
    lp.vcap = p.vcap;
    lp.vmap_stride = vmap_stride_for(p.vcap);
    lp.qe_max = p.qe_max;
    lp.dyn = p.dyn;
    lp.bnd = p.bnd;
    lp.stage_bytes = p.stage;
    lp.dfas = reinterpret_cast<const DevDfa*>(ws + p.ws.dfas);
    lp.tests = reinterpret_cast<const DevTest*>(ws + p.ws.tests);
    lp.groups = reinterpret_cast<const DevGroup*>(ws + p.ws.groups);
    bind(lp, ws, p.ws);
    lp.results = out;
}

int upload_desc(const Prepared& p, uint8_t* ws) {
    if (cudaMemcpy(ws + p.ws.dfas, p.dfas.data(), sizeof(DevDfa) * p.dfas.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ws + p.ws.tests, p.tests.data(), sizeof(DevTest) * p.tests.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(ws + p.ws.groups, p.groups.data(), sizeof(DevGroup) * p.groups.size(),
                   cudaMemcpyHostToDevice) != cudaSuccess)
        return DFA_ECUDA;
    return DFA_OK;
}

int upload_desc_async(const Prepared& p, uint8_t* ws, uint8_t* pinned, void* stream) {
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // pinned holds a host copy laid out like the workspace's descriptor area
    const uint64_t nd = sizeof(DevDfa) * p.dfas.size(), nt = sizeof(DevTest) * p.tests.size(),
                   ng = sizeof(DevGroup) * p.groups.size();
    std::memcpy(pinned + p.ws.dfas, p.dfas.data(), nd);
    std::memcpy(pinned + p.ws.tests, p.tests.data(), nt);
    std::memcpy(pinned + p.ws.groups, p.groups.data(), ng);
    const uint64_t span = p.ws.groups + ng;
    return cudaMemcpyAsync(ws, pinned, span, cudaMemcpyHostToDevice, st) == cudaSuccess ? DFA_OK
                                                                                          : DFA_ECUDA;
}

uint64_t desc_span(const Prepared& p) { return p.ws.groups + sizeof(DevGroup) * p.groups.size(); }

int launch_prepared(const Prepared& p, uint8_t* ws, dfa_result_t* out, void* stream) {
    LaunchPlan lp;
    fill_plan(p, lp, ws, out);
    return launch_plan(lp, p.kmax, p.smem, static_cast<cudaStream_t>(stream), nullptr);
}

int launch_single(const Single& s, void* stream, void* ev_begin, void* ev_end) {
    return launch_plan(s.lp, s.kmax, s.smem, static_cast<cudaStream_t>(stream), nullptr, ev_begin,
                       ev_end);
}

// Single-test plan with descriptors carried by value (no upload needed).
int plan_single(const dfa_t* d, uint64_t len, const dfa_match_opts_t* opts, Single* s) {
    if (!d) return DFA_EINVAL;
    if (!d->on_device) return DFA_EHOSTONLY;
    if (!opts_valid(opts) || !lookahead_ok(d, opts)) return DFA_EINVAL;
    const uint32_t lookahead = opts_lookahead(opts), slot = opts_slot(opts);
    const uint32_t m = (opts && opts->multiplicity) ? opts->multiplicity : 1u;
    DevDfa x = launch_desc(d, slot);
    const dfa_tuning_t& tu = d->tuning_for(slot);
    // Byte rows serve latency-bound launches: few chains in all, at most 128 per
    // SM (one warp per scheduler).  With more chains the launch is bound by the
    // shared-memory pipe, where a row read per step (16 bytes) costs more than a
    // table lookup, so the class-major table is used.
    bool nib = false;
    if (x.nib) {
        const uint32_t sms = device_sms();
        const uint64_t P0 = plan_chunks(d, len, std::max(sms, 1u) * 2, opts, false, 0);
        nib = sms && P0 * std::max(x.imax, 1u) <= (uint64_t)sms * 128u;
        x.nib = nib ? 1u : 0u;
    }
    const uint32_t tcap = x.placement == kSmem ? smem_table_bytes(x) : 0u;
    // byte-row launches take the kernel variant with the larger register
    // budget, for the rows loaded ahead of the chains, and by default one CTA
    // per SM (4 MiB in 1024 chunks, 16 states: 87 us against 98 us with two).
    // (Giving that variant to every two-CTA launch with K <= 4 left the
    // device-resident time unchanged and slowed the pipelined host path, whose
    // consecutive launches overlap only when the three-CTA variant leaves room
    // on each SM.)
    s->kmax = nib ? std::max(x.K, 8u) : x.K;
    const uint32_t want_ctas = tu.ctas_per_sm ? tu.ctas_per_sm : (nib ? 1u : 0u);
    uint32_t stage = 0;
    s->smem = match_smem_bytes(tcap, s->kmax, x.vcap, stage_esz(x.stage_fmt), &stage,
                               match_target_ctas(s->kmax, want_ctas));
    uint32_t grid = 0;
    int rc = match_grid(s->smem, s->kmax, &grid);
    if (rc != DFA_OK) return rc;
    // chunks are planned for one resident wave; more waves only cut the same
    // work into more, smaller CTA shares
    const uint32_t P = plan_chunks(d, len, grid, opts, false, 0);
    const uint32_t gw = d->tuning_for(slot).grid_waves;
    const uint32_t waves = gw ? std::min(gw, kMaxWaves) : 1u;
    LaunchPlan& lp = s->lp;
    std::memset(&lp, 0, sizeof lp);
    lp.ntests = 1;
    lp.ngroups = 1;
    lp.ptot = P;
    lp.nblk = (P + 1023) / 1024;
    lp.grid = grid * waves;
    lp.waves = waves;
    grid = lp.grid;
    lp.seg_stride = seg_stride_for(x.qe);
    lp.smem_table_cap = tcap;
    lp.vcap = x.vcap;
    lp.vmap_stride = vmap_stride_for(x.vcap);
    lp.stage_bytes = stage;
    lp.qe_max = x.qe;
    lp.dyn = lookahead >= 2 ? 1u : 0u;
    lp.no_nib = (d->dev.nib && !nib) ? 1u : 0u;
    lp.dfas = d->dev_desc_for(slot);
    lp.tests = nullptr;
    lp.groups = nullptr;
    lp.test1.str = nullptr;
    lp.test1.n = len;
    lp.test1.dfa = 0;
    lp.test1.P = P;
    lp.test1.m = m;
    lp.test1.qinv = recip64((uint64_t)m + P - 1);
    lp.test1.chunk_base = 0;
    lp.test1.group = 0;
    lp.test1.lookahead = lookahead;
    lp.test1.window = test_window(opts, len, P, m);
    lp.bnd = lp.test1.window ? 1u : 0u;
    lp.test1.out = 0;
    lp.group1.first_chunk = 0;
    lp.group1.end_chunk = P;
    lp.group1.dfa = 0;
    lp.group1.first_test = 0;
    lp.group1.set_stride = std::max(d->h.imax, 1u);
    lp.group1.set_base = 0;
    s->ws = ws_layout(1, 1, 1, P, lp.nblk, grid, lp.seg_stride, true, lp.dyn != 0,
                      (uint64_t)P * lp.group1.set_stride, lp.bnd != 0, x.vcap);
    return DFA_OK;
}

// The launches of one batch: tests whose DFA table is read from shared
// memory in a launch of several DFAs, then tests whose table is read through
// L2.  Each part has its own shared-memory layout, so the L2 part takes small
// stage buffers and leaves L1 to the hot table rows (one layout for both
// would give L1 little).  A batch of one DFA, or with tables of one kind,
// has one part.  ws_off receives each part's workspace offset and *ws_total
// their sum (256-byte aligned parts).
int prepare_parts(uint32_t count, const dfa_t* const* dfas, const uint8_t* const* strs,
                  const uint64_t* lens, const dfa_match_opts_t* opts, std::vector<Prepared>* parts,
                  std::vector<uint64_t>* ws_off, uint64_t* ws_total) {
    if (count == 0 || !dfas || !strs || !lens) return DFA_EINVAL;
    if (!opts_valid(opts)) return DFA_EINVAL;
    const uint32_t slot = opts_slot(opts);
    std::vector<uint32_t> ids[2];
    const dfa_t* first = dfas[0];
    bool several = false;
    for (uint32_t i = 0; i < count; ++i) {
        if (!dfas[i]) return DFA_EINVAL;
        several |= dfas[i] != first;
        const DevDfa x = launch_desc(dfas[i], slot);
        const bool smem = x.placement == kSmem && smem_table_bytes(x) <= kBatchSmemTable;
        ids[smem ? 0 : 1].push_back(i);
    }
    if (!several || ids[0].empty() || ids[1].empty()) {
        ids[0].clear();
        ids[1].clear();
        for (uint32_t i = 0; i < count; ++i) ids[0].push_back(i);
    }
    parts->clear();
    ws_off->clear();
    uint64_t total = 0;
    for (int k = 0; k < 2; ++k) {
        if (ids[k].empty()) continue;
        std::vector<const dfa_t*> pd;
        std::vector<const uint8_t*> ps;
        std::vector<uint64_t> pl;
        for (uint32_t i : ids[k]) {
            pd.push_back(dfas[i]);
            ps.push_back(strs[i]);
            pl.push_back(lens[i]);
        }
        Prepared p;
        int rc = prepare((uint32_t)ids[k].size(), pd.data(), ps.data(), pl.data(), opts, true, &p,
                         ids[k].data());
        if (rc != DFA_OK) return rc;
        ws_off->push_back(total);
        total += up(p.ws.total, 256);
        parts->push_back(std::move(p));
    }
    *ws_total = total;
    return DFA_OK;
}

}  // namespace dfam

using namespace dfam;

// ------------------------------------------------------------------ dfa_t

const DevDfa* dfa_s::dev_desc_for(uint32_t slot) const { return dev_desc + slot; }

// Uploads the launch descriptors of every tuning slot (their K follows the
// slot's tuning record).
static int upload_descs(dfa_t* d) {
    if (!d->dev_desc) return DFA_OK;  // a host-only DFA
    DevDfa descs[kTuningSlots];
    for (uint32_t r = 0; r < kTuningSlots; ++r) descs[r] = launch_desc(d, r);
    return cudaMemcpy(d->dev_desc, descs, sizeof descs, cudaMemcpyHostToDevice) == cudaSuccess
               ? DFA_OK
               : DFA_ECUDA;
}

static int create_common(uint32_t Q, uint32_t S, const int32_t* delta, uint32_t q0,
                         const uint32_t* finals, uint32_t nf, const uint8_t* b2s, bool device,
                         dfa_t** out) {
    if (!out) return DFA_EINVAL;
    *out = nullptr;
    dfa_t* d = new (std::nothrow) dfa_t();
    if (!d) return DFA_ENOMEM;
    int rc = compile_dfa(Q, S, delta, q0, finals, nf, b2s, &d->h);
    if (rc != DFA_OK) {
        delete d;
        return rc;
    }
    const HostDfa& h = d->h;
    // device-side descriptor (pointers filled below)
    DevDfa& x = d->dev;
    std::memset(&x, 0, sizeof x);
    x.qe = h.qe;
    x.qpad = h.qpad;
    x.C = h.C;
    x.sb = h.sb;
    x.placement = h.placement;
    x.table_bytes = (uint32_t)h.table.size();
    x.q0 = h.q0;
    x.imax = h.imax;
    x.K = h.K;
    x.stage_fmt = h.placement == kGlobal ? kOff32 : (h.C + 1 <= 255 ? kCls8 : kOff16);
    x.n_all = h.iset_off[h.C + 2] - h.iset_off[h.C + 1];
    x.nib = h.nib_rows.empty() ? 0u : 1u;
    // with byte rows, 16-bit stage entries are row offsets into them (class * 16)
    std::vector<uint16_t> nib16(256, kNone16);
    for (int b = 0; b < 256; ++b)
        if (h.byte_class[b] != kNone16) nib16[b] = (uint16_t)(h.byte_class[b] * 16u);
    // planning lookup: one load gives a lookahead byte's class and |I_class|
    uint32_t byte_plan[256];
    for (int b = 0; b < 256; ++b) {
        const uint32_t c = h.byte_class[b];
        byte_plan[b] = c == kNone16 ? kNone32 : (c << 16) | (h.iset_off[c + 1] - h.iset_off[c]);
    }
    if (device) {
        if (cudaGetDevice(&d->device) != cudaSuccess) {
            delete d;
            return DFA_ECUDA;
        }
        uint64_t o = 0;
        auto take = [&](uint64_t bytes) { uint64_t r = o; o = up(o + bytes, 256); return r; };
        const uint64_t o_desc = take(kTuningSlots * sizeof(DevDfa));
        const uint64_t o_table = take(h.table.size());
        const uint64_t o_b16 = take(512), o_b32 = take(1024), o_bc = take(512);
        const uint64_t o_ioff = take(4 * h.iset_off.size()), o_iset = take(2 * h.iset.size());
        const uint64_t o_pos = take(2 * h.pos.size()), o_acc = take(h.accept.size());
        const uint64_t o_exc = take(h.excluded.size()), o_bp = take(sizeof byte_plan);
        const uint64_t o_nib = take(h.nib_rows.size()), o_n16 = take(x.nib ? 512 : 0);
        uint8_t* blk = nullptr;
        if (cudaMalloc(&blk, o) != cudaSuccess) {
            cudaGetLastError();
            delete d;
            return DFA_ENOMEM;
        }
        d->dev_block = blk;
        d->dev_bytes = o;
        x.table = blk + o_table;
        x.byte_off16 = reinterpret_cast<const uint16_t*>(blk + o_b16);
        x.byte_off32 = reinterpret_cast<const uint32_t*>(blk + o_b32);
        x.byte_class = reinterpret_cast<const uint16_t*>(blk + o_bc);
        x.iset_off = reinterpret_cast<const uint32_t*>(blk + o_ioff);
        x.iset = reinterpret_cast<const uint16_t*>(blk + o_iset);
        x.pos = reinterpret_cast<const uint16_t*>(blk + o_pos);
        x.accept = blk + o_acc;
        x.excluded = blk + o_exc;
        x.byte_plan = reinterpret_cast<const uint32_t*>(blk + o_bp);
        x.nib_rows = x.nib ? blk + o_nib : nullptr;
        x.nib_off16 = x.nib ? reinterpret_cast<const uint16_t*>(blk + o_n16) : nullptr;
        d->dev_desc = reinterpret_cast<DevDfa*>(blk + o_desc);
        bool ok = upload_descs(d) == DFA_OK &&
                  cudaMemcpy(blk + o_table, h.table.data(), h.table.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemcpy(blk + o_b16, h.byte_off16.data(), 512, cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemcpy(blk + o_b32, h.byte_off32.data(), 1024, cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemcpy(blk + o_bc, h.byte_class.data(), 512, cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemcpy(blk + o_ioff, h.iset_off.data(), 4 * h.iset_off.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemcpy(blk + o_iset, h.iset.data(), 2 * h.iset.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemcpy(blk + o_pos, h.pos.data(), 2 * h.pos.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemcpy(blk + o_acc, h.accept.data(), h.accept.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemcpy(blk + o_exc, h.excluded.data(), h.excluded.size(), cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaMemcpy(blk + o_bp, byte_plan, sizeof byte_plan, cudaMemcpyHostToDevice) == cudaSuccess &&
                  (!x.nib || (cudaMemcpy(blk + o_nib, h.nib_rows.data(), h.nib_rows.size(),
                                         cudaMemcpyHostToDevice) == cudaSuccess &&
                              cudaMemcpy(blk + o_n16, nib16.data(), 512, cudaMemcpyHostToDevice) ==
                                  cudaSuccess));
        if (!ok) {
            cudaFree(blk);
            delete d;
            return DFA_ECUDA;
        }
        d->on_device = true;
    }
    *out = d;
    return DFA_OK;
}

extern "C" {

int dfa_create(uint32_t Q, uint32_t S, const int32_t* delta, uint32_t q0, const uint32_t* finals,
               uint32_t nf, const uint8_t* b2s, dfa_t** out) {
    return dfam::no_throw([&]() -> int {
        return create_common(Q, S, delta, q0, finals, nf, b2s, true, out);
    });
}

int dfa_create_host(uint32_t Q, uint32_t S, const int32_t* delta, uint32_t q0,
                    const uint32_t* finals, uint32_t nf, const uint8_t* b2s, dfa_t** out) {
    return dfam::no_throw([&]() -> int {
        return create_common(Q, S, delta, q0, finals, nf, b2s, false, out);
    });
}

void dfa_destroy(dfa_t* d) {
    if (!d) return;
    if (d->dev_block) cudaFree(d->dev_block);
    delete d;
}

int dfa_info(const dfa_t* d, dfa_info_t* o) {
    if (!d || !o) return DFA_EINVAL;
    const HostDfa& h = d->h;
    std::memset(o, 0, sizeof *o);
    o->num_states = h.Q;
    o->num_symbols = h.S;
    o->num_states_ext = h.qe;
    o->num_classes = h.C;
    o->i_max = h.imax;
    o->num_excluded = h.num_excluded;
    o->state_bytes = h.sb;
    o->placement = h.placement;
    o->states_per_thread = h.K;
    o->q0 = h.q0;
    o->table_bytes = h.table.size();
    o->device_bytes = d->dev_bytes;
    o->gamma = h.gamma;
    o->mean_iset = h.mean_iset;
    o->byte_rows = h.nib_rows.empty() ? 0u : 1u;
    return DFA_OK;
}

// Tuning record of a slot (lookahead depth, placed or not): the base record
// for depth 1 unplaced (and for slots without their own record when read).
static int get_tuning_r(const dfa_t* d, uint32_t r, dfa_tuning_t* out) {
    if (!d || !out || r >= kTuningSlots) return DFA_EINVAL;
    *out = d->tuning_for(r);
    if (!out->states_per_thread) out->states_per_thread = d->h.K;
    return DFA_OK;
}

static int set_tuning_r(dfa_t* d, uint32_t r, const dfa_tuning_t* t) {
    if (!d || !t || r >= kTuningSlots) return DFA_EINVAL;
    const uint32_t K = t->states_per_thread ? t->states_per_thread : d->h.K;
    if (K != 1 && K != 2 && K != 4 && K != 8 && K != 16) return DFA_EINVAL;
    if (!k_allowed(d, K)) return DFA_EINVAL;
    if (t->grid_waves > kMaxWaves) return DFA_EINVAL;
    dfa_tuning_t v = *t;
    v.states_per_thread = K;
    if (r == 1) {
        d->tuning = v;
        d->h.K = K;
        d->dev.K = K;
    } else {
        d->tuning_r[r] = v;
        d->has_tuning_r[r] = true;
    }
    return upload_descs(d);
}

// Times every candidate tuning on a device sample with the lookahead and
// placement window of `base` (NULL: lookahead 1, no placement) and keeps the
// fastest in that slot's record.
static int autotune_r(dfa_t* d, const dfa_match_opts_t* base, const uint8_t* dev_sample,
                      uint64_t len, void* stream, dfa_tuning_t* chosen, double* best_ms) {
    if (!d || (len && !dev_sample) || !opts_valid(base) || !lookahead_ok(d, base)) return DFA_EINVAL;
    if (!d->on_device) return DFA_EHOSTONLY;
    const uint32_t r = opts_slot(base);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    dfa_tuning_t saved;
    get_tuning_r(d, r, &saved);
    dfa_match_opts_t o{};
    o.lookahead = opts_lookahead(base);
    o.boundary_window = opts_window(base);
    std::vector<dfa_tuning_t> cands;
    for (uint32_t K : {1u, 2u, 4u, 8u, 16u}) {
        if (!k_allowed(d, K)) continue;
        for (uint32_t tpc : {1u, 2u, 4u, 8u, 16u}) {
            for (uint32_t ctas : {2u, 3u}) {
                if (ctas == 3 && K > 4) continue;
                dfa_tuning_t t = saved;
                t.states_per_thread = K;
                t.tiles_per_cta = tpc;
                t.ctas_per_sm = ctas;
                t.grid_waves = 1;
                cands.push_back(t);
                // more, smaller CTA shares over the same chunks (each CTA still
                // gets at least one full tile)
                for (uint32_t w : {2u, 4u}) {
                    if (w > tpc || tpc > 4) continue;
                    t.grid_waves = w;
                    cands.push_back(t);
                }
            }
        }
    }
    // Where the chunk count is bound by the shortest chunk (sets so small that
    // filling the CTAs would need ever shorter chunks), longer chunks are tried
    // too: per-chunk work (metadata, composition) then stops dominating.
    const size_t nbase = cands.size();
    for (size_t ci = 0; ci < nbase; ++ci) {
        const uint32_t min_chunk = cands[ci].min_chunk_bytes ? cands[ci].min_chunk_bytes : kMinChunk;
        Single s;
        if (set_tuning_r(d, r, &cands[ci]) != DFA_OK || plan_single(d, len, &o, &s) != DFA_OK)
            continue;
        if (s.lp.ptot < std::max<uint64_t>(len / min_chunk, 1)) continue;
        for (uint32_t mc : {2048u, 8192u}) {
            if (mc <= min_chunk) continue;
            dfa_tuning_t t = cands[ci];
            t.min_chunk_bytes = mc;
            cands.push_back(t);
        }
    }
    // workspace for the largest plan
    uint64_t ws_need = 0;
    for (const dfa_tuning_t& t : cands) {
        if (set_tuning_r(d, r, &t) != DFA_OK) continue;
        Single s;
        if (plan_single(d, len, &o, &s) == DFA_OK) ws_need = std::max(ws_need, s.ws.total);
    }
    uint8_t* ws = nullptr;
    if (cudaMalloc(&ws, ws_need + 256) != cudaSuccess) {
        cudaGetLastError();
        set_tuning_r(d, r, &saved);
        return DFA_ENOMEM;
    }
    dfa_result_t* dres = reinterpret_cast<dfa_result_t*>(ws + ws_need);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    // median time per candidate; among those within 1% of the fastest the one
    // with the most CTAs per SM wins (more, smaller CTAs also let consecutive
    // or concurrent launches share the SMs, as in the host pipeline)
    std::vector<double> med_ms(cands.size(), 1e30);
    std::vector<uint32_t> cand_P(cands.size(), 1);
    int rc = DFA_OK;
    for (size_t ci = 0; ci < cands.size(); ++ci) {
        const dfa_tuning_t& t = cands[ci];
        if (set_tuning_r(d, r, &t) != DFA_OK) continue;
        Single s;
        if (plan_single(d, len, &o, &s) != DFA_OK) continue;
        s.lp.test1.str = dev_sample;
        bind(s.lp, ws, s.ws);
        s.lp.results = dres;
        std::vector<float> ms;
        for (int i = 0; i < 4 && rc == DFA_OK; ++i) {
            cudaEventRecord(e0, st);
            rc = launch_plan(s.lp, s.kmax, s.smem, st, nullptr);
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess) rc = DFA_ECUDA;
            float x = 0;
            cudaEventElapsedTime(&x, e0, e1);
            if (i > 0) ms.push_back(x);  // the first launch is a warm-up
        }
        if (rc != DFA_OK) break;
        std::sort(ms.begin(), ms.end());
        med_ms[ci] = ms[ms.size() / 2];
        cand_P[ci] = s.lp.ptot;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(ws);
    double best = 1e30;
    for (double m : med_ms) best = std::min(best, m);
    dfa_tuning_t best_t = saved;
    uint32_t best_P = 1;
    int pick = -1;
    for (size_t ci = 0; ci < cands.size(); ++ci) {
        if (med_ms[ci] > best * 1.01) continue;
        if (pick < 0 || cands[ci].ctas_per_sm > cands[pick].ctas_per_sm ||
            (cands[ci].ctas_per_sm == cands[pick].ctas_per_sm && med_ms[ci] < med_ms[pick]))
            pick = (int)ci;
    }
    if (pick >= 0) {
        best_t = cands[pick];
        best_P = cand_P[pick];
        best = med_ms[pick];
    }
    uint64_t clen = best_P ? len / best_P : kBatchChunk;
    // batched launches: chunks of 8-32 KiB measure best on the 64-DFA mix
    best_t.batch_chunk_bytes = (uint32_t)std::min<uint64_t>(std::max<uint64_t>(clen, 8192), 65536);
    int rc2 = set_tuning_r(d, r, &best_t);
    if (rc == DFA_OK) rc = rc2;
    if (chosen) get_tuning_r(d, r, chosen);
    if (best_ms) *best_ms = best;
    if (rc == DFA_OK && best > 0 && best < 1e29) d->tuned_gbs[r] = (double)len / (best * 1e6);
    return rc;
}

int dfa_get_tuning(const dfa_t* d, dfa_tuning_t* out) { return get_tuning_r(d, 1, out); }

int dfa_set_tuning(dfa_t* d, const dfa_tuning_t* t) { return dfam::no_throw([&]() -> int { return set_tuning_r(d, 1, t); }); }

int dfa_autotune(dfa_t* d, const uint8_t* dev_sample, uint64_t len, void* stream,
                 dfa_tuning_t* chosen, double* best_ms) {
    return dfam::no_throw([&]() -> int {
        return autotune_r(d, nullptr, dev_sample, len, stream, chosen, best_ms);
    });
}

int dfa_get_tuning_opts(const dfa_t* d, const dfa_match_opts_t* opts, dfa_tuning_t* out) {
    if (!opts_valid(opts)) return DFA_EINVAL;
    return get_tuning_r(d, opts_slot(opts), out);
}

int dfa_set_tuning_opts(dfa_t* d, const dfa_match_opts_t* opts, const dfa_tuning_t* t) {
    return dfam::no_throw([&]() -> int {
        if (!opts_valid(opts)) return DFA_EINVAL;
        return set_tuning_r(d, opts_slot(opts), t);
    });
}

int dfa_autotune_opts(dfa_t* d, const uint8_t* dev_sample, uint64_t len,
                      const dfa_match_opts_t* opts, void* stream, dfa_tuning_t* chosen,
                      double* best_ms) {
    return dfam::no_throw([&]() -> int {
        return autotune_r(d, opts, dev_sample, len, stream, chosen, best_ms);
    });
}

int dfa_class_of_bytes(const dfa_t* d, uint16_t* out) {
    if (!d || !out) return DFA_EINVAL;
    std::memcpy(out, d->h.byte_class.data(), 512);
    return DFA_OK;
}

int dfa_iset(const dfa_t* d, uint32_t c, uint32_t* states, uint32_t cap, uint32_t* count) {
    if (!d || !count || c > d->h.C + 1) return DFA_EINVAL;
    const HostDfa& h = d->h;
    const uint32_t a = h.iset_off[c], b = h.iset_off[c + 1];
    *count = b - a;
    for (uint32_t i = 0; i < b - a && i < cap; ++i) states[i] = h.iset[a + i];
    return DFA_OK;
}

int dfa_partition(uint64_t n, uint32_t P, uint32_t m, uint64_t* starts) {
    if (P == 0 || m == 0 || !starts) return DFA_EINVAL;
    for (uint32_t k = 0; k <= P; ++k) starts[k] = chunk_start(n, P, m, k);
    return DFA_OK;
}

__global__ void k_identity_maps(uint16_t* maps, uint64_t P, uint32_t qe) {
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < P * qe;
         i += (uint64_t)gridDim.x * blockDim.x)
        maps[i] = (uint16_t)(i % qe);
}

int dfa_debug_chunk_maps(const dfa_t* d, const uint8_t* dev_str, uint64_t len,
                         const dfa_match_opts_t* opts, uint16_t* maps, uint32_t cap, uint32_t* P,
                         uint32_t* final_state) {
    return dfam::no_throw([&]() -> int {
        if (!P || (len && !dev_str)) return DFA_EINVAL;
        Single s;
        int rc = plan_single(d, len, opts, &s);
        if (rc != DFA_OK) return rc;
        *P = s.lp.ptot;
        if (!maps || cap == 0) return DFA_OK;
        const uint32_t qe = s.lp.qe_max;
        const uint64_t map_bytes = up(2ull * s.lp.ptot * qe, 256);  // keeps the result 256-byte aligned
        uint8_t* ws = nullptr;
        if (cudaMalloc(&ws, s.ws.total + map_bytes + 256) != cudaSuccess) {
            cudaGetLastError();
            return DFA_ENOMEM;
        }
        uint16_t* dmaps = reinterpret_cast<uint16_t*>(ws + s.ws.total);
        dfa_result_t* dres = reinterpret_cast<dfa_result_t*>(ws + s.ws.total + map_bytes);
        k_identity_maps<<<1024, 256>>>(dmaps, s.lp.ptot, qe);
        s.lp.test1.str = dev_str;
        bind(s.lp, ws, s.ws);
        s.lp.results = dres;
        s.lp.dbg_maps = dmaps;
        rc = launch_plan(s.lp, s.kmax, s.smem, 0, nullptr);
        dfa_result_t r{};
        const uint32_t n = std::min(cap, s.lp.ptot);
        if (rc == DFA_OK && cudaMemcpy(maps, dmaps, 2ull * n * qe, cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = DFA_ECUDA;
        if (rc == DFA_OK && cudaMemcpy(&r, dres, sizeof r, cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = DFA_ECUDA;
        cudaFree(ws);
        if (rc == DFA_OK && final_state) *final_state = r.final_state;
        if (rc == DFA_OK && r.status != DFA_OK) rc = r.status;
        return rc;
    });
}

int dfa_match_num_kernels(const dfa_t* d, uint64_t len, const dfa_match_opts_t* opts, uint32_t* n) {
    return dfam::no_throw([&]() -> int {
        if (!n) return DFA_EINVAL;
        Single s;
        int rc = plan_single(d, len, opts, &s);
        if (rc != DFA_OK) return rc;
        *n = launch_kernel_count(s.lp.ptot, s.lp.grid, s.lp.dyn != 0, s.lp.bnd != 0);
        return DFA_OK;
    });
}

int dfa_plan_sets(const dfa_t* d, const uint8_t* dev_str, uint64_t len,
                  const dfa_match_opts_t* opts, uint32_t* sizes, uint32_t cap, uint32_t* P) {
    return dfam::no_throw([&]() -> int {
        if (!P || (len && !dev_str)) return DFA_EINVAL;
        Single s;
        int rc = plan_single(d, len, opts, &s);
        if (rc != DFA_OK) return rc;
        *P = s.lp.ptot;
        uint8_t* ws = nullptr;
        if (cudaMalloc(&ws, s.ws.total) != cudaSuccess) { cudaGetLastError(); return DFA_ENOMEM; }
        s.lp.test1.str = dev_str;
        bind(s.lp, ws, s.ws);
        s.lp.results = nullptr;
        rc = launch_plan(s.lp, s.kmax, s.smem, 0, nullptr, nullptr, nullptr, true);
        const uint32_t n = std::min(cap, s.lp.ptot);
        std::vector<uint16_t> cls(n);
        std::vector<uint32_t> dyn(n);
        if (rc == DFA_OK && n) {
            if (cudaMemcpy(cls.data(), s.lp.chunk_cls, 2ull * n, cudaMemcpyDeviceToHost) != cudaSuccess)
                rc = DFA_ECUDA;
            if (rc == DFA_OK && s.lp.dyn &&
                cudaMemcpy(dyn.data(), s.lp.set_size, 4ull * n, cudaMemcpyDeviceToHost) != cudaSuccess)
                rc = DFA_ECUDA;
        }
        if (cudaDeviceSynchronize() != cudaSuccess) rc = DFA_ECUDA;
        cudaFree(ws);
        if (rc != DFA_OK) return rc;
        const HostDfa& h = d->h;
        for (uint32_t k = 0; k < n; ++k)
            sizes[k] = cls[k] == dyn_set(h.C) ? dyn[k] : h.iset_off[cls[k] + 1] - h.iset_off[cls[k]];
        return DFA_OK;
    });
}

int dfa_plan_starts(const dfa_t* d, const uint8_t* dev_str, uint64_t len,
                    const dfa_match_opts_t* opts, uint64_t* starts, uint32_t cap, uint32_t* P) {
    return dfam::no_throw([&]() -> int {
        if (!P || (len && !dev_str)) return DFA_EINVAL;
        Single s;
        int rc = plan_single(d, len, opts, &s);
        if (rc != DFA_OK) return rc;
        *P = s.lp.ptot;
        if (!starts || cap == 0) return DFA_OK;
        const uint32_t P1 = s.lp.ptot + 1, n = std::min(cap, P1);
        std::vector<uint64_t> placed;
        if (s.lp.bnd) {
            uint8_t* ws = nullptr;
            if (cudaMalloc(&ws, s.ws.total) != cudaSuccess) { cudaGetLastError(); return DFA_ENOMEM; }
            s.lp.test1.str = dev_str;
            bind(s.lp, ws, s.ws);
            s.lp.results = nullptr;
            rc = launch_plan(s.lp, s.kmax, s.smem, 0, nullptr, nullptr, nullptr, true);
            placed.resize(s.lp.ptot);
            if (rc == DFA_OK &&
                cudaMemcpy(placed.data(), s.lp.starts, 8ull * s.lp.ptot, cudaMemcpyDeviceToHost) != cudaSuccess)
                rc = DFA_ECUDA;
            if (cudaDeviceSynchronize() != cudaSuccess) rc = DFA_ECUDA;
            cudaFree(ws);
            if (rc != DFA_OK) return rc;
        }
        const DevTest& t = s.lp.test1;
        for (uint32_t k = 0; k < n; ++k)
            starts[k] = (k == 0) ? 0 : (k >= t.P ? len : (t.window ? placed[k] : chunk_start(len, t.P, t.m, k)));
        return DFA_OK;
    });
}

int dfa_match_workspace_size(const dfa_t* d, uint64_t len, const dfa_match_opts_t* opts,
                             uint64_t* bytes) {
    return dfam::no_throw([&]() -> int {
        if (!bytes) return DFA_EINVAL;
        Single s;
        int rc = plan_single(d, len, opts, &s);
        if (rc != DFA_OK) return rc;
        *bytes = s.ws.total;
        return DFA_OK;
    });
}

int dfa_match_async(const dfa_t* d, const uint8_t* dev_str, uint64_t len,
                    const dfa_match_opts_t* opts, dfa_result_t* dev_out, void* ws,
                    uint64_t ws_bytes, void* stream) {
    return dfam::no_throw([&]() -> int {
        if (!dev_out || (len && !dev_str) || !ws) return DFA_EINVAL;
        if ((reinterpret_cast<uintptr_t>(dev_out) & 3u) || (reinterpret_cast<uintptr_t>(ws) & 255u))
            return DFA_EINVAL;  // results are 4-byte aligned, the workspace 256-byte aligned
        Single s;
        int rc = plan_single(d, len, opts, &s);
        if (rc != DFA_OK) return rc;
        if (ws_bytes < s.ws.total) return DFA_ENOSPACE;
        s.lp.test1.str = dev_str;
        bind(s.lp, static_cast<uint8_t*>(ws), s.ws);
        s.lp.results = dev_out;
        return launch_plan(s.lp, s.kmax, s.smem, static_cast<cudaStream_t>(stream), nullptr,
                           opts ? opts->match_begin_event : nullptr,
                           opts ? opts->match_end_event : nullptr);
    });
}

// Per-device buffers of the synchronous path (grown on demand, never shrunk).
struct SyncBuffers {
    std::mutex mu;
    uint8_t* str = nullptr;
    uint64_t str_cap = 0;
    uint8_t* ws = nullptr;
    uint64_t ws_cap = 0;
    cudaStream_t ks[2] = {nullptr, nullptr};  // compute streams of the host pipeline
    cudaStream_t cs = nullptr;                 // copy stream of the host pipeline
    cudaEvent_t join = nullptr;                // the second compute stream's last launch
    std::vector<cudaEvent_t> ev;               // one "segment copied" event per segment
};
static SyncBuffers g_sync[64];

// Segment lengths of the pipelined host path.  The first segment is short,
// so little copy time is exposed before the first launch.  Later ones double
// (fewer launches while the matching is slower than the copies) up to an
// eighth of the string: the last segment's match starts only once its copy
// has landed, so its length bounds the match time left exposed at the end.
// A remainder shorter than half the next length joins the last segment.
// Returns false when the input is too short to pipeline.
static bool host_segments(uint64_t len, uint32_t first_bytes, uint64_t cap_div,
                          std::vector<uint64_t>* seg) {
    constexpr uint64_t kMin = 16ull << 20, kMax = 256ull << 20;
    if (first_bytes == 0xFFFFFFFFu) return false;
    uint64_t first = first_bytes ? first_bytes : std::min(kMax, std::max(kMin, len / 32));
    if (first < 4096 || len < 2 * first) return false;
    const uint64_t cap = std::max(first, len / cap_div);
    seg->clear();
    uint64_t pos = 0, next = first;
    while (pos < len) {
        uint64_t take = std::min(next, len - pos);
        if (len - pos - take < next / 2) take = len - pos;
        seg->push_back(take);
        pos += take;
        next = std::min(next * 2, cap);
    }
    return seg->size() > 1;
}

// The largest host-pipeline segment as a fraction of the string.  When the
// matching is slower than the copies (the DFA's autotuned device rate below
// kCopyBoundGbs), the copies stay ahead of the matching, so larger segments
// (a quarter of the string) only save launches: measured on the regex-shaped
// DFA, 87.7 GB/s end to end against 84.0 with eighths.  When the matching is
// faster, the last segment's matching runs after every copy has landed, so
// segments stop at an eighth.
constexpr double kCopyBoundGbs = 150.0;
static uint64_t segment_cap_div(const dfa_t* d, const dfa_match_opts_t* o) {
    const double r = d->tuned_gbs[opts_slot(o)];
    return (r > 0 && r < kCopyBoundGbs) ? 4u : 8u;
}

static int pipeline_resources(SyncBuffers& B, size_t nseg) {
    for (cudaStream_t* s : {&B.ks[0], &B.ks[1], &B.cs})
        if (!*s && cudaStreamCreateWithFlags(s, cudaStreamNonBlocking) != cudaSuccess)
            return DFA_ECUDA;
    if (!B.join && cudaEventCreateWithFlags(&B.join, cudaEventDisableTiming) != cudaSuccess)
        return DFA_ECUDA;
    while (B.ev.size() < nseg) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return DFA_ECUDA;
        B.ev.push_back(e);
    }
    return DFA_OK;
}

static int grow_dev(uint8_t** p, uint64_t* cap, uint64_t need) {
    if (*cap >= need) return DFA_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    if (cudaMalloc(p, need) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return DFA_ENOMEM;
    }
    *cap = need;
    return DFA_OK;
}

int dfa_plan_chunks(const dfa_t* d, uint64_t len, const dfa_match_opts_t* opts, uint32_t* P) {
    return dfam::no_throw([&]() -> int {
        if (!P) return DFA_EINVAL;
        Single s;
        int rc = plan_single(d, len, opts, &s);
        if (rc != DFA_OK) return rc;
        *P = s.lp.ptot;
        return DFA_OK;
    });
}

// Host input in segments: segment i is copied on B.cs and matched once its
// copy has landed, on compute stream i % 2 with its own workspace, so the
// tail of one launch overlaps the start of the next.  Segment 0 is a plain
// test; later segments are map tests (kTestCont | kTestMap) that need nothing
// from the launches before them, and k_compose_segments applies their maps
// to segment 0's final state (Eq. 8) once both streams are done.
static int match_pipelined(const dfa_t* d, const uint8_t* str, const std::vector<uint64_t>& seg,
                           const dfa_match_opts_t* opts, SyncBuffers& B, dfa_result_t* out) {
    const size_t ns = seg.size();
    std::vector<Single> plan(ns);
    uint64_t len = 0, ws_need = 0;
    for (uint64_t x : seg) len += x;
    // every segment keeps the chunk length the whole string would get (the
    // planner sizes chunk counts for a full GPU, which would cut the short
    // early segments into needlessly short chunks)
    Single whole;
    int rc = plan_single(d, len, opts, &whole);
    if (rc != DFA_OK) return rc;
    dfa_match_opts_t so = opts ? *opts : dfa_match_opts_t{};
    if (!opts) so.lookahead = 1;
    for (size_t i = 0; i < ns; ++i) {
        const uint64_t p = (uint64_t)whole.lp.ptot * seg[i] / len;
        so.num_chunks = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(p, 1u << 30));
        if ((rc = plan_single(d, seg[i], &so, &plan[i])) != DFA_OK) return rc;
        ws_need = std::max(ws_need, plan[i].ws.total);
    }
    if ((rc = pipeline_resources(B, ns)) != DFA_OK) return rc;
    const uint32_t stride = (d->h.qe + 1) & ~1u;
    const uint64_t res_off = 2 * ws_need, map_off = up(res_off + sizeof(dfa_result_t) * (ns + 1), 256);
    if ((rc = grow_dev(&B.str, &B.str_cap, len)) != DFA_OK) return rc;
    if ((rc = grow_dev(&B.ws, &B.ws_cap, map_off + 2ull * stride * ns + 256)) != DFA_OK) return rc;
    dfa_result_t* dres = reinterpret_cast<dfa_result_t*>(B.ws + res_off);  // [ns] + the answer
    uint16_t* maps = reinterpret_cast<uint16_t*>(B.ws + map_off);
    uint64_t pos = 0;
    for (size_t i = 0; i < ns; ++i) {
        cudaStream_t ks = B.ks[i & 1];
        if (cudaMemcpyAsync(B.str + pos, str + pos, seg[i], cudaMemcpyHostToDevice, B.cs) !=
                cudaSuccess ||
            cudaEventRecord(B.ev[i], B.cs) != cudaSuccess ||
            cudaStreamWaitEvent(ks, B.ev[i], 0) != cudaSuccess)
            return DFA_ECUDA;
        Single& s = plan[i];
        s.lp.test1.str = B.str + pos;
        s.lp.test1.flags = i ? (kTestCont | kTestMap) : 0u;
        bind(s.lp, B.ws + (i & 1) * ws_need, s.ws);
        s.lp.results = dres + i;
        s.lp.maps = maps + i * stride;
        s.lp.map_stride = stride;
        rc = launch_plan(s.lp, s.kmax, s.smem, ks, nullptr,
                         (opts && i == 0) ? opts->match_begin_event : nullptr, nullptr);
        if (rc != DFA_OK) return rc;
        pos += seg[i];
    }
    if (cudaEventRecord(B.join, B.ks[1]) != cudaSuccess ||
        cudaStreamWaitEvent(B.ks[0], B.join, 0) != cudaSuccess)
        return DFA_ECUDA;
    if ((rc = launch_compose_segments(dres, maps, stride, (uint32_t)ns, d->dev.accept, dres + ns,
                                      B.ks[0])) != DFA_OK)
        return rc;
    if (opts && opts->match_end_event &&
        cudaEventRecord(static_cast<cudaEvent_t>(opts->match_end_event), B.ks[0]) != cudaSuccess)
        return DFA_ECUDA;
    if (cudaMemcpyAsync(out, dres + ns, sizeof *out, cudaMemcpyDeviceToHost, B.ks[0]) !=
            cudaSuccess ||
        cudaStreamSynchronize(B.ks[0]) != cudaSuccess)
        return DFA_ECUDA;
    return out->status != DFA_OK ? out->status : DFA_OK;
}

int dfa_match(const dfa_t* d, const uint8_t* str, uint64_t len, const dfa_match_opts_t* opts,
              dfa_result_t* out) {
    return dfam::no_throw([&]() -> int {
        if (!d || !out || (len && !str)) return DFA_EINVAL;
        if (!d->on_device) return DFA_EHOSTONLY;
        bool on_dev = false;
        if (len) {
            cudaPointerAttributes at;
            if (cudaPointerGetAttributes(&at, str) == cudaSuccess)
                on_dev = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
            cudaGetLastError();
        }
        Single s;
        int rc = plan_single(d, len, opts, &s);
        if (rc != DFA_OK) return rc;
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return DFA_ECUDA;
        SyncBuffers& B = g_sync[dev];
        std::lock_guard<std::mutex> lock(B.mu);
        std::vector<uint64_t> seg;
        if (len && !on_dev && !(opts && (opts->num_chunks || opts->multiplicity)) &&
            d->h.qe <= kMaxSmallQe &&
            host_segments(len, d->tuning.host_segment_bytes, segment_cap_div(d, opts), &seg))
            return match_pipelined(d, str, seg, opts, B, out);
        const uint8_t* use = str;
        if (len && !on_dev) {
            if ((rc = grow_dev(&B.str, &B.str_cap, len)) != DFA_OK) return rc;
            if (cudaMemcpyAsync(B.str, str, len, cudaMemcpyHostToDevice, 0) != cudaSuccess)
                return DFA_ECUDA;
            use = B.str;
        }
        if ((rc = grow_dev(&B.ws, &B.ws_cap, s.ws.total + 256)) != DFA_OK) return rc;
        dfa_result_t* dres = reinterpret_cast<dfa_result_t*>(B.ws + s.ws.total);
        s.lp.test1.str = use;
        bind(s.lp, B.ws, s.ws);
        s.lp.results = dres;
        rc = launch_plan(s.lp, s.kmax, s.smem, 0, nullptr,
                         opts ? opts->match_begin_event : nullptr, opts ? opts->match_end_event : nullptr);
        if (rc == DFA_OK && cudaMemcpy(out, dres, sizeof *out, cudaMemcpyDeviceToHost) != cudaSuccess)
            rc = DFA_ECUDA;
        if (rc == DFA_OK && out->status != DFA_OK) rc = out->status;
        return rc;
    });
}

}  // extern "C"

// ------------------------------------------------------------------ batches

// A batch runs as one launch per part (prepare_parts).
struct dfa_batch_s {
    std::vector<Prepared> parts;
    std::vector<uint64_t> ws_off;  // each part's offset in ws
    uint8_t* ws = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    dfa_result_t* graph_out = nullptr;
    void* ev_begin = nullptr;
    void* ev_end = nullptr;
};

// Every part of the batch in order on `st` (the events bracket all match kernels).
static int launch_parts(const dfa_batch_t* b, dfa_result_t* dev_out, cudaStream_t st, void* ev_begin,
                        void* ev_end) {
    const size_t n = b->parts.size();
    for (size_t i = 0; i < n; ++i) {
        LaunchPlan lp;
        fill_plan(b->parts[i], lp, b->ws + b->ws_off[i], dev_out);
        int rc = launch_plan(lp, b->parts[i].kmax, b->parts[i].smem, st, nullptr,
                             i == 0 ? ev_begin : nullptr, i + 1 == n ? ev_end : nullptr);
        if (rc != DFA_OK) return rc;
    }
    return DFA_OK;
}

extern "C" {

int dfa_batch_prepare(uint32_t count, const dfa_t* const* dfas, const uint8_t* const* strs,
                      const uint64_t* lens, const dfa_match_opts_t* opts, dfa_batch_t** out) {
    return dfam::no_throw([&]() -> int {
        if (!out) return DFA_EINVAL;
        *out = nullptr;
        dfa_batch_t* b = new (std::nothrow) dfa_batch_t();
        if (!b) return DFA_ENOMEM;
        uint64_t total = 0;
        int rc = prepare_parts(count, dfas, strs, lens, opts, &b->parts, &b->ws_off, &total);
        if (rc != DFA_OK) {
            delete b;
            return rc;
        }
        if (cudaMalloc(&b->ws, total) != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return DFA_ENOMEM;
        }
        for (size_t i = 0; i < b->parts.size(); ++i) {
            rc = upload_desc(b->parts[i], b->ws + b->ws_off[i]);
            if (rc != DFA_OK) {
                cudaFree(b->ws);
                delete b;
                return rc;
            }
        }
        *out = b;
        return DFA_OK;
    });
}

int dfa_batch_launch(dfa_batch_t* b, dfa_result_t* dev_out, void* stream) {
    return dfam::no_throw([&]() -> int {
        if (!b || !dev_out || (reinterpret_cast<uintptr_t>(dev_out) & 3u)) return DFA_EINVAL;
        return launch_parts(b, dev_out, static_cast<cudaStream_t>(stream), b->ev_begin, b->ev_end);
    });
}

int dfa_batch_set_events(dfa_batch_t* b, void* ev_begin, void* ev_end) {
    if (!b) return DFA_EINVAL;
    b->ev_begin = ev_begin;
    b->ev_end = ev_end;
    return DFA_OK;
}

int dfa_batch_graph_launch(dfa_batch_t* b, dfa_result_t* dev_out, void* stream) {
    return dfam::no_throw([&]() -> int {
        if (!b || !dev_out || (reinterpret_cast<uintptr_t>(dev_out) & 3u)) return DFA_EINVAL;
        cudaStream_t st = static_cast<cudaStream_t>(stream);
        if (!b->exec || b->graph_out != dev_out) {
            if (b->exec) { cudaGraphExecDestroy(b->exec); b->exec = nullptr; }
            if (b->graph) { cudaGraphDestroy(b->graph); b->graph = nullptr; }
            cudaStream_t cap = st;
            bool own = false;
            if (!cap) {  // the legacy default stream cannot be captured
                if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return DFA_ECUDA;
                own = true;
            }
            if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
                if (own) cudaStreamDestroy(cap);
                return DFA_ECUDA;
            }
            int rc = launch_parts(b, dev_out, cap, nullptr, nullptr);
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(cap, &g);
            if (own) cudaStreamDestroy(cap);
            if (rc != DFA_OK || e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                cudaGetLastError();
                return DFA_ECUDA;
            }
            if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
                cudaGraphDestroy(g);
                return DFA_ECUDA;
            }
            b->graph = g;
            b->graph_out = dev_out;
        }
        return cudaGraphLaunch(b->exec, st) == cudaSuccess ? DFA_OK : DFA_ECUDA;
    });
}

int dfa_batch_num_kernels(const dfa_batch_t* b, uint32_t* n) {
    if (!b || !n) return DFA_EINVAL;
    uint32_t k = 0;
    for (const Prepared& p : b->parts) k += launch_kernel_count(p.ptot, p.grid, p.dyn != 0, p.bnd != 0);
    *n = k;
    return DFA_OK;
}

void dfa_batch_destroy(dfa_batch_t* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->ws) cudaFree(b->ws);
    delete b;
}

int dfa_match_batch(uint32_t count, const dfa_t* const* dfas, const uint8_t* const* strs,
                    const uint64_t* lens, const dfa_match_opts_t* opts, dfa_result_t* dev_out,
                    void* stream) {
    return dfam::no_throw([&]() -> int {
        dfa_batch_t* b = nullptr;
        int rc = dfa_batch_prepare(count, dfas, strs, lens, opts, &b);
        if (rc != DFA_OK) return rc;
        rc = dfa_batch_launch(b, dev_out, stream);
        if (rc == DFA_OK && cudaStreamSynchronize(static_cast<cudaStream_t>(stream)) != cudaSuccess)
            rc = DFA_ECUDA;
        dfa_batch_destroy(b);
        return rc;
    });
}

const char* dfa_strerror(int s) {
    switch (s) {
        case DFA_OK: return "ok";
        case DFA_EINVAL: return "invalid argument";
        case DFA_ESYMBOL: return "input byte not in the alphabet";
        case DFA_ENOMEM: return "out of memory";
        case DFA_ECUDA: return "CUDA error";
        case DFA_ETIMEOUT: return "timed out";
        case DFA_EBUDGET: return "request exceeds the memory budget";
        case DFA_EAGAIN: return "try again";
        case DFA_ENOSPACE: return "workspace too small";
        case DFA_EHOSTONLY: return "DFA has no device image";
        case DFA_EBOUNDS: return "device-side bounds check failed";
        default: return "unknown status";
    }
}

}  // extern "C"
