/*
 * dfamatch.h - C ABI of the GB300 speculative chunked DFA membership test.
 *
 * The operation is the DFA membership test of Ko, Jung, Han & Burgstaller,
 * "A Speculative Parallel DFA Membership Test for Multicore, SIMD and Cloud
 * Computing Environments": given A = (Q, Sigma, delta, q0, F) and a string
 * Str, compute delta*(q0, Str) and whether it lies in F (Sec. 2.1,
 * Algorithm 1).  The library computes it with the paper's speculative method
 * (Algorithm 3): the input is partitioned into chunks (Eqs. 6, 7, 10), every
 * chunk after the first is matched from each state of the initial-state set
 * I_sigma of its reverse-lookahead symbol (Eq. 11), and the resulting state
 * maps are combined in order (Eqs. 8, 9).  The result is identical to
 * Algorithm 1 for every input (the method is failure-free, Sec. 4.4).
 *
 * All entry points return an int status: DFA_OK (0) or a negative DFA_E*
 * code.  No function throws, exits or prints; a failed host allocation is
 * DFA_ENOMEM.  A dfa_t changes only through the tuning calls (dfa_set_tuning*,
 * dfa_autotune*), which must not run while another call uses the same dfa_t;
 * every other call only reads it and may run from several host threads at
 * once.  A dfa_group_t likewise changes only through dfa_group_autotune
 * (dfa_group_match serialises its own use of the group's buffers).  A
 * dfa_batch_t and a dfa_server_t are each used from one host thread at a time
 * (the server's worker runs internally).
 * Device pointers are CUDA device addresses of the current device; "stream"
 * arguments are cudaStream_t values passed as void* (NULL = legacy default
 * stream).
 */
#ifndef DFAMATCH_H
#define DFAMATCH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------ status codes */
#define DFA_OK 0
#define DFA_EINVAL (-1)   /* bad argument: delta entry out of range, q0/finals >= num_states, ... */
#define DFA_ESYMBOL (-2)  /* an input byte is not in Sigma (byte_to_symbol maps it to 0xFF) */
#define DFA_ENOMEM (-3)   /* host or device allocation failed */
#define DFA_ECUDA (-4)    /* a CUDA call failed (no device, launch error, ...) */
#define DFA_ETIMEOUT (-5) /* a bounded device wait gave up (server only) */
#define DFA_EBUDGET (-6)  /* server admission refused: request larger than the HBM budget */
#define DFA_EAGAIN (-7)   /* server: queue full, retry later */
#define DFA_ENOSPACE (-8) /* caller's workspace is smaller than the size query returned */
#define DFA_EHOSTONLY (-9)/* the dfa_t was created with dfa_create_host and has no device image */
#define DFA_EBOUNDS (-10) /* a device-side index check failed: reported only by the library's
                             debug build (libdfamatch_debug.so, compiled with DFA_DEBUG_BOUNDS),
                             which checks every state, class, set slot and chunk bound the
                             kernels use and skips the access instead of making it; the
                             result's final_state then holds the source line of the check */

typedef struct dfa_s dfa_t;
typedef struct dfa_batch_s dfa_batch_t;
typedef struct dfa_server_s dfa_server_t;

/* Result of one membership test (12 bytes, also the device-side layout). */
typedef struct {
    uint32_t final_state; /* delta*(q0, Str) in the caller's state numbering;
                             == num_states when the run ended in the implicit
                             error state q_e (a -1 entry of delta was taken)  */
    uint8_t accept;       /* 1 iff final_state is in F                          */
    uint8_t reserved[3];
    int32_t status;       /* DFA_OK, or DFA_ESYMBOL (then final_state/accept are 0);
                             DFA_EBOUNDS only in the debug build                  */
} dfa_result_t;

/* Static properties of a compiled DFA (Eqs. 11, 12, 18 and the device layout). */
typedef struct {
    uint32_t num_states;     /* |Q| as given                                       */
    uint32_t num_symbols;    /* |Sigma| as given                                   */
    uint32_t num_states_ext; /* |Q| + 1: the implicit error state q_e is state |Q| */
    uint32_t num_classes;    /* alphabet classes after merging identical columns   */
    uint32_t i_max;          /* Eq. (12): max_sigma |I_sigma|                      */
    uint32_t num_excluded;   /* non-accepting absorbing states left out of every I */
    uint32_t state_bytes;    /* table entry size: 1 (|Q|+1 <= 256), 2 (<= 32768), else 4 */
    uint32_t placement;      /* 0 = table in shared memory, 1 = table read through L2 */
    uint32_t states_per_thread; /* chains one thread advances together (planner's K) */
    uint32_t q0;
    uint64_t table_bytes;    /* device transition-table image, incl. identity row  */
    uint64_t device_bytes;   /* all device memory held by this dfa_t               */
    double gamma;            /* Eq. (18): I_max / |Q|                              */
    double mean_iset;        /* mean |I_c| over the classes                        */
    uint32_t byte_rows;      /* 1: chains visit at most 16 states, so single-test
                                launches with few chains (at most 128 per SM, where
                                the chains are latency-bound) step them by byte
                                permutes of 16-byte class rows held in shared memory
                                instead of table loads; other launches use the table */
    uint32_t reserved;
} dfa_info_t;

/* Per-DFA tuning record (the GPU counterpart of the paper's per-processor
 * profiling, Sec. 4.1): how many chains one thread advances and how long the
 * chunks are.  Zero fields mean "library default". */
typedef struct {
    uint32_t states_per_thread; /* K in {2, 4, 8, 16}; ceil(I_max/K) must be <= 256
                                   unless K = 16 (Algorithm 2 launches raise K as
                                   needed, up to 16)                                  */
    uint32_t tiles_per_cta;     /* single tests: aim for this many tiles per CTA (default 8) */
    uint32_t min_chunk_bytes;   /* single tests: shortest chunk (default 512)          */
    uint32_t batch_chunk_bytes; /* batched and served tests: chunk length (default 8192) */
    uint32_t ctas_per_sm;       /* single tests: match-kernel CTAs per SM to aim for
                                   (0 = 3 when K <= 4, else 2)                          */
    uint32_t host_segment_bytes; /* dfa_match on a host buffer: length of the first
                                   segment of the copy/match pipeline (later segments
                                   double); 0 = automatic (len/32 clamped to
                                   [16 MiB, 256 MiB]), 0xFFFFFFFF = copy the whole
                                   string before matching                              */
    uint32_t grid_waves;        /* single tests: match-kernel CTAs as a multiple (1-4) of
                                   those that fit the GPU at once (0 = 1, one resident
                                   wave).  The work and chunks stay the same; each CTA
                                   takes 1/waves of a resident CTA's share, and the
                                   hardware starts the next CTA wherever one finished,
                                   which evens out SMs that run at different speeds.
                                   Safe because no CTA waits for another.              */
} dfa_tuning_t;

/* Optional per-call planning overrides; pass NULL for the defaults. */
typedef struct {
    uint32_t num_chunks;   /* P; 0 = chosen by the planner                         */
    uint32_t multiplicity; /* the per-chunk state count m in Eqs. (5)-(7)/(10);
                              0 = 1 (a chunk's states run on parallel lanes)      */
    uint32_t lookahead;    /* reverse-lookahead symbols r: 1 = Algorithm 3 (the
                              default; pass 1 explicitly when using this struct),
                              0 = Algorithm 2 (every chunk matched from all of Q),
                              2..8 = the r-symbol sets of Eq. (13), computed per
                              chunk on the device                                 */
    uint32_t boundary_window; /* Sec. 4.2's boundary placement (chunks cut right
                              after symbols whose initial-state set is small, an
                              optimization the paper suggests): 0 = the chunk starts of
                              Eqs. (6)-(7) (the default); w > 0 = on the device,
                              each start S of a chunk k >= 1 moves to the position
                              p in [S - w', S + w'] whose preceding byte has the
                              smallest |I_class| (a byte outside Sigma counts as
                              larger than any set), ties to the p nearest S, then
                              to the smaller p.  w' = min(w, floor(len / (m + P -
                              1)) / 4): a quarter of the shortest later chunk, so
                              starts stay increasing.  Chunk k's set (and, for
                              lookahead >= 2, its Eq. (13) set) is then taken at
                              the placed start.  Ignored by Algorithm 2
                              (lookahead 0).  At most 65536 (DFA_EINVAL above).
                              The answer never depends on it (failure-freedom);
                              the work sum_k L_k |I_k| usually drops.           */
    void *match_begin_event; /* optional cudaEvent_t recorded on the stream right before  */
    void *match_end_event;   /* ... and right after the match kernel (for timing it alone) */
} dfa_match_opts_t;

/* ------------------------------------------------------------- DFA objects */

/*
 * Compile a DFA (Sec. 2.1) and upload it to the current CUDA device.
 *   delta          num_states*num_symbols int32, row-major: delta[q*num_symbols + a]
 *                  is the target of state q on symbol a, or -1 for the implicit
 *                  error state q_e (numbered num_states).  Copied.
 *   q0             start state, < num_states.
 *   finals         num_finals accepting states (< num_states, duplicates allowed). Copied.
 *   byte_to_symbol 256 entries mapping an input byte to a symbol (< num_symbols),
 *                  or 0xFF for "not in Sigma"; NULL = identity (needs num_symbols == 256).
 * Limits: 1 <= num_states <= 65534 (states, q_e included, are 16-bit ids with
 * 0xFFFF reserved), 1 <= num_symbols <= 256.  A chunk whose initial-state set
 * holds more chains than one thread block runs them in several passes over the
 * chunk, and launches with sets above 4096 states keep their running state
 * maps in global memory (part of the workspace); the r-symbol sets of Eq. (13)
 * (opts->lookahead >= 2) are available for num_states <= 4095 (DFA_EINVAL
 * above), and dfa_match pipelines host input only for such DFAs.
 * Compilation (the set computation of Algorithm 3, done once): bytes with identical delta
 * columns share a class; I_c (Eq. 11) and I_max (Eq. 12) are computed; the
 * class-major table (uint8 states if |Q|+1 <= 256, uint16 up to 32768, else
 * uint32) is placed in shared memory if it fits, otherwise read through L2.
 * Errors: DFA_EINVAL, DFA_ENOMEM, DFA_ECUDA.  *out is NULL on error.
 */
int dfa_create(uint32_t num_states, uint32_t num_symbols, const int32_t *delta, uint32_t q0,
               const uint32_t *finals, uint32_t num_finals, const uint8_t *byte_to_symbol,
               dfa_t **out);

/* Same compilation without any CUDA call; the result supports dfa_info,
 * dfa_class_of_bytes and dfa_iset only (match calls return DFA_EHOSTONLY). */
int dfa_create_host(uint32_t num_states, uint32_t num_symbols, const int32_t *delta,
                    uint32_t q0, const uint32_t *finals, uint32_t num_finals,
                    const uint8_t *byte_to_symbol, dfa_t **out);

/* Free a DFA and its device memory.  NULL is ignored.  No launch may still use it. */
void dfa_destroy(dfa_t *dfa);

int dfa_info(const dfa_t *dfa, dfa_info_t *out);

/* Read / replace the tuning record.  dfa_set_tuning re-uploads the DFA's
 * device descriptor (synchronous); no launch may use the DFA meanwhile.
 * Errors: DFA_EINVAL (K not allowed), DFA_ECUDA. */
int dfa_get_tuning(const dfa_t *dfa, dfa_tuning_t *out);
int dfa_set_tuning(dfa_t *dfa, const dfa_tuning_t *tuning);

/*
 * Autotuner: times single-test launches of the device string dev_sample
 * (len bytes) for every allowed K in {2, 4, 8, 16}, tiles-per-CTA in
 * {1, 2, 4, 8, 16} and, for K <= 4, 2 or 3 CTAs per SM, plus shortest chunks of
 * 2 and 8 KiB where the default shortest chunk bounds the chunk count
 * (median of 3 timed launches each, CUDA events on `stream`),
 * keeps the fastest as the DFA's tuning record (of the candidates within 1%
 * of the fastest, the one with the most CTAs per SM: more, smaller CTAs let
 * consecutive or concurrent launches share the SMs) and returns it in
 * *chosen and its time in *best_ms (either may be NULL).  The batched chunk
 * length is set to the chosen single-test chunk length, clamped to
 * [8 KiB, 64 KiB].  Launches of several DFAs (batches, the server) use each
 * DFA's compiler K (from its mean set size; with Sec. 4.2 placement, from its
 * smallest set) capped at 8 rather than the tuned K: one kernel variant
 * serves the whole launch.
 * Allocates a temporary workspace; synchronises the stream.
 */
int dfa_autotune(dfa_t *dfa, const uint8_t *dev_sample, uint64_t len, void *stream,
                 dfa_tuning_t *chosen, double *best_ms);

/*
 * Tuning records per lookahead depth.  A DFA keeps one base record (the one
 * dfa_get_tuning / dfa_set_tuning / dfa_autotune read and write, used for
 * lookahead 1) and may keep one record per other depth r = opts->lookahead
 * (0 = Algorithm 2, 2..8 = Eq. (13) sets): the sets shrink as r grows, so the
 * best chains per thread and tiles per CTA differ.  Each depth r >= 1 also
 * has a record for launches with Sec. 4.2 boundary placement
 * (opts->boundary_window > 0), whose sets are smaller still.  A placed record
 * that was never set reads as its depth's record, and a depth without its own
 * record as the base record.  These three calls read, write or autotune the
 * record of (opts->lookahead, opts->boundary_window > 0) (opts NULL =
 * lookahead 1 without placement = the base record).  dfa_autotune_opts times
 * launches with that lookahead and window (k_lookahead, k_boundaries
 * included).  Errors: as dfa_get_tuning / dfa_set_tuning / dfa_autotune, and
 * DFA_EINVAL for a lookahead above 8 or a window above 65536.
 */
int dfa_get_tuning_opts(const dfa_t *dfa, const dfa_match_opts_t *opts, dfa_tuning_t *out);
int dfa_set_tuning_opts(dfa_t *dfa, const dfa_match_opts_t *opts, const dfa_tuning_t *tuning);
int dfa_autotune_opts(dfa_t *dfa, const uint8_t *dev_sample, uint64_t len,
                      const dfa_match_opts_t *opts, void *stream, dfa_tuning_t *chosen,
                      double *best_ms);

/* out[256]: alphabet class of every byte, 0xFFFF for bytes not in Sigma. */
int dfa_class_of_bytes(const dfa_t *dfa, uint16_t *out);

/* Initial-state set I_c of class c (Eq. 11, ascending state ids), written to
 * states[0..cap); *count receives |I_c| (even when larger than cap).
 * c == num_classes returns the start set {q0} used for the first chunk;
 * c == num_classes + 1 returns all of Q (the set Algorithm 2 matches). */
int dfa_iset(const dfa_t *dfa, uint32_t c, uint32_t *states, uint32_t cap, uint32_t *count);

/*
 * Eqs. (6)-(7) with unit weights and per-chunk state count m (Eq. 10):
 * starts[0] = 0, starts[k] = floor(n*(m+k-1)/(m+P-1)) for 1 <= k < P,
 * starts[P] = n; chunk k covers [starts[k], starts[k+1]).  starts has P+1
 * entries, caller-owned.  Host only.  Errors: DFA_EINVAL (P == 0 or m == 0).
 */
int dfa_partition(uint64_t n, uint32_t P, uint32_t m, uint64_t *starts);

/* ------------------------------------------------------------- matching */

/*
 * Synchronous membership test.  str may be a host or a device pointer
 * (detected with cudaPointerGetAttributes).  Host input of at least two
 * first-segment lengths (dfa_tuning_t.host_segment_bytes) is copied and
 * matched as a pipeline when opts sets neither num_chunks nor multiplicity
 * (segments double in length up to an eighth of the string, or up to a
 * quarter when the DFA's autotuned device rate is below 150 GB/s, so that the
 * copies stay ahead of the matching and fewer launches are needed):
 * each segment is copied on a library-owned copy stream and matched, once its
 * copy has landed, as its own launch on one of two library-owned compute
 * streams (so consecutive launches overlap).  Every segment after the first
 * takes its first chunk's reverse lookahead from the previous segment's last
 * bytes and yields the state map of the whole segment; a final kernel applies
 * those maps to the first segment's final state (Eq. 8), so the answer equals
 * the unsegmented one.  Shorter or
 * explicitly partitioned host input is copied whole first.  The copies
 * overlap only when the host buffer is pinned.  Device staging buffer,
 * workspace and streams are kept per device between calls (grown on demand;
 * calls are serialised by a lock).  *out is a host struct.  Errors:
 * DFA_EINVAL, DFA_ESYMBOL (also in out->status), DFA_ENOMEM, DFA_ECUDA,
 * DFA_EHOSTONLY.
 */
int dfa_match(const dfa_t *dfa, const uint8_t *str, uint64_t len, const dfa_match_opts_t *opts,
              dfa_result_t *out);

/* Number of chunks P the planner uses for a single test of len bytes
 * (opts->num_chunks when given); the partition is then dfa_partition(len, P, m),
 * or, with opts->boundary_window, the placed starts of dfa_plan_starts. */
int dfa_plan_chunks(const dfa_t *dfa, uint64_t len, const dfa_match_opts_t *opts, uint32_t *P);

/*
 * Inspection: the chunk boundaries a single test of dev_str (device, len
 * bytes) uses: starts[0] = 0, starts[k] = the start of chunk k, starts[P] =
 * len (P + 1 entries; at most cap written; *P receives the chunk count).
 * Without a placement window these are Eqs. (6)-(7) and nothing runs on the
 * device; with opts->boundary_window the placement kernel runs on dev_str
 * (Sec. 4.2) and its starts are copied back (temporary workspace, device
 * synchronised).  Errors: DFA_EINVAL, DFA_ENOMEM, DFA_ECUDA, DFA_EHOSTONLY.
 */
int dfa_plan_starts(const dfa_t *dfa, const uint8_t *dev_str, uint64_t len,
                    const dfa_match_opts_t *opts, uint64_t *starts, uint32_t cap, uint32_t *P);

/*
 * Inspection: run only the planning kernels of a single test on dev_str and
 * return, for each of its P chunks, the size of the initial-state set it is
 * matched from (sizes[k] = |I_k|; chunk 0 and chunks preceded only by empty
 * chunks have 1).  *P receives the chunk count; at most cap sizes are
 * written.  Allocates a temporary workspace and synchronises the device.
 */
int dfa_plan_sets(const dfa_t *dfa, const uint8_t *dev_str, uint64_t len,
                  const dfa_match_opts_t *opts, uint32_t *sizes, uint32_t cap, uint32_t *P);

/* Kernel launches one dfa_match_async / dfa_match call issues for (dfa, len,
 * opts): the planning kernels (one fused kernel for plans of at most 2048
 * chunks, else four), k_boundaries when a placement window applies,
 * k_lookahead when opts->lookahead >= 2, and the match kernel. */
int dfa_match_num_kernels(const dfa_t *dfa, uint64_t len, const dfa_match_opts_t *opts,
                          uint32_t *n);

/*
 * Inspection: run a single test on dev_str and return its chunk maps, the
 * vectors L_k of Sec. 4.1: maps[k*(num_states+1) + j] = delta*(j, chunk k)
 * for every j in the chunk's initial-state set I_k, and j (the identity, as
 * in Algorithm 3's initialisation) for the other states.  maps has
 * P*(num_states+1) entries, P as returned in *P (at most cap chunks are
 * written).  *final_state receives the test's answer.  Allocates temporary
 * device memory and synchronises the device.
 */
int dfa_debug_chunk_maps(const dfa_t *dfa, const uint8_t *dev_str, uint64_t len,
                         const dfa_match_opts_t *opts, uint16_t *maps, uint32_t cap, uint32_t *P,
                         uint32_t *final_state);

/* Device workspace needed by dfa_match_async for (dfa, len, opts). */
int dfa_match_workspace_size(const dfa_t *dfa, uint64_t len, const dfa_match_opts_t *opts,
                             uint64_t *bytes);

/*
 * Asynchronous membership test on `stream`: dev_str (device, len bytes) ->
 * dev_out (one device dfa_result_t).  dev_workspace must hold at least the
 * size returned by dfa_match_workspace_size; it is owned by the caller and
 * must not be used by another launch until this one completes.  Launches
 * only kernels and memsets (no allocation, no host synchronisation), so it
 * can be captured in a CUDA graph.  A byte outside Sigma is reported in
 * dev_out->status.  dev_out must be 4-byte aligned and dev_workspace
 * 256-byte aligned (DFA_EINVAL otherwise).
 * Errors (returned): DFA_EINVAL, DFA_ENOSPACE, DFA_ECUDA.
 */
int dfa_match_async(const dfa_t *dfa, const uint8_t *dev_str, uint64_t len,
                    const dfa_match_opts_t *opts, dfa_result_t *dev_out, void *dev_workspace,
                    uint64_t workspace_bytes, void *stream);

/*
 * Allocation-free variant of dfa_match_async, for callers that cannot call
 * cudaMalloc at all and have no workspace to hand over (for example a loop
 * that gave all device memory to its own pool, or code that must not enter
 * the CUDA allocator while serving).  The paper has no counterpart: this is
 * a property of the library, not of the method.
 * The scratch space is a fixed 16 MiB device array inside the library
 * (dfa_noalloc_scratch_bytes()), held by every GPU that loads the library
 * until the process exits.  The caller still passes the input (device,
 * len bytes) and dev_out (one device dfa_result_t).  A call whose plan needs
 * more scratch than that returns DFA_ENOSPACE before launching anything;
 * lower opts->num_chunks or use dfa_match_async.  No call allocates memory
 * (no cudaMalloc, cudaFree or allocating library routine); the parts of the
 * scratch that must start at zero are cleared on the stream by each call.
 * All calls on a device share the one array, which keeps the last call's
 * contents: calls whose work overlaps on the GPU (other streams, or another
 * host thread) race and give wrong results; order them on one stream.  Each
 * call made outside stream capture looks up the array's device address on the
 * current device (cheap after the first time), so a cudaDeviceReset between
 * calls, which reloads the library's device code at a new address, is
 * harmless; a call made while `stream` is being captured uses the address
 * found by the last call outside capture on that device.  So make the first
 * call on each device, and the first call after a device reset, before any
 * stream capture (during capture without one: DFA_ECUDA).
 */
int dfa_match_noalloc(const dfa_t *dfa, const uint8_t *dev_str, uint64_t len,
                      const dfa_match_opts_t *opts, dfa_result_t *dev_out, void *stream);
/* Size in bytes of the scratch array dfa_match_noalloc uses. */
uint64_t dfa_noalloc_scratch_bytes(void);

/*
 * Batched membership tests: count independent tests (dfas[i], strs[i],
 * lens[i]), each computed by the same method as dfa_match (Algorithm 3 on its
 * own partition, Eqs. 6-7, combined by Eqs. 8-9), run in one persistent
 * launch (plus four small planning launches).  Several tests may share one
 * string under different DFAs, the paper's use of one symbol-index input by
 * several DFAs (Sec. 5).
 * dfas may repeat (tests are grouped by DFA); strs are device pointers;
 * results go to dev_out[0..count) (device).  Host arrays are read before
 * the call returns; strings must stay valid until the stream reaches the end
 * of the work.  Allocates and frees its own workspace and synchronises the
 * stream.  For repeated launches use dfa_batch_prepare / dfa_batch_launch.
 */
int dfa_match_batch(uint32_t count, const dfa_t *const *dfas, const uint8_t *const *strs,
                    const uint64_t *lens, const dfa_match_opts_t *opts, dfa_result_t *dev_out,
                    void *stream);

/*
 * Prepared batch: plans the tests on the host (chunk counts per test chosen
 * from each DFA's tuning record), uploads the descriptors and allocates the
 * workspace once (synchronous).  dfa_batch_launch then issues only kernels
 * and memsets on `stream` (capturable); dfa_batch_graph_launch captures the
 * launch into a CUDA graph on first use and replays it afterwards.  The
 * dfas and strings must outlive the batch.
 */
int dfa_batch_prepare(uint32_t count, const dfa_t *const *dfas, const uint8_t *const *strs,
                      const uint64_t *lens, const dfa_match_opts_t *opts, dfa_batch_t **out);
int dfa_batch_launch(dfa_batch_t *batch, dfa_result_t *dev_out, void *stream);
int dfa_batch_graph_launch(dfa_batch_t *batch, dfa_result_t *dev_out, void *stream);
/* Optional cudaEvent_t pair recorded around the match kernel by later
 * dfa_batch_launch calls (NULL, NULL to stop).  Not applied to graph launches. */
int dfa_batch_set_events(dfa_batch_t *batch, void *match_begin_event, void *match_end_event);
/* Kernel launches one dfa_batch_launch issues (for accounting). */
int dfa_batch_num_kernels(const dfa_batch_t *batch, uint32_t *n);
void dfa_batch_destroy(dfa_batch_t *batch);

/*
 * Measurement: the rate, in lookups per second, of the match kernel's unit of
 * work - one dependent table lookup s <- T[row(class)][s] (Algorithm 3's inner
 * step; Eq. 16 counts these) - on this DFA's own table and placement, with no
 * staging, planning or composition: every thread of a full-GPU launch
 * advances 8 independent chains for `steps` steps, all threads taking the
 * same class per step (as one chunk's lanes do).  For a table in shared
 * memory this probes the shared-memory lookup roof; for a table read through
 * L2, the random-gather rate.  Best of three timed launches (CUDA events on
 * `stream`), after a warm-up launch; synchronises the stream.  Tables with
 * 1- or 2-byte entries.  Errors: DFA_EINVAL, DFA_ECUDA, DFA_ENOMEM,
 * DFA_EHOSTONLY.
 */
int dfa_probe_lookup_rate(const dfa_t *dfa, uint32_t steps, void *stream, double *lookups_per_s);

/* Human-readable text for a status code (static storage). */
const char *dfa_strerror(int status);

/* ---------------------------------------------- several DFAs on one input */

/*
 * A group matches several DFAs against one input string and reads and
 * converts that input once for all of them.  This is the arrangement of
 * Sec. 5: the tables of several DFAs stored side by side (SBase), and one
 * input converted to symbol indices (IBase) that every DFA reads.  Each DFA's
 * answer is computed by the method dfa_match uses (Algorithm 3 with one
 * reverse-lookahead symbol, Eqs. 8-9 to combine), on chunk starts shared by
 * the whole group (Eqs. 6-7 with unit weights and m = 1), so it equals the
 * answer dfa_match gives for that DFA alone.
 *
 * Joint classes: two bytes share a joint class iff they share a class in
 * every DFA of the group (or lie outside Sigma for the same DFAs).  The input
 * is staged once as joint-class indices, and the group holds a copy of every
 * DFA's table with one row per joint class.  This suits DFAs over one
 * alphabet, such as protein patterns over the 20 amino-acid letters (at most
 * 21 joint classes); DFAs with unrelated byte classes give many joint classes
 * and large tables.
 *
 * Limits (DFA_EINVAL at creation): 1 <= count <= 16 DFAs, each with at most
 * 4095 states; at most 255 joint classes; all joint tables together at most
 * 160 KiB (every thread block holds all of them in shared memory); the sum
 * over the DFAs of their largest initial-state set (Eq. 12, or 1) at most 8192,
 * and at most 512 thread slots for one chunk's sets at K = 16.
 */
typedef struct dfa_group_s dfa_group_t;

typedef struct {
    uint32_t num_dfas;
    uint32_t joint_classes;     /* J                                                  */
    uint32_t state_bytes;       /* joint-table entry size: 1 if every |Q|+1 <= 256, else 2 */
    uint32_t states_per_thread; /* default K (chains one thread advances together):
                                   for one DFA the compiler's rule on its mean set size,
                                   for several at most 2 (raised until one chunk's sets
                                   fit 512 threads), or what dfa_group_autotune chose   */
    uint32_t ctas_per_sm;       /* default thread blocks per SM (0: 2 where shared
                                   memory allows), or what dfa_group_autotune chose    */
    uint32_t max_states_ext;    /* largest |Q|+1 of the group: the row stride of
                                   dfa_group_debug_chunk_maps                          */
    uint32_t sum_max_set;       /* sum over the DFAs of their largest initial-state set */
    uint32_t reserved;
    uint64_t table_bytes;       /* all joint tables (J+1 rows per DFA)                */
    uint64_t device_bytes;      /* device memory held by the group (0: host-only)     */
} dfa_group_info_t;

/* Optional per-call settings; NULL for the defaults. */
typedef struct {
    uint32_t num_chunks;        /* P, shared by the group's DFAs; 0 = planner default  */
    uint32_t states_per_thread; /* K in {1, 2, 4, 8, 16}; 0 = the group's default. One
                                   chunk's sets must fit 512 threads (DFA_EINVAL)      */
    uint32_t ctas_per_sm;       /* 1 or 2; 0 = the group's default                     */
    uint32_t reserved;          /* 0                                                   */
    uint64_t *dev_work;         /* optional device uint64 (8-byte aligned): receives the
                                   launch's lookups, the sum over DFAs and chunks of
                                   L_k |I_k| (the work term of Eq. 16)                 */
    void *match_begin_event;    /* optional cudaEvent_t pair recorded right before and */
    void *match_end_event;      /* after the match kernel                              */
} dfa_group_opts_t;

/*
 * Builds a group of count DFAs (joint classes, joint tables) and uploads it to
 * the current device, which must be the DFAs' device.  The DFAs must outlive
 * the group.  DFAs made by dfa_create_host give a host-only group:
 * dfa_group_info and dfa_group_joint_classes work, the other calls return
 * DFA_EHOSTONLY.  Mixing device and host-only DFAs is DFA_EINVAL.
 * Errors: DFA_EINVAL (limits above), DFA_ENOMEM, DFA_ECUDA.  *out is NULL on error.
 */
int dfa_group_create(const dfa_t *const *dfas, uint32_t count, dfa_group_t **out);
void dfa_group_destroy(dfa_group_t *group);
int dfa_group_info(const dfa_group_t *group, dfa_group_info_t *out);
/* out[b] (256 entries): the joint class of byte b. */
int dfa_group_joint_classes(const dfa_group_t *group, uint16_t *out);
/*
 * Tuning (the GPU counterpart of the paper's per-processor profiling, Sec. 4.1):
 * times every K in {1, 2, 4, 8, 16} whose chunk sets fit 512 threads, with 1
 * and 2 thread blocks per SM, on a device sample of len bytes (one warm-up and
 * two timed launches each, CUDA events on `stream`), and keeps the fastest as
 * the group's default.  *states_per_thread, *ctas_per_sm and *best_ms (each
 * optional) receive it.  Allocates a workspace and synchronises the stream.
 * Errors: DFA_EINVAL, DFA_EHOSTONLY, DFA_ENOMEM, DFA_ECUDA.
 */
int dfa_group_autotune(dfa_group_t *group, const uint8_t *dev_sample, uint64_t len, void *stream,
                       uint32_t *states_per_thread, uint32_t *ctas_per_sm, double *best_ms);
/* P that dfa_group_match_async uses for (group, len, opts). */
int dfa_group_plan_chunks(const dfa_group_t *group, uint64_t len, const dfa_group_opts_t *opts,
                          uint32_t *P);
int dfa_group_workspace_size(const dfa_group_t *group, uint64_t len, const dfa_group_opts_t *opts,
                             uint64_t *bytes);

/*
 * Asynchronous membership test of every DFA of the group on dev_str (device,
 * len < 2^46 bytes), on `stream`: dev_out[i] (device, count entries, 4-byte
 * aligned) receives DFA i's result, with DFA_ESYMBOL in its status when the
 * input holds a byte outside that DFA's Sigma (the other DFAs' results are
 * unaffected).  dev_workspace (256-byte aligned, at least
 * dfa_group_workspace_size bytes) is the caller's and must not be used by
 * another launch until this one completes.  Issues one memset and two kernels
 * (no allocation, no host synchronisation).
 * Errors (returned): DFA_EINVAL, DFA_ENOSPACE, DFA_EHOSTONLY, DFA_ECUDA.
 */
int dfa_group_match_async(const dfa_group_t *group, const uint8_t *dev_str, uint64_t len,
                          const dfa_group_opts_t *opts, dfa_result_t *dev_out, void *dev_workspace,
                          uint64_t workspace_bytes, void *stream);

/*
 * Synchronous form of dfa_group_match_async for host or device input: str is
 * len bytes of host memory or a device pointer.  Host input of at least
 * 32 MiB is copied in segments (doubling from len/32, clamped to
 * [16 MiB, 256 MiB], up to a quarter of the string) on a stream of the group
 * while the earlier segments are matched on another: every segment after the
 * first is matched from the sets of its lookahead byte and yields each DFA's
 * state map of the segment, and Eq. (8) over those maps gives the answer
 * (groups whose DFAs' |Q|+1, rounded up to 8, sum to at most 8192, and calls
 * without num_chunks, dev_work or events; otherwise the string is copied
 * whole first).  Pinned host memory copies fastest.  out[i] (host, count entries) receives
 * DFA i's result, its status DFA_ESYMBOL when the input holds a byte outside
 * DFA i's Sigma.  The call returns DFA_OK when the launch ran, whatever the
 * results' status.  The group keeps the input copy, workspace and results
 * buffers between calls (freed by dfa_group_destroy); calls on one group are
 * serialised.  Runs on the legacy default stream and synchronises it.
 * Errors: DFA_EINVAL, DFA_EHOSTONLY, DFA_ENOMEM, DFA_ECUDA.
 */
int dfa_group_match(dfa_group_t *group, const uint8_t *str, uint64_t len,
                    const dfa_group_opts_t *opts, dfa_result_t *out);

/*
 * Inspection: the chunk maps L_k (Sec. 4.1) of every DFA of the group, as the
 * match kernel computed them: maps[(i*np + k)*stride + j] = delta_i*(j, chunk k)
 * for j in DFA i's I_k and j otherwise, with np = min(cap, P) and stride =
 * max_states_ext of dfa_group_info.  final_states[i] (optional, count
 * entries) gets DFA i's final state (0xFFFFFFFF for a failed test).  *P
 * receives the chunk count; with maps and final_states both NULL nothing is
 * launched.  Allocates device memory and synchronises the device.
 */
int dfa_group_debug_chunk_maps(const dfa_group_t *group, const uint8_t *dev_str, uint64_t len,
                               const dfa_group_opts_t *opts, uint16_t *maps, uint32_t cap,
                               uint32_t *P, uint32_t *final_states);

/* ------------------------------------------------------------- serving */

typedef struct {
    uint64_t ticket;        /* value returned by dfa_server_submit            */
    dfa_result_t result;
    double submit_s;        /* host steady-clock seconds at submission        */
    double done_s;          /* host seconds when the result was on the host   */
} dfa_completion_t;

typedef struct {
    uint64_t submitted, completed, rejected, launches, bytes_matched;
    uint64_t bytes_in_flight, max_bytes_in_flight;
    uint64_t max_concurrent;  /* most batches that were on the device at once */
} dfa_server_stats_t;

/*
 * A serving loop on the current device: requests (dfa, host string) are
 * admitted while the bytes in flight stay within hbm_budget_bytes, grouped
 * into batches as they arrive and launched on max_inflight streams (0 = 8,
 * at most 64), so new requests start while earlier batches still run
 * (continuous batching).  A batch takes at most hbm_budget_bytes /
 * max_inflight bytes and at most 512 MiB, so one batch's copies overlap
 * another's matching.  While two batches and 512 MiB are on the device, a
 * queue shorter than 512 MiB is held back to grow into the next batch (fewer,
 * larger launches under load); otherwise requests are launched at once.
 * Input copies run in launch order on one copy stream.
 * DFAs must stay alive while requests on them are pending.
 */
int dfa_server_create(uint64_t hbm_budget_bytes, uint32_t max_inflight, dfa_server_t **out);
/* Planning options of the batches formed from now on: opts->lookahead (Algorithm
 * 2/3, Eq. 13) and opts->boundary_window (Sec. 4.2 placement); NULL restores the
 * default (lookahead 1, no placement).  num_chunks, multiplicity and the events
 * must be 0 (they are per test, the server plans per batch).  The answers never
 * depend on it.  Errors: DFA_EINVAL. */
int dfa_server_set_opts(dfa_server_t *srv, const dfa_match_opts_t *opts);
/* Queues the test (dfa, str): str is host memory of len bytes that the server
 * copies to the device when it forms the request's batch, so it must stay valid
 * and unchanged until the request's completion has been polled.  The copy is
 * asynchronous (and overlaps other batches' matching) only when str is pinned
 * host memory (cudaHostAlloc / cudaHostRegister); from pageable memory it is
 * synchronous.  *ticket receives the request's id.
 * Errors: DFA_EBUDGET (len > budget), DFA_EAGAIN, DFA_EINVAL, DFA_ENOMEM. */
int dfa_server_submit(dfa_server_t *srv, const dfa_t *dfa, const uint8_t *str, uint64_t len,
                      uint64_t *ticket);
/* Moves up to max finished requests into out[0..*n). Non-blocking. */
int dfa_server_poll(dfa_server_t *srv, dfa_completion_t *out, uint32_t max, uint32_t *n);
/* Blocks until every submitted request has completed (or timeout_s passes: DFA_ETIMEOUT). */
int dfa_server_drain(dfa_server_t *srv, double timeout_s);
int dfa_server_stats(const dfa_server_t *srv, dfa_server_stats_t *out);
void dfa_server_destroy(dfa_server_t *srv);

#ifdef __cplusplus
}
#endif
#endif /* DFAMATCH_H */
