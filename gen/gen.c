/*
 * Seeded, counter-based input generators shared by the tests, the benchmark and
 * the smoke check.  Nothing here computes anything the membership test
 * computes: these routines only produce byte strings (uniform, categorical,
 * with planted words).  DFA tables are built in gen/__init__.py from the same
 * random stream.
 *
 * Random stream: SplitMix64 (G. Steele, D. Lea, C. Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014).  The i-th draw of stream
 * `key` is the (i+1)-th output of a SplitMix64 generator whose state starts at
 * `key`, i.e. mix(key + (i+1) * 0x9E3779B97F4A7C15).  Because the state of
 * SplitMix64 advances by a constant, the i-th draw is a pure function of
 * (key, i): every position of a string can be generated independently, so the
 * generators split a string across threads and stay bit-identical to a
 * single-threaded run.
 */
#include <pthread.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t draw(uint64_t key, uint64_t i) { return mix64(key + (i + 1) * GOLDEN); }

/* Stream key for (seed, stream id). */
uint64_t gen_key(uint64_t seed, uint64_t stream) {
    return mix64(mix64(seed + GOLDEN) ^ (stream * 0xD1B54A32D192ED03ULL));
}

/* out[j] = draw(key, start + j) */
void gen_u64(uint64_t key, uint64_t start, uint64_t n, uint64_t *out) {
    for (uint64_t j = 0; j < n; ++j) out[j] = draw(key, start + j);
}

/* ---------------------------------------------------------------- threads */

typedef struct {
    int kind;
    uint64_t key, key2;
    uint8_t *out;
    uint64_t lo, hi, n;
    const uint64_t *cdf; /* k cumulative thresholds in units of 2^32, last == 2^32 */
    const uint8_t *syms;
    int k;
    uint64_t rate;       /* planting probability times 2^64 */
    const uint8_t *words;
    const uint32_t *word_off; /* nwords + 1 offsets into words */
    int nwords;
    uint32_t maxlen;
} job_t;

static void run_uniform(job_t *j) {
    for (uint64_t i = j->lo; i < j->hi; ++i) j->out[i] = (uint8_t)(draw(j->key, i) >> 56);
}

/* The first index a with r < cdf[a], found from a per-bucket starting index
 * (bucket = top 12 bits of r) and a short forward scan: the same index the
 * plain binary search gives, without its unpredictable branches. */
#define CAT_BUCKET_BITS 12
static void run_categorical(job_t *j) {
    uint16_t first[1u << CAT_BUCKET_BITS];
    for (uint32_t bkt = 0, a = 0; bkt < (1u << CAT_BUCKET_BITS); ++bkt) {
        const uint64_t lo = (uint64_t)bkt << (32 - CAT_BUCKET_BITS);
        while (a + 1 < (uint32_t)j->k && lo >= j->cdf[a]) ++a;
        first[bkt] = (uint16_t)a;
    }
    for (uint64_t i = j->lo; i < j->hi; ++i) {
        uint64_t r = draw(j->key, i) >> 32; /* uniform in [0, 2^32) */
        uint32_t a = first[r >> (32 - CAT_BUCKET_BITS)];
        while (a + 1 < (uint32_t)j->k && r >= j->cdf[a]) ++a;
        j->out[i] = j->syms[a];
    }
}

/* Word planting.  A word starts at position p when draw(key, p) < rate; which
 * word is chosen by draw(key2, p).  Where planted words overlap, the word that
 * starts later wins.  Each thread owns the output range [lo, hi) and replays
 * every start that can reach it, so the result does not depend on threading. */
static void run_plant(job_t *j) {
    uint64_t first = j->lo >= j->maxlen ? j->lo - j->maxlen + 1 : 0;
    for (uint64_t p = first; p < j->hi; ++p) {
        if (draw(j->key, p) >= j->rate) continue;
        uint64_t w = ((draw(j->key2, p) >> 32) * (uint64_t)j->nwords) >> 32;
        uint32_t a = j->word_off[w], b = j->word_off[w + 1];
        for (uint32_t t = a; t < b; ++t) {
            uint64_t q = p + (t - a);
            if (q >= j->n) break;
            if (q >= j->lo && q < j->hi) j->out[q] = j->words[t];
        }
    }
}

static void *worker(void *arg) {
    job_t *j = (job_t *)arg;
    if (j->kind == 0) run_uniform(j);
    else if (j->kind == 1) run_categorical(j);
    else run_plant(j);
    return NULL;
}

static void run_parallel(job_t proto, uint64_t n, int threads) {
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    if (n < (1u << 20)) threads = 1;
    pthread_t tid[256];
    job_t jobs[256];
    uint64_t per = (n + (uint64_t)threads - 1) / (uint64_t)threads;
    int started = 0;
    for (int t = 0; t < threads; ++t) {
        jobs[t] = proto;
        jobs[t].lo = (uint64_t)t * per;
        jobs[t].hi = jobs[t].lo + per > n ? n : jobs[t].lo + per;
        if (jobs[t].lo >= jobs[t].hi) break;
        if (threads == 1 || pthread_create(&tid[t], NULL, worker, &jobs[t]) != 0) {
            worker(&jobs[t]);
            tid[t] = 0;
        }
        started = t + 1;
    }
    for (int t = 0; t < started; ++t)
        if (threads > 1 && tid[t]) pthread_join(tid[t], NULL);
}

/* out[i] = top byte of draw(key, i) */
void gen_bytes_uniform(uint64_t key, uint8_t *out, uint64_t n, int threads) {
    job_t j;
    memset(&j, 0, sizeof j);
    j.kind = 0; j.key = key; j.out = out; j.n = n;
    run_parallel(j, n, threads);
}

/* out[i] = syms[a] where a is the first index with (draw(key,i) >> 32) < cdf[a] */
void gen_bytes_categorical(uint64_t key, const uint64_t *cdf, const uint8_t *syms, int k,
                           uint8_t *out, uint64_t n, int threads) {
    job_t j;
    memset(&j, 0, sizeof j);
    j.kind = 1; j.key = key; j.out = out; j.n = n; j.cdf = cdf; j.syms = syms; j.k = k;
    run_parallel(j, n, threads);
}

void gen_plant_words(uint64_t key, uint64_t key2, uint64_t rate, const uint8_t *words,
                     const uint32_t *word_off, int nwords, uint8_t *out, uint64_t n, int threads) {
    if (nwords <= 0 || rate == 0 || n == 0) return;
    job_t j;
    memset(&j, 0, sizeof j);
    j.kind = 2; j.key = key; j.key2 = key2; j.out = out; j.n = n; j.rate = rate;
    j.words = words; j.word_off = word_off; j.nwords = nwords;
    uint32_t maxlen = 1;
    for (int w = 0; w < nwords; ++w)
        if (word_off[w + 1] - word_off[w] > maxlen) maxlen = word_off[w + 1] - word_off[w];
    j.maxlen = maxlen;
    run_parallel(j, n, threads);
}
