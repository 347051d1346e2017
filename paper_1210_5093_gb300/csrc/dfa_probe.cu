// Lookup-rate probe: the throughput of the match kernel's unit of work (one
// dependent table lookup s <- T[row(class)][s]) on a compiled DFA's own table
// and placement, with no staging, planning or composition around it.  It
// measures the roofs the match kernel is compared with: for a table in shared
// memory the shared-memory lookup rate (whose derived value is SMs x 32 lanes
// x clock), for a table read through L2 the random-gather rate of L2/L1.
//
// Every thread advances kProbeChains independent chains; all threads take the
// same class at each step (as the lanes of one chunk do), drawn from a
// counter-based hash of the step, so the rows are the table's rows in a
// random order and the states within a row are the chains' own.
#include <cuda_runtime.h>

#include "dfa_internal.h"

namespace {

constexpr int kProbeThreads = 512;
constexpr int kProbeChains = 8;

__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    // a 32-bit finaliser (xorshift-multiply), used only to pick rows and seeds
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

template <int SB, bool SMEM>
__global__ void __launch_bounds__(kProbeThreads) k_probe(const uint8_t* table, uint32_t table_bytes,
                                                         uint32_t rowbytes, uint32_t C, uint32_t qe,
                                                         uint32_t steps, uint32_t* sink) {
    extern __shared__ __align__(16) uint8_t sm[];
    if (SMEM) {
        const uint4* src = reinterpret_cast<const uint4*>(table);
        uint4* dst = reinterpret_cast<uint4*>(sm);
        for (uint32_t i = threadIdx.x; i < (table_bytes + 15) / 16; i += kProbeThreads)
            dst[i] = __ldg(src + i);
        __syncthreads();
    }
    const uint32_t gid = blockIdx.x * kProbeThreads + threadIdx.x;
    uint32_t s[kProbeChains];
#pragma unroll
    for (int u = 0; u < kProbeChains; ++u) s[u] = (mix32(gid * kProbeChains + u) % qe) * SB;
    const uint32_t tb = (uint32_t)__cvta_generic_to_shared(sm);
    for (uint32_t t = 0; t < steps; ++t) {
        const uint32_t row = (mix32(t + 0x9e3779b9u) % C) * rowbytes;
#pragma unroll
        for (int u = 0; u < kProbeChains; ++u) {
            uint32_t v;
            if (SMEM) {
                if (SB == 1) asm volatile("ld.shared.u8 %0, [%1];" : "=r"(v) : "r"(tb + row + s[u]));
                else asm volatile("ld.shared.u16 %0, [%1];" : "=r"(v) : "r"(tb + row + s[u]));
            } else {
                const uint8_t* p = table + row + s[u];
                if (SB == 1) asm volatile("ld.global.nc.u8 %0, [%1];" : "=r"(v) : "l"(p));
                else asm volatile("ld.global.nc.u16 %0, [%1];" : "=r"(v) : "l"(p));
            }
            s[u] = v;
        }
    }
    uint32_t x = 0;
#pragma unroll
    for (int u = 0; u < kProbeChains; ++u) x ^= s[u];
    if (x == 0xFFFFFFFFu) sink[0] = x;  // keeps the chains live; never true for valid states
}

template <int SB, bool SMEM>
int run_probe(const dfam::DevDfa& x, uint32_t steps, cudaStream_t st, double* rate) {
    int dev = 0, sms = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return DFA_ECUDA;
    const uint32_t smem = SMEM ? (x.table_bytes + 15) / 16 * 16 : 0u;
    if (smem > (uint32_t)optin) return DFA_EINVAL;
    if (cudaFuncSetAttribute(k_probe<SB, SMEM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem) != cudaSuccess)
        return DFA_ECUDA;
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_probe<SB, SMEM>, kProbeThreads,
                                                      smem) != cudaSuccess ||
        per_sm < 1)
        return DFA_ECUDA;
    const uint32_t grid = (uint32_t)(sms * per_sm);
    uint32_t* sink = nullptr;
    if (cudaMalloc(&sink, 4) != cudaSuccess) {
        cudaGetLastError();
        return DFA_ENOMEM;
    }
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const uint32_t rowbytes = x.qpad * x.sb;
    int rc = DFA_OK;
    float best = 1e30f;
    for (int rep = 0; rep < 4 && rc == DFA_OK; ++rep) {  // the first launch warms up
        cudaEventRecord(e0, st);
        k_probe<SB, SMEM><<<grid, kProbeThreads, smem, st>>>(x.table, x.table_bytes, rowbytes, x.C,
                                                             x.qe, steps, sink);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = DFA_ECUDA;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(sink);
    if (rc == DFA_OK)
        *rate = (double)grid * kProbeThreads * kProbeChains * steps / (best * 1e-3);
    return rc;
}

}  // namespace

extern "C" int dfa_probe_lookup_rate(const dfa_t* dfa, uint32_t steps, void* stream, double* rate) {
    if (!dfa || !rate || steps == 0) return DFA_EINVAL;
    if (!dfa->on_device) return DFA_EHOSTONLY;
    const dfam::DevDfa& x = dfa->dev;
    if (x.C == 0) return DFA_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool smem = x.placement == dfam::kSmem;
    if (x.sb == 1) return smem ? run_probe<1, true>(x, steps, st, rate) : run_probe<1, false>(x, steps, st, rate);
    if (x.sb == 2) return smem ? run_probe<2, true>(x, steps, st, rate) : run_probe<2, false>(x, steps, st, rate);
    return DFA_EINVAL;
}
