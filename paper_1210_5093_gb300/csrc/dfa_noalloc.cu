// dfa_match_noalloc: the single-test membership test without any device
// allocation by the caller or by the library at call time.
//
// The planning and match kernels need scratch memory (per-chunk classes and
// offsets, tile boundaries, per-test counters and the state maps of the CTAs
// that share a test).  dfa_match_async takes that scratch from the caller and
// dfa_match allocates it; some callers can do neither - for example a host
// loop that has handed all device memory to its own pool, or code that must
// not enter the CUDA allocator while it serves requests.  For them the scratch
// lives in the fixed array below, which every GPU that loads this library
// holds until the process exits.
#include <cuda_runtime.h>

#include <mutex>

#include "dfa_internal.h"

namespace {

constexpr uint64_t kScratchBytes = 16ull << 20;  // 16 MiB per device

// Shared by every call on a device; only host code needs its address, which
// it looks up with cudaGetSymbolAddress (the array's host-side name is not a
// device address and must never be passed to a kernel).
static __device__ __align__(256) uint8_t g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
uint8_t* g_ptr[kMaxDevices] = {};

// The array's device address on the current device.  Outside stream capture
// it is looked up again on every call (a device reset reloads the module at a
// new address, so a cached one could be stale); while `stream` is being
// captured the address from the last lookup on this device is used.
int scratch_ptr(void* stream, uint8_t** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return DFA_ECUDA;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cap) != cudaSuccess) {
        cudaGetLastError();
        return DFA_ECUDA;
    }
    std::lock_guard<std::mutex> g(g_mu);
    if (cap == cudaStreamCaptureStatusNone) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return DFA_ECUDA;
        }
        g_ptr[dev] = static_cast<uint8_t*>(p);
    }
    if (!g_ptr[dev]) return DFA_ECUDA;
    *out = g_ptr[dev];
    return DFA_OK;
}

}  // namespace

extern "C" int dfa_match_noalloc(const dfa_t* dfa, const uint8_t* dev_str, uint64_t len,
                                 const dfa_match_opts_t* opts, dfa_result_t* dev_out,
                                 void* stream) {
    return dfam::no_throw([&]() -> int {
        if (!dfa || !dev_out || (len && !dev_str)) return DFA_EINVAL;
        if (reinterpret_cast<uintptr_t>(dev_out) & 3u) return DFA_EINVAL;  // results are 4-byte aligned
        dfam::Single s;
        int rc = dfam::plan_single(dfa, len, opts, &s);
        if (rc != DFA_OK) return rc;
        if (s.ws.total > kScratchBytes) return DFA_ENOSPACE;
        uint8_t* base = nullptr;
        if ((rc = scratch_ptr(stream, &base)) != DFA_OK) return rc;
        s.lp.test1.str = dev_str;
        dfam::bind(s.lp, base, s.ws);
        s.lp.results = dev_out;
        // the per-test counters that must start at zero are cleared by the launch itself
        return dfam::launch_single(s, stream, opts ? opts->match_begin_event : nullptr,
                                   opts ? opts->match_end_event : nullptr);
    });
}

extern "C" uint64_t dfa_noalloc_scratch_bytes(void) { return kScratchBytes; }
