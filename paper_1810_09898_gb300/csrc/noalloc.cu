// Keys + sort for callers that cannot allocate device memory.
//
// Some callers of this library may not call cudaMalloc / cudaFree at all: plug-ins
// whose host application owns every byte of device memory through its own pool and
// budget, and latency-critical paths where the implicit device-wide synchronisation
// of cudaMalloc / cudaFree is not acceptable.  For them sphgrp_sfc_keys_sort_static
// runs the same key and radix-sort kernels as sphgrp_sfc_keys_sort, with the sort's
// scratch (the second ping-pong buffer pair, the digit histograms, the scan's block
// sums and the error flag) in one file-scope __device__ array of fixed size instead of
// a context's workspace.  Every GPU that loads the library holds that array until the
// process exits.
#include <mutex>

#include "sph_internal.cuh"

namespace sphgrp {
int sort_keys_scratch(int64_t n, const double* pos, uint64_t* keys_out, int32_t* perm_out,
                      uint64_t* keys_alt, int32_t* perm_alt, uint32_t* hist, int64_t hist_words,
                      int32_t* scan_aux, int64_t scan_aux_words, unsigned* err, cudaStream_t s);
}

using namespace sphgrp;

namespace {

constexpr int64_t kMaxN = SPHGRP_STATIC_SORT_MAX_N;
constexpr size_t kAlign = 256;
constexpr size_t round_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
constexpr size_t kHistWords = 256 * ((kMaxN + kSortTile - 1) / kSortTile);   // one row per sort tile
constexpr size_t kAuxWords = 4096;
constexpr size_t kOffErr = 0;
constexpr size_t kOffKeys = round_up(kOffErr + sizeof(unsigned));
constexpr size_t kOffPerm = round_up(kOffKeys + sizeof(uint64_t) * kMaxN);
constexpr size_t kOffHist = round_up(kOffPerm + sizeof(int32_t) * kMaxN);
constexpr size_t kOffAux = round_up(kOffHist + sizeof(uint32_t) * kHistWords);
constexpr size_t kBytes = round_up(kOffAux + sizeof(int32_t) * kAuxWords);

// The scratch itself.  Host code must not use its name as a device address (on the
// host it names a stand-in); the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_sort_scratch[kBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_base[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per device and
// kept for the process: it assumes the device keeps one primary context for that time
// (a cudaDeviceReset that destroys it leaves a stale address behind).
int scratch_base(unsigned char** out) {
    int dev = 0;
    int rc = check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (rc) return rc;
    if (dev < 0 || dev >= kMaxDevices) return set_error(SPHGRP_EINVAL, "device ordinal out of range");
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_base[dev]) {
        void* p = nullptr;
        rc = check_cuda(cudaGetSymbolAddress(&p, g_sort_scratch), "cudaGetSymbolAddress");
        if (rc) return rc;
        g_base[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_base[dev];
    return SPHGRP_OK;
}

}  // namespace

extern "C" int sphgrp_sfc_keys_sort_static(int64_t n, const double* pos, uint64_t* keys_out,
                                           int32_t* perm_out, cudaStream_t stream) {
    if (n < 1 || n > kMaxN)
        return set_error(SPHGRP_EINVAL, "n outside [1, SPHGRP_STATIC_SORT_MAX_N] for the static-scratch sort");
    if (!pos || !keys_out || !perm_out) return set_error(SPHGRP_EINVAL, "null positions or outputs");
    unsigned char* base = nullptr;
    int rc = scratch_base(&base);
    if (rc) return rc;
    unsigned* err = reinterpret_cast<unsigned*>(base + kOffErr);
    // the array keeps the previous call's contents: the flag must start at zero
    rc = check_cuda(cudaMemsetAsync(err, 0, sizeof(unsigned), stream), "clear error flag");
    if (rc) return rc;
    rc = sort_keys_scratch(n, pos, keys_out, perm_out, reinterpret_cast<uint64_t*>(base + kOffKeys),
                           reinterpret_cast<int32_t*>(base + kOffPerm), reinterpret_cast<uint32_t*>(base + kOffHist),
                           (int64_t)kHistWords, reinterpret_cast<int32_t*>(base + kOffAux), (int64_t)kAuxWords,
                           err, stream);
    if (rc) return rc;
    unsigned flag = 0;
    rc = check_cuda(cudaMemcpyAsync(&flag, err, sizeof(unsigned), cudaMemcpyDeviceToHost, stream), "read error flag");
    if (rc) return rc;
    rc = check_cuda(cudaStreamSynchronize(stream), "stream");
    if (rc) return rc;
    if (flag & kErrRange) return set_error(SPHGRP_EINVAL, "a position is outside [0,1) or not finite");
    return SPHGRP_OK;
}
