// pinv_apply_noalloc: image = Recon x data without any device allocation.
//
// Some callers cannot allocate device memory at reconstruction time: a
// scanner's real-time reconstruction loop that runs under a fixed, pre-reserved
// memory budget, or a host application whose device memory is owned by
// another allocator (a framework's caching pool) that must not be bypassed.
// A cudaMalloc there can also stall the whole device while it synchronises,
// which breaks the loop's latency budget. pinv_apply grows plan-owned scratch
// on first use; this variant takes its scratch from one file-scope device
// array of PINV_NOALLOC_SCRATCH_BYTES instead, so it allocates nothing.
//
// The array exists once per GPU that loads the library and lives until the
// process exits. Every call on a device shares it and it keeps the last
// call's contents (nothing in it has to start at zero: every buffer carved
// from it is fully written before it is read). Calls whose GPU work overlaps
// (different streams, or different host threads) race on it.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <string>
#include <vector>

#include "plan_impl.h"

using namespace pinv;

static __device__ __align__(256) unsigned char g_noalloc_scratch[PINV_NOALLOC_SCRATCH_BYTES];

namespace {

std::mutex g_mu;
std::vector<void*> g_addr;  // device index -> device address of g_noalloc_scratch

pinv_status cuda_err(cudaError_t e, const char* where) {
    return set_error(e == cudaErrorMemoryAllocation ? PINV_ERR_OOM : PINV_ERR_CUDA,
                     std::string(where) + ": " + cudaGetErrorString(e));
}
#define CKN(call)                                              \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_err(e_, #call);     \
    } while (0)

// Device address of the scratch array on the current device, looked up once
// per device with that device current. In host code the symbol itself is only
// a host-side stand-in, so kernels must be given this address.
pinv_status scratch_address(unsigned char** out) {
    int dev = 0;
    CKN(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mu);
    if ((int)g_addr.size() <= dev) g_addr.resize(dev + 1, nullptr);
    if (!g_addr[dev]) {
        void* ptr = nullptr;
        CKN(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
        g_addr[dev] = ptr;
    }
    *out = static_cast<unsigned char*>(g_addr[dev]);
    return PINV_OK;
}

}  // namespace

extern "C" pinv_status pinv_apply_noalloc(pinv_plan* p, const void* d_data, void* d_image, int64_t F, int dtype,
                                          void* stream) {
    pinv_status st = apply_check(p, d_data, d_image, F, dtype);
    if (st != PINV_OK || F == 0) return st;
    const size_t need = apply_scratch_layout(p, F, dtype, nullptr, nullptr);
    if (need > (size_t)PINV_NOALLOC_SCRATCH_BYTES)
        return set_error(PINV_ERR_INVALID_ARG,
                         "pinv_apply_noalloc needs " + std::to_string(need) + " B of scratch for " +
                             std::to_string(F) + " frames; its fixed scratch holds " +
                             std::to_string((size_t)PINV_NOALLOC_SCRATCH_BYTES) + " B (use fewer frames per call)");
    unsigned char* base = nullptr;
    if ((st = scratch_address(&base)) != PINV_OK) return st;
    ApplyScratch sc;
    apply_scratch_layout(p, F, dtype, base, &sc);
    return apply_impl(p, d_data, d_image, F, dtype, (cudaStream_t)stream, sc);
}
