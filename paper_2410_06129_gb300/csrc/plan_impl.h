// Definition of the opaque pinv_plan handle, shared by the C ABI's translation units.
#pragma once

#include <string>
#include <vector>

#include "pinv_internal.h"

namespace pinv {
// Record an error message for pinv_last_error() and return the status.
pinv_status set_error(pinv_status st, const std::string& msg);
}  // namespace pinv

struct pinv_plan {
    int ndim = 0;
    int dims[3] = {1, 1, 1};
    double fov[3] = {1, 1, 1};
    int64_t N = 0, Mk = 0, M = 0;
    int C = 1;
    double lambda_abs = 0;
    int precision = PINV_FP64;
    int recon = 1;
    int refine_iters = 0;
    double refine_tol = 0;
    int refine_residual = PINV_RESIDUAL_DOUBLE_FLOAT;
    bool keep_gram = false;
    bool built = false;

    std::vector<void*> allocs;
    size_t bytes = 0, bytes_recon = 0;

    pinv::EncodeDev enc{};
    double* traj = nullptr;
    double2* G = nullptr;      // Gram, then L in place (lower)
    double2* Gkeep = nullptr;  // copy of G if requested
    double2* Dinv = nullptr;   // inverses of the diagonal blocks
    double2* Ginv = nullptr;   // full G^-1 (FP64 plans)
    double2* W = nullptr;      // L^-1, lower (mixed plans)
    float2* W32 = nullptr;     // FP32 copy of W (mixed plans)
    void* R = nullptr;         // Recon [N][M], c128 (FP64) or c64 (mixed)
    pinv::DevStatus* st = nullptr;

    // apply scratch (grown on demand)
    int64_t scratch_frames = 0;
    double2 *d128 = nullptr, *x128 = nullptr, *u128 = nullptr, *r128 = nullptr;
    float2 *d64 = nullptr, *x64 = nullptr;
    double* norms = nullptr;
    std::vector<void*> scratch;

    cudaEvent_t ev[6] = {};
    int last_refine_iters = 0;
    double last_refine_resid = 0;
    int info = -1;

    pinv_status alloc(void** p, size_t n, const char* what) {
        if (n == 0) n = 16;
        cudaError_t e = cudaMalloc(p, n);
        if (e != cudaSuccess) {
            *p = nullptr;
            return pinv::set_error(e == cudaErrorMemoryAllocation ? PINV_ERR_OOM : PINV_ERR_CUDA,
                        std::string("cudaMalloc(") + what + ", " + std::to_string(n) + " B): " +
                            cudaGetErrorString(e));
        }
        allocs.push_back(*p);
        bytes += n;
        return PINV_OK;
    }
    ~pinv_plan() {
        for (void* p : scratch) cudaFree(p);
        for (void* p : allocs) cudaFree(p);
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
    }
};

