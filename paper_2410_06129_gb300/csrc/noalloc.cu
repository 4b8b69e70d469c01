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

// Sequential 256-byte-aligned carving of the scratch array.
struct Carver {
    unsigned char* base;
    size_t used = 0;
    template <class T>
    T* take(size_t count) {
        used = (used + 255) & ~size_t(255);
        T* p = reinterpret_cast<T*>(base ? base + used : nullptr);
        used += count * sizeof(T);
        return p;
    }
};

}  // namespace

extern "C" pinv_status pinv_apply_noalloc(pinv_plan* p, const void* d_data, void* d_image, int64_t F, int dtype,
                                          void* stream) {
    if (!p) return set_error(PINV_ERR_INVALID_ARG, "null plan");
    if (F < 0) return set_error(PINV_ERR_INVALID_ARG, "n_frames < 0");
    if (dtype != PINV_C64 && dtype != PINV_C128) return set_error(PINV_ERR_INVALID_ARG, "dtype");
    if (!p->built) return set_error(PINV_ERR_NOT_BUILT, "plan not built");
    if (F == 0) return PINV_OK;
    if (!d_data || !d_image) return set_error(PINV_ERR_INVALID_ARG, "null data or image");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = p->N, M = p->M;
    const bool mixed = p->precision != PINV_FP64;
    const bool refine = p->refine_iters > 0;
    const bool stop_rule = refine && p->refine_tol > 0.0;
    const bool dfres = mixed && p->refine_residual == PINV_RESIDUAL_DOUBLE_FLOAT;

    // which scratch buffers this call needs (same roles as pinv_apply's)
    const bool need_d128 = dtype == PINV_C64 && (!mixed || !p->recon || refine);
    const bool need_x128 = dtype == PINV_C64;
    const bool need_u128 = refine || (mixed && !p->recon);
    const bool need_r128 = refine || !p->recon;
    const bool need_d64 = mixed && p->recon && dtype == PINV_C128;
    const bool need_x64 = mixed && (p->recon || (refine && dfres));
    Carver size{nullptr};
    if (need_d128) size.take<double2>((size_t)(F * M));
    if (need_x128) size.take<double2>((size_t)(F * N));
    if (need_u128) size.take<double2>((size_t)(F * M));
    if (need_r128) size.take<double2>((size_t)(F * N));
    if (need_d64) size.take<float2>((size_t)(F * M));
    if (need_x64) size.take<float2>((size_t)(F * N));
    if (stop_rule) size.take<double>((size_t)(2 * F));
    if (size.used > (size_t)PINV_NOALLOC_SCRATCH_BYTES)
        return set_error(PINV_ERR_INVALID_ARG,
                         "pinv_apply_noalloc needs " + std::to_string(size.used) + " B of scratch for " +
                             std::to_string(F) + " frames; its fixed scratch holds " +
                             std::to_string((size_t)PINV_NOALLOC_SCRATCH_BYTES) + " B (use fewer frames per call)");

    unsigned char* base = nullptr;
    pinv_status st = scratch_address(&base);
    if (st != PINV_OK) return st;
    Carver cv{base};
    double2* d128 = need_d128 ? cv.take<double2>((size_t)(F * M)) : nullptr;
    double2* x128 = need_x128 ? cv.take<double2>((size_t)(F * N)) : nullptr;
    double2* u128 = need_u128 ? cv.take<double2>((size_t)(F * M)) : nullptr;
    double2* r128 = need_r128 ? cv.take<double2>((size_t)(F * N)) : nullptr;
    float2* d64 = need_d64 ? cv.take<float2>((size_t)(F * M)) : nullptr;
    float2* x64 = need_x64 ? cv.take<float2>((size_t)(F * N)) : nullptr;
    double* norms = stop_rule ? cv.take<double>((size_t)(2 * F)) : nullptr;

    p->last_refine_iters = 0;
    p->last_refine_resid = 0;
    const double2* D = nullptr;
    if (dtype == PINV_C128) {
        D = (const double2*)d_data;
    } else if (need_d128) {
        CKN(launch_c64_to_c128((const float2*)d_data, d128, F * M, s));
        D = d128;
    }
    double2* X = dtype == PINV_C128 ? (double2*)d_image : x128;

    if (!mixed) {
        if (p->recon) {
            CKN(launch_apply64((const double2*)p->R, N, M, D, F, X, s));
        } else {
            CKN(launch_adjoint64(p->enc, D, F, 0.0, nullptr, r128, s));
            CKN(launch_hemv64(p->Ginv, N, N, r128, F, nullptr, X, s));
        }
    } else if (p->recon) {
        const float2* D32 = (const float2*)d_data;
        if (dtype == PINV_C128) {
            CKN(launch_c128_to_c64((const double2*)d_data, d64, F * M, s));
            D32 = d64;
        }
        CKN(launch_apply32((const float2*)p->R, N, M, D32, F, x64, s));
        CKN(launch_c64_to_c128(x64, X, F * N, s));
    } else {
        CKN(launch_adjoint64(p->enc, D, F, 0.0, nullptr, r128, s));
        CKN(launch_trmv64(p->W, N, r128, F, u128, s));
        CKN(launch_trmv_h64(p->W, N, u128, F, nullptr, X, s));
    }
    if (refine) {
        if (stop_rule) {
            CKN(launch_adjoint64(p->enc, D, F, 0.0, nullptr, r128, s));  // b = E^H d
            CKN(launch_frame_norms(r128, F, N, norms + F, s));
        }
        for (int it = 0; it < p->refine_iters; ++it) {
            if (dfres) {
                CKN(launch_forward_df(p->enc, X, F, D, u128, s));  // u = d - E x
                CKN(launch_adjoint_df(p->enc, u128, F, p->lambda_abs, X, r128, s));
            } else {
                CKN(launch_forward64(p->enc, X, F, D, u128, s));
                CKN(launch_adjoint64(p->enc, u128, F, p->lambda_abs, X, r128, s));
            }
            if (stop_rule) CKN(launch_frame_norms(r128, F, N, norms, s));
            if (dfres) {
                CKN(launch_correct32(p->W32, N, r128, F, x64, X, s));
            } else if (mixed) {
                CKN(launch_trmv64(p->W, N, r128, F, u128, s));
                CKN(launch_trmv_h64(p->W, N, u128, F, X, X, s));
            } else {
                CKN(launch_hemv64(p->Ginv, N, N, r128, F, X, X, s));
            }
            p->last_refine_iters = it + 1;
            if (!stop_rule) continue;
            // per-frame ||r|| / ||E^H d||, read back in fixed-size chunks (no allocation)
            double worst = 0.0, hn[128], hb[128];
            for (int64_t f0 = 0; f0 < F; f0 += 128) {
                const int64_t nf = std::min<int64_t>(128, F - f0);
                CKN(cudaMemcpyAsync(hn, norms + f0, sizeof(double) * nf, cudaMemcpyDeviceToHost, s));
                CKN(cudaMemcpyAsync(hb, norms + F + f0, sizeof(double) * nf, cudaMemcpyDeviceToHost, s));
                CKN(cudaStreamSynchronize(s));
                for (int64_t f = 0; f < nf; ++f) worst = std::max(worst, std::sqrt(hn[f] / std::max(hb[f], 1e-300)));
            }
            p->last_refine_resid = worst;
            if (worst <= p->refine_tol) break;
        }
    }
    if (dtype == PINV_C64) CKN(launch_c128_to_c64(X, (float2*)d_image, F * N, s));
    return PINV_OK;
}
