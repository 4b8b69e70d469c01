// Definition of the opaque pinv_plan handle and the apply entry points shared
// by the C ABI's translation units.
#pragma once

#include <string>
#include <vector>

#include "pinv_internal.h"

struct pinv_plan;

namespace pinv {
// Record an error message for pinv_last_error() and return the status.
pinv_status set_error(pinv_status st, const std::string& msg);

// Scratch buffers of one apply, carved from one contiguous device region.
struct ApplyScratch {
    double2* d128;  // FP64 copy of c64 data [F][M]
    double2* x128;  // FP64 image for c64 output [F][N]
    double2* u128;  // data-space residual / trmv temporary [F][M]
    double2* r128;  // image-space residual [F][N]
    double2* b128;  // E^H d [F][N] (factor-only and exact-Gram refinement)
    float2* d64;    // c64 copy of c128 data [F][M]
    float2* x64;    // c64 image / FP32 correction temporary [F][N]
    double* norms;  // per-frame squared norms [2F]
    float4* dfw;    // partial sums of the split double-float products
    int* fexp;      // per-frame exponents of the data / image [F] (exact tensor-core products)
    uint8_t* xbd;   // digit tiles of their B operand
    bool xadj;      // E^H d by the exact tensor-core kernel
    bool xfwd;      // the residual's E x and E^H u by the exact tensor-core kernels (plans with B0)
    double2* y128;  // s_c o x [F][C][N] for the exact E x
    float2* apw;    // partials of the tensor-core Recon x data
    float2* cw;     // partials of the tensor-core correction x += W^H (W r)
    DevStatus* sched;  // tile counter of those launches: one per scratch region, since
                       // applies of one plan may run concurrently on several streams
};
// Bytes an apply of F frames of `dtype` needs; with base != nullptr also
// carves the region at base into *sc.
size_t apply_scratch_layout(const pinv_plan* p, int64_t F, int dtype, void* base, ApplyScratch* sc);
// Argument checks shared by the apply entry points.
pinv_status apply_check(const pinv_plan* p, const void* d_data, void* d_image, int64_t F, int dtype);
// image = Recon x data (or G^-1 E^H data) plus refinement on stream s, using
// only the given scratch: no allocation, no host synchronisation unless the
// refinement's stopping rule (refine_tol > 0) is on.
pinv_status apply_impl(pinv_plan* p, const void* d_data, void* d_image, int64_t F, int dtype, cudaStream_t s,
                       const ApplyScratch& sc);

// Build stages, in order (pinv_build runs them all on one stream; the batch
// runs the tensor-core Gram and Recon of several plans as shared launches).
pinv_status reset_status(pinv_plan* p, cudaStream_t s);
pinv_status build_begin(pinv_plan* p, cudaStream_t s);
// main_gram: the plan's own Gram launch (false when a batched launch formed G)
pinv_status build_gram(pinv_plan* p, cudaStream_t s, bool main_gram);
// Cholesky, pivot statistics and the inverse (W = L^-1, or G^-1 for FP64 plans)
pinv_status build_factor(pinv_plan* p, cudaStream_t s, bool events);
pinv_status build_recon(pinv_plan* p, cudaStream_t s);
// kappa_1(G) estimate into the status word (cond.cu); run after the factorisation
pinv_status build_condition(pinv_plan* p, cudaStream_t s);
// status word to pinned host memory
pinv_status build_end(pinv_plan* p, cudaStream_t s);
}  // namespace pinv

struct pinv_plan {
    int ndim = 0;
    int dims[3] = {1, 1, 1};
    double fov[3] = {1, 1, 1};
    int64_t N = 0, Mk = 0, M = 0;
    int C = 1;
    double lambda_abs = 0;
    int eexp = 0;  // every component of E is at most 2^eexp in magnitude
    int precision = PINV_FP64;
    int recon = 1;
    int refine_iters = 0;
    double refine_tol = 0;
    int refine_residual = PINV_RESIDUAL_DOUBLE_FLOAT;
    bool keep_gram = false;
    bool lean = false;  // G and W are build temporaries
    bool built = false;

    std::vector<void*> allocs;
    size_t bytes = 0, bytes_recon = 0;

    pinv::EncodeDev enc{};
    double* traj = nullptr;
    double2* G = nullptr;      // Gram, then L in place (lower); mixed plans: double-float storage (float4)
    double2* Gkeep = nullptr;  // copy of G if requested
    double2* Dinv = nullptr;   // inverses of the diagonal blocks
    double2* Ginv = nullptr;   // full G^-1 (FP64 plans)
    double2* W = nullptr;      // L^-1, lower (mixed plans)
    float2* W32 = nullptr;     // FP32 copy of W (mixed plans)
    void* R = nullptr;         // Recon [N][M], c128 (FP64) or c64 (mixed)
    double2* Ttab = nullptr;   // Toeplitz table of A^H A (TOEPLITZ residual)
    float4* Gx = nullptr;      // exact Gram, double-float [N][N] (TOEPLITZ residual)
    uint8_t* Gd = nullptr;     // its fixed-point digit tiles for the tensor-core residual
    uint8_t* Ad = nullptr;     // digit tiles of conj(A) for the exact E^H d (mixed, not lean)
    uint8_t* Af = nullptr;     // digit tiles of A for the exact E x (mixed with B0, not lean)
    int* eG = nullptr;         // |G| <= 2^eG (device)
    pinv::DevStatus* st = nullptr;        // device status word
    pinv::DevStatus* st_host = nullptr;   // pinned copy, written at the end of each build
    // mixed plans: the triangular inverse runs beside the Cholesky on its own stream,
    // one panel behind (its tile counter and timeout record; one event per panel)
    pinv::DevStatus* st_inv = nullptr;
    cudaStream_t s_inv = nullptr;
    // the Cholesky chain's stream, at the device's highest priority: its small
    // launches get SMs ahead of the inverse's tiles (and of other work)
    cudaStream_t s_chol = nullptr;
    // the Cholesky's trailing updates beyond the next panel run beside the chain on
    // this stream, with their own tile counter and timeout record (lookahead)
    cudaStream_t s_trail = nullptr;
    pinv::DevStatus* st_trail = nullptr;
    cudaEvent_t ev_tab = nullptr, ev_trail = nullptr;
    // inside a panel, the solves and updates beyond the next diagonal block run on
    // this stream (high priority) beside that block (block lookahead)
    cudaStream_t s_pnl = nullptr;
    cudaEvent_t ev_next = nullptr, ev_side = nullptr;
    // the refinement's exact Gram and digit tables, at the device's lowest stream
    // priority beside the Cholesky and the inverse (only applies and the condition
    // check read them; x_pending: the build has not waited for them yet)
    cudaStream_t s_x = nullptr;
    cudaEvent_t ev_xjoin = nullptr;
    bool x_pending = false;
    std::vector<cudaEvent_t> ev_panel;
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_xfork = nullptr, ev_chol = nullptr;

    // pinv_apply's scratch region, grown on demand
    void* scratch_buf = nullptr;
    size_t scratch_bytes = 0;

    cudaEvent_t ev[10] = {};  // build stages 0-5; 6-7 around the Gram kernels; 8-9 around the condition estimate
    int last_refine_iters = 0;
    double last_refine_resid = 0;
    double last_refine_bound = 0;
    int info = -1;

    int slices() const { return precision == PINV_MIXED_BF16X6 ? 3 : 2; }
    // a lean mixed plan keeps only W32 when its residual does not use the FP64 W
    bool lean_w() const { return lean && precision != PINV_FP64 && refine_residual != PINV_RESIDUAL_FP64; }
    // a lean TOEPLITZ plan keeps only the digit tiles of its exact Gram
    bool lean_gx() const { return lean && refine_residual == PINV_RESIDUAL_TOEPLITZ && precision != PINV_FP64; }

    // Free the stored Recon; later applies take the factor-only path (x from
    // W^H W E^H d, then the same refinement). Returns the bytes released.
    size_t drop_recon() {
        if (!recon || !R) return 0;
        cudaDeviceSynchronize();  // applies on any stream may still read it
        cudaFreeAsync(R, 0);
        cudaStreamSynchronize(0);
        for (auto& a : allocs)
            if (a == R) a = nullptr;
        const size_t b = bytes_recon;
        bytes -= b;
        bytes_recon = 0;
        R = nullptr;
        recon = 0;
        return b;
    }

    // Plan memory comes from the library's pool (kept between plans, so creating a
    // plan again does not map GBs of memory again), ordered on the legacy stream and
    // complete before this returns, so any stream may use it.
    pinv_status alloc(void** p, size_t n, const char* what) {
        if (n == 0) n = 16;
        cudaError_t e = pinv::work_alloc(p, n, 0);
        if (e == cudaSuccess) e = cudaStreamSynchronize(0);
        if (e != cudaSuccess) {
            *p = nullptr;
            return pinv::set_error(e == cudaErrorMemoryAllocation ? PINV_ERR_OOM : PINV_ERR_CUDA,
                                   std::string("alloc(") + what + ", " + std::to_string(n) + " B): " +
                                       cudaGetErrorString(e));
        }
        allocs.push_back(*p);
        bytes += n;
        return PINV_OK;
    }
    ~pinv_plan() {
        cudaDeviceSynchronize();  // nothing of this plan may still run
        if (scratch_buf) cudaFreeAsync(scratch_buf, 0);
        for (void* p : allocs)
            if (p) cudaFreeAsync(p, 0);
        cudaStreamSynchronize(0);
        if (st_host) cudaFreeHost(st_host);
        for (auto& e : ev)
            if (e) cudaEventDestroy(e);
        for (auto& e : ev_panel)
            if (e) cudaEventDestroy(e);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (ev_xfork) cudaEventDestroy(ev_xfork);
        if (ev_chol) cudaEventDestroy(ev_chol);
        if (ev_tab) cudaEventDestroy(ev_tab);
        if (ev_trail) cudaEventDestroy(ev_trail);
        if (ev_next) cudaEventDestroy(ev_next);
        if (ev_side) cudaEventDestroy(ev_side);
        if (s_pnl) cudaStreamDestroy(s_pnl);
        if (ev_xjoin) cudaEventDestroy(ev_xjoin);
        if (s_x) cudaStreamDestroy(s_x);
        if (s_trail) cudaStreamDestroy(s_trail);
        if (s_inv) cudaStreamDestroy(s_inv);
        if (s_chol) cudaStreamDestroy(s_chol);
    }
};
