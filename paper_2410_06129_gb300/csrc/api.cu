// C ABI of the Pinv-Recon library: plan creation, build, apply, export.
//
// A plan owns the device copies of its encoding description (trajectory
// tables, voxel coordinates, coil maps, B0 table), the factor L (stored over
// G), G^-1 and optionally Recon = E^+. Building enqueues the stages on the
// caller's stream; nothing blocks until pinv_plan_sync.
#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "plan_impl.h"

using namespace pinv;

namespace {
thread_local std::string g_err;

pinv_status fail(pinv_status st, const std::string& msg) {
    g_err = msg;
    return st;
}
pinv_status cuda_fail(cudaError_t e, const char* where) {
    g_err = std::string(where) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PINV_ERR_OOM : PINV_ERR_CUDA;
}
#define CK(call)                                              \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(e_, #call);   \
    } while (0)
}  // namespace

namespace pinv {
std::atomic<unsigned long long> g_launches{0};
pinv_status set_error(pinv_status st, const std::string& msg) { return fail(st, msg); }
static std::atomic<long long> g_wait_limit{0};
long long wait_limit_setting() { return g_wait_limit.load(); }
}

namespace pinv {

pinv_status reset_status(pinv_plan* p, cudaStream_t s) {
    CK(launch_reset_status(p->st, s));
    if (p->st_inv) CK(launch_reset_status(p->st_inv, s));
    if (p->st_trail) CK(launch_reset_status(p->st_trail, s));
    return PINV_OK;
}

pinv_status build_begin(pinv_plan* p, cudaStream_t s) {
    p->built = false;
    pinv_status rs = reset_status(p, s);
    if (rs != PINV_OK) return rs;
    if (p->lean) {  // stream-ordered temporaries, released by build_end
        CK(work_alloc((void**)&p->G, sizeof(double2) * p->N * p->N, s));
        if (p->lean_w()) CK(work_alloc((void**)&p->W, sizeof(double2) * p->N * p->N, s));
        if (p->lean_gx()) CK(work_alloc((void**)&p->Gx, sizeof(float4) * p->N * p->N, s));
    }
    if (p->keep_gram && !p->Gkeep) {
        pinv_status st = p->alloc((void**)&p->Gkeep, sizeof(double2) * p->N * p->N, "Gkeep");
        if (st != PINV_OK) return st;
    }
    return PINV_OK;
}

pinv_status build_gram(pinv_plan* p, cudaStream_t s, bool main_gram) {
    const int64_t N = p->N, ld = p->N;
    CK(cudaEventRecord(p->ev[6], s));
    if (main_gram) {
        if (p->precision == PINV_FP64) {
            CK(launch_gram64(p->enc, p->lambda_abs, p->G, ld, s));
        } else {
            // bulk-fed Gram from a split operand table; without room for the table
            // (or with PINV_GRAM_BULK=0) the kernel generates its operands itself
            void* work = nullptr;
            const char* env = std::getenv("PINV_GRAM_BULK");
            const bool bulk = !(env && std::strcmp(env, "0") == 0);
            if (bulk && work_alloc(&work, gram_bulk_bytes(p->enc, p->slices()), s) == cudaSuccess) {
                CK(launch_gram_bulk(p->enc, p->lambda_abs, p->slices(), (float4*)p->G, ld, work, p->st, s));
                CK(cudaFreeAsync(work, s));
            } else {
                cudaGetLastError();
                CK(launch_gram_tc(p->enc, p->lambda_abs, p->slices(), (float4*)p->G, ld, p->st, s));
            }
        }
    }
    CK(cudaEventRecord(p->ev[7], s));
    // mixed plans hold G in double-float storage (float4 per entry) until it is factored
    const bool gdf = p->precision != PINV_FP64;
    if (p->Gkeep) {
        if (gdf)
            CK(launch_df_to_f64((const float4*)p->G, N * N, p->Gkeep, s));
        else
            CK(cudaMemcpyAsync(p->Gkeep, p->G, sizeof(double2) * N * N, cudaMemcpyDeviceToDevice, s));
    }
    // ||G||_1 for the condition estimate: from the exact Gram where the plan forms
    // one (below, beside the Cholesky), else from G before the Cholesky overwrites it
    if (!p->Gx) CK(launch_gram_norm1(gdf ? nullptr : p->G, gdf ? (const float4*)p->G : nullptr, nullptr, N, ld, p->st, s));
    if (p->Gx) {
        // exact Gram for the refinement residual (Toeplitz table, then coil products,
        // then its digit tiles). Only applies and the condition check read it, so mixed
        // plans form it on their lowest-priority stream beside the Cholesky and the
        // inverse, in the SMs their launches leave free (build_factor joins that stream).
        cudaStream_t sx = s;
        if (p->s_x) {
            CK(cudaEventRecord(p->ev_xfork, s));
            CK(cudaStreamWaitEvent(p->s_x, p->ev_xfork, 0));
            sx = p->s_x;
        }
        float4* work = nullptr;
        CK(work_alloc((void**)&work, toeplitz_work_bytes(p->enc), sx));
        CK(launch_toeplitz(p->enc, work, p->Ttab, sx));
        CK(cudaFreeAsync(work, sx));
        CK(launch_gram_exact(p->enc, p->Ttab, p->lambda_abs, p->Gx, sx));
        CK(launch_gram_norm1(nullptr, nullptr, p->Gx, N, N, p->st, sx));
        if (p->Gd) CK(launch_gram_digits(p->Gx, N, p->eG, p->Gd, sx));
        if (p->Ad) CK(launch_adj_digits(p->enc, p->Ad, sx));
        if (sx != s) {
            CK(cudaEventRecord(p->ev_xjoin, sx));
            p->x_pending = true;
        }
    } else if (p->Ad || p->Af) {
        // plans with B0: the digit tables of conj(A) and A for the exact products of
        // the refinement, formed beside the Cholesky (build_factor joins that stream)
        cudaStream_t sx = s;
        if (p->s_x) {
            CK(cudaEventRecord(p->ev_xfork, s));
            CK(cudaStreamWaitEvent(p->s_x, p->ev_xfork, 0));
            sx = p->s_x;
        }
        if (p->Ad) CK(launch_adj_digits(p->enc, p->Ad, sx));
        if (p->Af) CK(launch_fwd_digits(p->enc, p->Af, sx));
        if (sx != s) {
            CK(cudaEventRecord(p->ev_xjoin, sx));
            p->x_pending = true;
        }
    }
    return PINV_OK;
}

// ------------------------------------------------------------------ build temporaries
// Builds allocate several GB of stream-ordered temporaries (operand tables, the
// FP32 factor). They come from one pool per device that keeps its memory between
// builds, so a build does not map it again; when the last plan is destroyed the
// pool is trimmed to a kept size (8 GiB, or PINV_POOL_KEEP_MB), so a program that
// creates, builds and destroys plans one after another does not unmap and map the
// same GBs each time (about 7 ms per cycle at the 64x64 SENSE workload). (The
// device's default pool returns its memory at every synchronisation.)
namespace {
std::mutex g_pool_mu;
cudaMemPool_t g_pools[64] = {};
std::atomic<int> g_live_plans{0};
cudaMemPool_t build_pool() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        g_pools[dev] = pool;
    }
    return g_pools[dev];
}
}  // namespace

cudaError_t work_alloc(void** ptr, size_t bytes, cudaStream_t s) {
    cudaMemPool_t pool = build_pool();
    return pool ? cudaMallocFromPoolAsync(ptr, bytes, pool, s) : cudaMallocAsync(ptr, bytes, s);
}

pinv_status build_factor(pinv_plan* p, cudaStream_t s, bool events) {
    const int64_t N = p->N, ld = p->N;
    if (p->precision != PINV_FP64) {
        // FP64 diagonal panels, tensor-core panel solves / trailing updates,
        // then the triangular inverse W = L^-1 on tensor cores
        const int64_t nblk = (N + 63) / 64;
        float2 *L32 = nullptr, *D32 = nullptr;
        CK(work_alloc((void**)&L32, sizeof(float2) * N * N, s));
        CK(work_alloc((void**)&D32, sizeof(float2) * nblk * 64 * 64, s));
        // operand tables of the bulk-fed panel updates, one region per stream
        // (PINV_CHOL_BULK=0: generated operands)
        void* tab = nullptr;
        const size_t tb = factor_table_bytes(N, p->slices());
        const char* env = std::getenv("PINV_CHOL_BULK");
        if (!(env && std::strcmp(env, "0") == 0) && work_alloc(&tab, 2 * tb, s) != cudaSuccess) {
            cudaGetLastError();
            tab = nullptr;
        }
        void* tab_inv = tab ? (void*)((uint8_t*)tab + tb) : nullptr;
        // W = L^-1 on the plan's second stream, one 256-wide panel behind the Cholesky
        // (it reads only the panel's L32 columns and diagonal inverses, final once the
        // panel's solves are done); the Cholesky chain leaves most SMs idle
        CK(cudaEventRecord(p->ev_fork, s));
        // the chain on the high-priority stream (PINV_CHOL_HI=0: on s)
        const char* hi = std::getenv("PINV_CHOL_HI");
        cudaStream_t sc = (p->s_chol && !(hi && std::strcmp(hi, "0") == 0)) ? p->s_chol : s;
        if (sc != s) CK(cudaStreamWaitEvent(sc, p->ev_fork, 0));
        // (the FP64 diagonal inverses are not needed: the inverse reads the FP32 ones)
        const TrailLookahead la{p->s_trail, p->st_trail, p->ev_tab, p->ev_trail, p->s_pnl, p->ev_next, p->ev_side};
        CK(cudaStreamWaitEvent(p->s_trail, p->ev_fork, 0));
        CK(cudaStreamWaitEvent(p->s_pnl, p->ev_fork, 0));
        CK(launch_potrf_tc((float4*)p->G, N, ld, nullptr, D32, L32, p->slices(), p->st, sc, tab, p->ev_panel.data(),
                           &la));
        CK(launch_merge_timeout(p->st, p->st_trail, sc));
        CK(launch_pivot_stats_df((const float4*)p->G, N, ld, p->st, sc));
        if (events) CK(cudaEventRecord(p->ev[3], sc));
        CK(cudaStreamWaitEvent(p->s_inv, p->ev_fork, 0));
        CK(launch_trtri_tc(L32, N, D32, (float4*)p->W, p->W32, p->slices(), p->st_inv, p->s_inv, tab_inv,
                           p->ev_panel.data()));
        if (sc != s) {
            CK(cudaEventRecord(p->ev_chol, sc));
            CK(cudaStreamWaitEvent(p->s_inv, p->ev_chol, 0));  // st is read below
        }
        CK(launch_merge_timeout(p->st, p->st_inv, p->s_inv));
        CK(cudaEventRecord(p->ev_join, p->s_inv));
        CK(cudaStreamWaitEvent(s, p->ev_join, 0));
        if (tab) CK(cudaFreeAsync(tab, s));
        CK(cudaFreeAsync(D32, s));
        CK(cudaFreeAsync(L32, s));
    } else {
        CK(launch_potrf64(p->G, N, ld, p->Dinv, p->st, s));
        CK(launch_pivot_stats(p->G, N, ld, p->st, s));
        if (events) CK(cudaEventRecord(p->ev[3], s));
        double2* W = nullptr;
        CK(work_alloc((void**)&W, sizeof(double2) * N * N, s));
        CK(launch_trtri64(p->G, N, ld, p->Dinv, W, s));
        CK(launch_lauum64(W, N, ld, p->Ginv, s));
        CK(cudaFreeAsync(W, s));
    }
    if (p->x_pending) {  // the exact Gram and digit tables formed beside the factor
        CK(cudaStreamWaitEvent(s, p->ev_xjoin, 0));
        p->x_pending = false;
    }
    // the lambda / condition check: kappa_1(G) from the factor (Section 2.1, 2.2)
    if (events) CK(cudaEventRecord(p->ev[8], s));
    pinv_status cs = build_condition(p, s);
    if (cs != PINV_OK) return cs;
    if (events) CK(cudaEventRecord(p->ev[9], s));
    return PINV_OK;
}

pinv_status build_recon(pinv_plan* p, cudaStream_t s) {
    if (!p->recon) return PINV_OK;
    const int64_t N = p->N;
    if (p->precision != PINV_FP64) {
        // Recon = W^H (W E^H) (Eq. 8): bulk-fed from split operand tables, or (no
        // room for the tables, or PINV_RECON_BULK=0) with operands generated in the
        // kernels through an [N][M] c64 intermediate
        void* work = nullptr;
        const char* env = std::getenv("PINV_RECON_BULK");
        const bool bulk = !(env && std::strcmp(env, "0") == 0);
        if (bulk && work_alloc(&work, recon_bulk_bytes(p->enc, p->slices()), s) == cudaSuccess) {
            CK(launch_recon_bulk(p->enc, p->W32, p->slices(), (float2*)p->R, work, p->st, s));
            CK(cudaFreeAsync(work, s));
        } else {
            cudaGetLastError();
            float2 *T = nullptr, *WT32 = nullptr;
            CK(work_alloc((void**)&T, sizeof(float2) * N * p->M, s));
            CK(work_alloc((void**)&WT32, sizeof(float2) * N * N, s));
            CK(launch_transpose32(p->W32, N, N, WT32, N, s));
            CK(launch_recon_tc(p->enc, p->W32, WT32, T, p->slices(), (float2*)p->R, p->st, s));
            CK(cudaFreeAsync(WT32, s));
            CK(cudaFreeAsync(T, s));
        }
    } else {
        CK(launch_recon64(p->enc, p->Ginv, N, (double2*)p->R, s));
    }
    return PINV_OK;
}

pinv_status build_end(pinv_plan* p, cudaStream_t s) {
    CK(cudaMemcpyAsync(p->st_host, p->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    if (p->lean) {
        CK(cudaFreeAsync(p->G, s));
        p->G = nullptr;
        if (p->lean_w()) {
            CK(cudaFreeAsync(p->W, s));
            p->W = nullptr;
        }
        if (p->lean_gx()) {
            CK(cudaFreeAsync(p->Gx, s));
            p->Gx = nullptr;
        }
    }
    return PINV_OK;
}

}  // namespace pinv

extern "C" {

int pinv_version(void) { return 100; }

pinv_status pinv_set_wait_limit(int64_t cycles) {
    if (cycles < 0) return fail(PINV_ERR_INVALID_ARG, "wait limit must be >= 0");
    g_wait_limit.store((long long)cycles);
    return PINV_OK;
}

unsigned long long pinv_kernel_launches(void) { return g_launches.load(); }

const char* pinv_last_error(void) { return g_err.c_str(); }

pinv_status pinv_plan_create(const pinv_plan_desc* d, void* stream, pinv_plan** out) {
    g_err.clear();
    if (!d || !out) return fail(PINV_ERR_INVALID_ARG, "null descriptor or output pointer");
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    if (d->ndim < 1 || d->ndim > 3) return fail(PINV_ERR_INVALID_ARG, "ndim must be 1, 2 or 3");
    int64_t grid = 1;
    for (int i = 0; i < d->ndim; ++i) {
        if (d->dims[i] < 1) return fail(PINV_ERR_INVALID_ARG, "dims must be >= 1");
        grid *= d->dims[i];
    }
    if (d->n_vox < 1) return fail(PINV_ERR_INVALID_ARG, "n_vox must be >= 1");
    if (!d->voxel_index && d->n_vox != grid)
        return fail(PINV_ERR_INVALID_ARG, "n_vox must equal prod(dims) without voxel_index");
    if (d->n_samples < 1 || !d->traj) return fail(PINV_ERR_INVALID_ARG, "need n_samples >= 1 and traj");
    if (d->n_coils < 1) return fail(PINV_ERR_INVALID_ARG, "n_coils must be >= 1");
    if (d->n_coils > 1 && !d->coil_maps) return fail(PINV_ERR_INVALID_ARG, "n_coils > 1 needs coil_maps");
    if (d->b0_hz && !d->times) return fail(PINV_ERR_INVALID_ARG, "b0_hz needs times");
    if (d->precision < PINV_FP64 || d->precision > PINV_MIXED_BF16X6)
        return fail(PINV_ERR_INVALID_ARG, "unknown precision");
    if (d->precision != PINV_FP64 && !tc_available())
        return fail(PINV_ERR_UNSUPPORTED, "mixed precision needs the tcgen05 kernels (sm_103a)");
    if (d->lambda_mode != PINV_LAMBDA_ABS && d->lambda_mode != PINV_LAMBDA_REL_MEAN_DIAG)
        return fail(PINV_ERR_INVALID_ARG, "unknown lambda_mode");
    if (!(d->lambda >= 0.0) || !std::isfinite(d->lambda))
        return fail(PINV_ERR_INVALID_ARG, "lambda must be finite and >= 0");
    if (d->refine_max_iters < 0) return fail(PINV_ERR_INVALID_ARG, "refine_max_iters must be >= 0");
    for (int64_t i = 0; i < d->n_samples * d->ndim; ++i)
        if (!std::isfinite(d->traj[i])) return fail(PINV_ERR_INVALID_ARG, "non-finite trajectory");

    auto* p = new pinv_plan();
    auto cleanup = [&](pinv_status st) { delete p; return st; };
    p->ndim = d->ndim;
    for (int i = 0; i < 3; ++i) {
        p->dims[i] = i < d->ndim ? d->dims[i] : 1;
        p->fov[i] = i < d->ndim ? d->fov[i] : 1.0;
    }
    p->N = d->n_vox;
    p->Mk = d->n_samples;
    p->C = d->n_coils;
    p->M = p->Mk * p->C;
    p->precision = d->precision;
    p->refine_iters = d->refine_max_iters;
    p->refine_tol = d->refine_tol;
    if (d->refine_residual != PINV_RESIDUAL_DOUBLE_FLOAT && d->refine_residual != PINV_RESIDUAL_FP64 &&
        d->refine_residual != PINV_RESIDUAL_TOEPLITZ)
        return cleanup(fail(PINV_ERR_INVALID_ARG, "unknown refine_residual"));
    if (d->refine_residual == PINV_RESIDUAL_TOEPLITZ && d->b0_hz && p->precision != PINV_FP64)
        return cleanup(fail(PINV_ERR_UNSUPPORTED, "the Toeplitz residual needs a plan without B0"));
    p->refine_residual = p->precision == PINV_FP64 ? PINV_RESIDUAL_FP64 : d->refine_residual;
    const bool toeplitz = p->refine_residual == PINV_RESIDUAL_TOEPLITZ;
    p->lean = d->lean != 0;

    // voxel grid coordinates
    std::vector<int> ijk(3 * p->N);
    for (int64_t n = 0; n < p->N; ++n) {
        int64_t g = d->voxel_index ? d->voxel_index[n] : n;
        if (g < 0 || g >= grid) return cleanup(fail(PINV_ERR_INVALID_ARG, "voxel_index out of range"));
        ijk[3 * n + 0] = (int)(g % p->dims[0]);
        ijk[3 * n + 1] = (int)((g / p->dims[0]) % p->dims[1]);
        ijk[3 * n + 2] = (int)(g / ((int64_t)p->dims[0] * p->dims[1]));
    }
    // lambda: trace(E^H E) / N = M_k * mean_n sum_c |s_c(n)|^2 since |A| = 1
    double sos = (double)p->N, smax = 1.0;
    if (d->coil_maps) {
        sos = 0.0;
        smax = 0.0;
        for (int64_t i = 0; i < 2 * p->N * p->C; ++i) {
            double v = d->coil_maps[i];
            if (!std::isfinite(v)) return cleanup(fail(PINV_ERR_INVALID_ARG, "non-finite coil map"));
            sos += v * v;
        }
        for (int64_t i = 0; i < p->N * p->C; ++i)
            smax = std::max(smax, std::hypot(d->coil_maps[2 * i], d->coil_maps[2 * i + 1]));
    }
    // |E| = |s_c(n)| (|A| = 1): the exponent bounding every component of E
    {
        int ex = 0;
        const double mant = smax > 0.0 ? std::frexp(smax * (1.0 + 1e-12), &ex) : 0.0;
        p->eexp = smax > 0.0 ? (mant == 0.5 ? ex - 1 : ex) : 0;
    }
    p->lambda_abs = d->lambda_mode == PINV_LAMBDA_ABS ? d->lambda
                                                      : d->lambda * (double)p->Mk * sos / (double)p->N;
    // B0: distinct sample times
    std::vector<double> tuniq;
    std::vector<int> tidx;
    if (d->b0_hz) {
        std::map<double, int> idx;
        for (int64_t m = 0; m < p->Mk; ++m) idx.emplace(d->times[m], 0);
        int u = 0;
        for (auto& kv : idx) { kv.second = u++; tuniq.push_back(kv.first); }
        tidx.resize(p->Mk);
        for (int64_t m = 0; m < p->Mk; ++m) tidx[m] = idx[d->times[m]];
        double tab_bytes = (double)tuniq.size() * (double)p->N * 24.0;
        if (tab_bytes > 16e9)
            return cleanup(fail(PINV_ERR_UNSUPPORTED, "too many distinct sample times for the B0 table"));
    }

    pinv_status st;
#define AL(ptr, n, what)                                               \
    do {                                                               \
        st = p->alloc((void**)&(ptr), (size_t)(n), what);             \
        if (st != PINV_OK) return cleanup(st);                        \
    } while (0)
#define CKC(call)                                                      \
    do {                                                               \
        cudaError_t e_ = (call);                                       \
        if (e_ != cudaSuccess) return cleanup(cuda_fail(e_, #call));  \
    } while (0)

    EncodeDev& e = p->enc;
    e.N = p->N;
    e.Mk = p->Mk;
    e.C = p->C;
    e.nx = p->dims[0];
    e.ny = p->dims[1];
    e.nz = p->dims[2];
    e.full_grid = d->voxel_index ? 0 : 1;
    AL(p->traj, sizeof(double) * p->Mk * p->ndim, "traj");
    double2 *ex, *ey, *ez;
    float2 *ex32, *ey32, *ez32;
    AL(ex, sizeof(double2) * p->Mk * e.nx, "ex");
    AL(ey, sizeof(double2) * p->Mk * e.ny, "ey");
    AL(ez, sizeof(double2) * p->Mk * e.nz, "ez");
    AL(ex32, sizeof(float2) * p->Mk * e.nx, "ex32");
    AL(ey32, sizeof(float2) * p->Mk * e.ny, "ey32");
    AL(ez32, sizeof(float2) * p->Mk * e.nz, "ez32");
    int* vox;
    AL(vox, sizeof(int) * 3 * p->N, "vox");
    AL(p->st, sizeof(DevStatus), "status");
    CKC(cudaMallocHost((void**)&p->st_host, sizeof(DevStatus)));
    *p->st_host = DevStatus{};
    p->st_host->not_pd_pivot = INT_MAX;
    e.ex = ex; e.ey = ey; e.ez = ez;
    e.ex32 = ex32; e.ey32 = ey32; e.ez32 = ez32;
    e.vox_ijk = vox;
    // inputs travel through pageable memory; the stream sync below makes the
    // host arrays free to reuse when this call returns
    CKC(cudaMemcpyAsync(p->traj, d->traj, sizeof(double) * p->Mk * p->ndim, cudaMemcpyHostToDevice, s));
    CKC(cudaMemcpyAsync(vox, ijk.data(), sizeof(int) * 3 * p->N, cudaMemcpyHostToDevice, s));
    if (d->coil_maps) {
        double2* cm;
        float2* cm32;
        AL(cm, sizeof(double2) * p->C * p->N, "coils");
        AL(cm32, sizeof(float2) * p->C * p->N, "coils32");
        CKC(cudaMemcpyAsync(cm, d->coil_maps, sizeof(double2) * p->C * p->N, cudaMemcpyHostToDevice, s));
        CKC(launch_to_f32(cm, cm32, p->C * p->N, s));
        e.coils = cm;
        e.coils32 = cm32;
    }
    if (d->b0_hz) {
        int T = (int)tuniq.size();
        double *b0, *tu;
        double2* tab;
        float2* tab32;
        int* ti;
        AL(b0, sizeof(double) * p->N, "b0");
        AL(tu, sizeof(double) * T, "tuniq");
        AL(tab, sizeof(double2) * T * p->N, "b0tab");
        AL(tab32, sizeof(float2) * T * p->N, "b0tab32");
        AL(ti, sizeof(int) * p->Mk, "tidx");
        CKC(cudaMemcpyAsync(b0, d->b0_hz, sizeof(double) * p->N, cudaMemcpyHostToDevice, s));
        CKC(cudaMemcpyAsync(tu, tuniq.data(), sizeof(double) * T, cudaMemcpyHostToDevice, s));
        CKC(cudaMemcpyAsync(ti, tidx.data(), sizeof(int) * p->Mk, cudaMemcpyHostToDevice, s));
        CKC(launch_b0_table(b0, tu, T, p->N, tab, tab32, s));
        e.b0tab = tab;
        e.b0tab32 = tab32;
        e.tidx = ti;
    }
    CKC(launch_tables(p->traj, p->ndim, p->Mk, p->dims, p->fov, ex, ey, ez, ex32, ey32, ez32, s));
    if (p->precision != PINV_FP64) {
        // sample-contiguous copies of the FP32 tables for the tensor-core producers
        const int64_t Mkp = (p->Mk + 7) / 8 * 8;
        float2 *xt, *yt, *zt;
        AL(xt, sizeof(float2) * Mkp * e.nx, "ext32");
        AL(yt, sizeof(float2) * Mkp * e.ny, "eyt32");
        AL(zt, sizeof(float2) * Mkp * e.nz, "ezt32");
        CKC(launch_transpose32(ex32, p->Mk, e.nx, xt, Mkp, s));
        CKC(launch_transpose32(ey32, p->Mk, e.ny, yt, Mkp, s));
        CKC(launch_transpose32(ez32, p->Mk, e.nz, zt, Mkp, s));
        e.ext32 = xt;
        e.eyt32 = yt;
        e.ezt32 = zt;
        e.Mkp = Mkp;
        if (e.b0tab32) {
            const int T = (int)tuniq.size();
            float2* bt;
            AL(bt, sizeof(float2) * T * p->N, "b0t32");
            CKC(launch_transpose32(e.b0tab32, T, p->N, bt, T, s));
            e.b0t32 = bt;
            e.T = T;
        }
    }
    if (p->refine_residual == PINV_RESIDUAL_DOUBLE_FLOAT || toeplitz) {
        // double-float copies of the tables for the refinement residual / E^H d
        float4 *xdf, *ydf, *zdf;
        AL(xdf, sizeof(float4) * p->Mk * e.nx, "exdf");
        AL(ydf, sizeof(float4) * p->Mk * e.ny, "eydf");
        AL(zdf, sizeof(float4) * p->Mk * e.nz, "ezdf");
        CKC(launch_to_df(ex, xdf, p->Mk * e.nx, s));
        CKC(launch_to_df(ey, ydf, p->Mk * e.ny, s));
        CKC(launch_to_df(ez, zdf, p->Mk * e.nz, s));
        e.exdf = xdf;
        e.eydf = ydf;
        e.ezdf = zdf;
        if (!d->b0_hz && e.Mkp > 0) {
            // sample-contiguous copies for the exact tensor-core E^H d
            float4 *xt, *yt, *zt;
            AL(xt, sizeof(float4) * e.Mkp * e.nx, "extdf");
            AL(yt, sizeof(float4) * e.Mkp * e.ny, "eytdf");
            AL(zt, sizeof(float4) * e.Mkp * e.nz, "eztdf");
            CKC(launch_transpose_df(xdf, p->Mk, e.nx, xt, e.Mkp, s));
            CKC(launch_transpose_df(ydf, p->Mk, e.ny, yt, e.Mkp, s));
            CKC(launch_transpose_df(zdf, p->Mk, e.nz, zt, e.Mkp, s));
            e.extdf = xt;
            e.eytdf = yt;
            e.eztdf = zt;
        }
        if (e.b0tab) {
            const int64_t nt = (int64_t)tuniq.size() * p->N;
            float4* bdf;
            AL(bdf, sizeof(float4) * nt, "b0df");
            CKC(launch_to_df(e.b0tab, bdf, nt, s));
            e.b0df = bdf;
        }
        if (e.coils) {
            float4* cdf;
            AL(cdf, sizeof(float4) * p->C * p->N, "coilsdf");
            CKC(launch_to_df(e.coils, cdf, p->C * p->N, s));
            e.coilsdf = cdf;
        }
    }
    // factor storage
    int64_t nblk = (p->N + 63) / 64;
    if (!p->lean) AL(p->G, sizeof(double2) * p->N * p->N, "G");
    AL(p->Dinv, sizeof(double2) * nblk * 64 * 64, "Dinv");
    if (p->precision == PINV_FP64) AL(p->Ginv, sizeof(double2) * p->N * p->N, "Ginv");
    else {
        if (!p->lean_w()) AL(p->W, sizeof(double2) * p->N * p->N, "W");
        AL(p->W32, sizeof(float2) * p->N * p->N, "W32");
    }
    if (toeplitz) {
        AL(p->Ttab, sizeof(double2) * (2 * e.nx - 1) * (2 * e.ny - 1) * (2 * e.nz - 1), "Toeplitz table");
        if (!p->lean_gx()) AL(p->Gx, sizeof(float4) * p->N * p->N, "exact Gram");
        AL(p->Gd, gram_digit_bytes(p->N), "exact Gram digits");
        {
            // digits of conj(A) for the exact E^H d, formed once per build (PINV_ADJ_TABLE=0: in every CTA)
            const char* env = std::getenv("PINV_ADJ_TABLE");
            if (!p->lean && !e.b0df && !e.b0tab && e.extdf && !(env && std::strcmp(env, "0") == 0))
                AL(p->Ad, adj_digit_bytes(e), "E^H digits");
        }
        AL(p->eG, sizeof(int), "exact Gram exponent");
    }
    if (p->precision != PINV_FP64 && !p->lean && e.b0df && p->refine_residual == PINV_RESIDUAL_DOUBLE_FLOAT) {
        // digits of conj(A) and of A for the exact E^H d and E x of the refinement
        // (48 bytes per entry of A). Without room for them the plan keeps the
        // double-float products (PINV_B0_EXACT=0: always).
        const char* env = std::getenv("PINV_B0_EXACT");
        if (!(env && std::strcmp(env, "0") == 0)) {
            void *ad = nullptr, *af = nullptr;
            const size_t ba = adj_digit_bytes(e), bf = fwd_digit_bytes(e);
            if (work_alloc(&ad, ba, 0) == cudaSuccess && work_alloc(&af, bf, 0) == cudaSuccess &&
                cudaStreamSynchronize(0) == cudaSuccess) {
                p->Ad = (uint8_t*)ad;
                p->Af = (uint8_t*)af;
                p->allocs.push_back(ad);
                p->allocs.push_back(af);
                p->bytes += ba + bf;
            } else {
                cudaGetLastError();
                if (ad) cudaFreeAsync(ad, 0);
                if (af) cudaFreeAsync(af, 0);
                cudaStreamSynchronize(0);
            }
        }
    }
    int rm = d->recon_mode;
    if (rm == PINV_RECON_AUTO) {
        size_t rb = (size_t)p->N * p->M * (p->precision == PINV_FP64 ? 16 : 8);
        rm = rb <= ((size_t)64 << 30) ? 1 : 0;
    }
    p->recon = rm ? 1 : 0;
    if (p->recon) {
        size_t rb = (size_t)p->N * p->M * (p->precision == PINV_FP64 ? sizeof(double2) : sizeof(float2));
        AL(p->R, rb, "Recon");
        p->bytes_recon = rb;
    }
    for (auto& ev : p->ev) CKC(cudaEventCreate(&ev));
    if (p->precision != PINV_FP64) {
        AL(p->st_inv, sizeof(DevStatus), "inverse status");
        CKC(cudaMemset(p->st_inv, 0, sizeof(DevStatus)));
        // stream priorities: the Cholesky chain, its in-panel side work and its trailing
        // updates first, the inverse (one panel behind) next, the exact Gram last
        int prio_lo = 0, prio_hi = 0;
        CKC(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
        CKC(cudaStreamCreateWithPriority(&p->s_inv, cudaStreamNonBlocking, (prio_lo + prio_hi) / 2));
        CKC(cudaStreamCreateWithPriority(&p->s_x, cudaStreamNonBlocking, prio_lo));
        CKC(cudaEventCreateWithFlags(&p->ev_xjoin, cudaEventDisableTiming));
        AL(p->st_trail, sizeof(DevStatus), "trailing-update status");
        CKC(cudaMemset(p->st_trail, 0, sizeof(DevStatus)));
        CKC(cudaStreamCreateWithPriority(&p->s_trail, cudaStreamNonBlocking, prio_hi));
        CKC(cudaEventCreateWithFlags(&p->ev_tab, cudaEventDisableTiming));
        CKC(cudaEventCreateWithFlags(&p->ev_trail, cudaEventDisableTiming));
        CKC(cudaStreamCreateWithPriority(&p->s_chol, cudaStreamNonBlocking, prio_hi));
        CKC(cudaStreamCreateWithPriority(&p->s_pnl, cudaStreamNonBlocking, prio_hi));
        CKC(cudaEventCreateWithFlags(&p->ev_next, cudaEventDisableTiming));
        CKC(cudaEventCreateWithFlags(&p->ev_side, cudaEventDisableTiming));
        CKC(cudaEventCreateWithFlags(&p->ev_chol, cudaEventDisableTiming));
        p->ev_panel.assign((size_t)((p->N + 255) / 256), nullptr);
        for (auto& ev : p->ev_panel) CKC(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
        CKC(cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming));
        CKC(cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming));
        CKC(cudaEventCreateWithFlags(&p->ev_xfork, cudaEventDisableTiming));
    }
    pinv_status rs = reset_status(p, s);
    if (rs != PINV_OK) return cleanup(rs);
    CKC(cudaStreamSynchronize(s));
#undef AL
#undef CKC
    *out = p;
    ++g_live_plans;
    return PINV_OK;
}

pinv_status pinv_plan_keep_gram(pinv_plan* p, int keep) {
    if (!p) return fail(PINV_ERR_INVALID_ARG, "null plan");
    p->keep_gram = keep != 0;
    return PINV_OK;
}

pinv_status pinv_build(pinv_plan* p, void* stream) {
    g_err.clear();
    if (!p) return fail(PINV_ERR_INVALID_ARG, "null plan");
    cudaStream_t s = (cudaStream_t)stream;
    pinv_status st = build_begin(p, s);
    if (st != PINV_OK) return st;
    CK(cudaEventRecord(p->ev[0], s));
    CK(cudaEventRecord(p->ev[1], s));  // tables were built at plan creation
    if ((st = build_gram(p, s, true)) != PINV_OK) return st;
    CK(cudaEventRecord(p->ev[2], s));
    if ((st = build_factor(p, s, true)) != PINV_OK) return st;
    CK(cudaEventRecord(p->ev[4], s));
    if ((st = build_recon(p, s)) != PINV_OK) return st;
    if ((st = build_end(p, s)) != PINV_OK) return st;
    CK(cudaEventRecord(p->ev[5], s));
    p->built = true;
    return PINV_OK;
}

pinv_status pinv_plan_sync(pinv_plan* p) {
    if (!p) return fail(PINV_ERR_INVALID_ARG, "null plan");
    // the build's last step copies the status word to pinned host memory
    // before its completion event, so no device-wide synchronisation is needed
    CK(cudaEventSynchronize(p->ev[5]));
    CK(cudaGetLastError());
    const DevStatus h = *p->st_host;
    p->info = -1;
    // a wait that gave up leaves everything after it incomplete (a pivot check
    // included), so it is reported first
    if (h.timeout_site) {
        p->built = false;
        return fail(PINV_ERR_TIMEOUT, "a bounded device wait gave up (site " +
                                          std::to_string(h.timeout_site) + ")");
    }
    if (h.not_pd_pivot != INT_MAX) {
        p->info = h.not_pd_pivot;
        p->built = false;
        return fail(PINV_ERR_NOT_PD, "Gram matrix not positive definite at pivot " +
                                         std::to_string(h.not_pd_pivot) + " (increase lambda)");
    }
    if (h.error_code) {
        p->built = false;
        return fail(PINV_ERR_INTERNAL, "device error code " + std::to_string(h.error_code));
    }
    return PINV_OK;
}

pinv_status pinv_plan_export(const pinv_plan* p, int what, void* dst, size_t bytes, void* stream) {
    g_err.clear();
    if (!p || !dst) return fail(PINV_ERR_INVALID_ARG, "null plan or destination");
    if (!p->built) return fail(PINV_ERR_NOT_BUILT, "plan not built");
    cudaStream_t s = (cudaStream_t)stream;
    size_t nn = sizeof(double2) * p->N * p->N;
    const void* src = nullptr;
    size_t need = nn;
    switch (what) {
        case PINV_EXPORT_GRAM:
            if (!p->Gkeep) return fail(PINV_ERR_NOT_BUILT, "Gram not kept (pinv_plan_keep_gram before build)");
            src = p->Gkeep;
            break;
        case PINV_EXPORT_CHOL:
            if (!p->G) return fail(PINV_ERR_UNSUPPORTED, "a lean plan keeps no Cholesky factor");
            src = p->G;
            break;
        case PINV_EXPORT_GINV:
            if (!p->Ginv && !p->W) return fail(PINV_ERR_UNSUPPORTED, "a lean mixed plan keeps no FP64 inverse");
            src = p->Ginv;
            break;
        case PINV_EXPORT_LINV:
            if (!p->W) return fail(PINV_ERR_UNSUPPORTED, "only mixed-precision plans that are not lean keep L^-1");
            src = p->W;
            break;
        case PINV_EXPORT_GRAM_EXACT:
            if (!p->Gx) return fail(PINV_ERR_UNSUPPORTED, "only TOEPLITZ-residual plans that are not lean keep the exact Gram");
            src = p->Gx;
            break;
        case PINV_EXPORT_RECON:
            if (!p->recon) return fail(PINV_ERR_UNSUPPORTED, "factor-only plan has no Recon");
            src = p->R;
            need = p->bytes_recon;
            break;
        default: return fail(PINV_ERR_INVALID_ARG, "unknown export");
    }
    if (bytes < need) return fail(PINV_ERR_INVALID_ARG, "destination too small");
    if (what == PINV_EXPORT_CHOL) {
        if (p->precision != PINV_FP64)  // L in double-float storage
            CK(launch_copy_lower_df((const float4*)p->G, p->N, p->N, (double2*)dst, s));
        else
            CK(launch_copy_lower(p->G, p->N, p->N, (double2*)dst, s));
    } else if (what == PINV_EXPORT_GRAM_EXACT) {
        CK(launch_from_df(p->Gx, p->N * p->N, (double2*)dst, s));
    } else if (what == PINV_EXPORT_GINV && !p->Ginv) {
        // mixed plans keep W = L^-1; G^-1 = W^H W is formed in FP64 on request
        CK(launch_lauum64(p->W, p->N, p->N, (double2*)dst, s));
    } else {
        CK(cudaMemcpyAsync(dst, src, need, cudaMemcpyDeviceToDevice, s));
    }
    return PINV_OK;
}

pinv_status pinv_plan_info(const pinv_plan* p, pinv_plan_info_t* o) {
    if (!p || !o) return fail(PINV_ERR_INVALID_ARG, "null plan or output");
    std::memset(o, 0, sizeof(*o));
    o->n_vox = p->N;
    o->n_samples = p->Mk;
    o->n_rows = p->M;
    o->n_coils = p->C;
    o->precision = p->precision;
    o->has_recon = p->recon;
    o->lambda_abs = p->lambda_abs;
    o->bytes_device = p->bytes;
    o->bytes_recon = p->bytes_recon;
    o->info = p->info;
    o->last_refine_iters = p->last_refine_iters;
    o->last_refine_resid = p->last_refine_resid;
    o->last_refine_bound = p->last_refine_bound;
    if (p->built) {
        CK(cudaEventSynchronize(p->ev[5]));
        float t[5] = {0};
        for (int i = 0; i < 5; ++i) CK(cudaEventElapsedTime(&t[i], p->ev[i], p->ev[i + 1]));
        o->ms_tables = t[0];
        o->ms_gram = t[1];
        o->ms_chol = t[2];
        o->ms_inverse = t[3];
        o->ms_recon = t[4];
        float tg = 0.f;
        if (cudaEventElapsedTime(&tg, p->ev[6], p->ev[7]) != cudaSuccess) {
            cudaGetLastError();
            tg = 0.f;
        }
        o->ms_gram_kernel = tg;
        float tc = 0.f;
        if (cudaEventElapsedTime(&tc, p->ev[8], p->ev[9]) != cudaSuccess) {
            cudaGetLastError();
            tc = 0.f;
        }
        o->ms_cond = tc;
        const DevStatus h = *p->st_host;
        o->min_pivot = h.min_pivot;
        o->max_pivot = h.max_pivot;
        o->norm1_g = h.norm1_g;
        o->kappa_est = h.kappa_est;
    }
    return PINV_OK;
}

void pinv_plan_destroy(pinv_plan* p) {
    if (!p) return;
    cudaDeviceSynchronize();
    delete p;
    if (--g_live_plans == 0) {
        cudaMemPool_t pool = build_pool();
        const char* env = std::getenv("PINV_POOL_KEEP_MB");
        const size_t keep = env ? (size_t)std::strtoull(env, nullptr, 10) << 20 : size_t(8) << 30;
        if (pool) cudaMemPoolTrimTo(pool, keep);
    }
}

}  // extern "C"
