// Applying a built plan: image = Recon x data (Eq. 3), or G^-1 E^H data for
// factor-only plans (Section 3.3), followed by residual refinement.
//
// apply_impl allocates nothing: its scratch comes from the caller, carved
// from one contiguous region by apply_scratch_layout. pinv_apply uses a
// plan-owned region grown on demand, pinv_apply_noalloc a fixed device array,
// and the serving loop one region per slot.
#include <algorithm>
#include <cmath>
#include <string>

#include "plan_impl.h"

namespace pinv {

namespace {
pinv_status cuda_err(cudaError_t e, const char* where) {
    return set_error(e == cudaErrorMemoryAllocation ? PINV_ERR_OOM : PINV_ERR_CUDA,
                     std::string(where) + ": " + cudaGetErrorString(e));
}
#define CKA(call)                                              \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_err(e_, #call);     \
    } while (0)

// Sequential 256-byte-aligned carving of a region (base == nullptr: sizing only).
struct Carver {
    unsigned char* base;
    size_t used = 0;
    template <class T>
    T* take(size_t count) {
        used = (used + 255) & ~size_t(255);
        T* q = reinterpret_cast<T*>(base ? base + used : nullptr);
        used += count * sizeof(T);
        return q;
    }
};
}  // namespace

// Which arithmetic an apply of plan p runs (shared by the layout and the apply).
struct ApplyModes {
    bool mixed, refine, stop_rule, toep, dfres, fpres, need_b;
};
static ApplyModes apply_modes(const pinv_plan* p) {
    ApplyModes m;
    m.mixed = p->precision != PINV_FP64;
    m.refine = p->refine_iters > 0;
    m.stop_rule = m.refine && p->refine_tol > 0.0;
    m.toep = m.mixed && p->refine_residual == PINV_RESIDUAL_TOEPLITZ;
    m.dfres = m.mixed && p->refine_residual == PINV_RESIDUAL_DOUBLE_FLOAT;
    m.fpres = m.mixed && p->refine_residual == PINV_RESIDUAL_FP64;
    // E^H d formed once in double-float: the exact-Gram residual needs it, and
    // mixed factor-only plans start from x = W^H W E^H d
    m.need_b = (m.toep && m.refine) || (m.mixed && !p->recon && !m.fpres);
    return m;
}

size_t apply_scratch_layout(const pinv_plan* p, int64_t F, int dtype, void* base, ApplyScratch* sc) {
    const int64_t N = p->N, M = p->M;
    const ApplyModes md = apply_modes(p);
    // FP64 copy of c64 data (every path but the mixed Recon-only apply reads
    // it), FP64 image for c64 output, data-space residual (E-generating
    // residuals and the FP64 factor-only temporary), image-space residual,
    // E^H d, the mixed path's c64 data / image / correction temporaries, and
    // the per-frame norms of the stopping rule
    const bool need_d128 = dtype == PINV_C64 && (!md.mixed || !p->recon || md.refine);
    const bool need_x128 = dtype == PINV_C64;
    const bool need_u128 = (md.refine && !md.toep) || (md.fpres && !p->recon);
    const bool need_r128 = md.refine || !p->recon;
    const bool need_d64 = md.mixed && p->recon && dtype == PINV_C128;
    const bool need_x64 = md.mixed && (p->recon || md.dfres || md.toep);
    Carver cv{static_cast<unsigned char*>(base)};
    ApplyScratch s{};
    s.d128 = need_d128 ? cv.take<double2>((size_t)(F * M)) : nullptr;
    s.x128 = need_x128 ? cv.take<double2>((size_t)(F * N)) : nullptr;
    s.u128 = need_u128 ? cv.take<double2>((size_t)(F * M)) : nullptr;
    s.r128 = need_r128 ? cv.take<double2>((size_t)(F * N)) : nullptr;
    s.b128 = md.need_b ? cv.take<double2>((size_t)(F * N)) : nullptr;
    s.d64 = need_d64 ? cv.take<float2>((size_t)(F * M)) : nullptr;
    s.x64 = need_x64 ? cv.take<float2>((size_t)(F * N)) : nullptr;
    s.norms = md.stop_rule ? cv.take<double>((size_t)(3 * F)) : nullptr;
    const bool atc = md.mixed && p->recon && apply_tc_ok(F);
    const bool ctc = md.mixed && (md.dfres || md.toep || !p->recon) && correct_tc_ok(F);
    if (atc) s.apw = cv.take<float2>(apply_tc_work_elems(N, M, F));
    if (ctc) s.cw = cv.take<float2>(correct_tc_work_elems(N, F));
    if (atc || ctc) s.sched = cv.take<DevStatus>(1);
    if (md.dfres || md.toep || md.need_b) {
        // E^H u (rows N, length M), E x (rows M, length N), G x (rows N, length N),
        // and the exact tensor-core E^H d
        size_t w = std::max(df_work_elems(N, F, M), std::max(df_work_elems(M, F, N), df_work_elems(N, F, N)));
        const bool xadj = md.need_b && exact_adjoint_ok(p->enc, F, p->Ad != nullptr);
        const bool xres = md.toep && md.refine && p->Gd;
        // plans with B0 and the digit tables: E x and E^H u of every residual exactly
        const bool xfwd = md.dfres && md.refine && p->Af && p->Ad && exact_adjoint_ok(p->enc, F, true);
        if (xadj || xfwd) w = std::max(w, exact_work_elems(p->enc, F));
        if (xres) w = std::max(w, resid_exact_work_elems(N, F));
        if (xfwd) w = std::max(w, exact_fwd_work_elems(p->enc, F));
        if (xadj || xres || xfwd) {
            s.fexp = cv.take<int>((size_t)F);
            size_t bd = std::max(xadj || xfwd ? exact_bdigit_bytes(p->enc, F) : 0,
                                 xres ? resid_bdigit_bytes(N, F) : 0);
            if (xfwd) bd = std::max(bd, exact_fwd_bdigit_bytes(p->enc, F));
            s.xbd = cv.take<uint8_t>(bd);
        }
        if (xfwd) s.y128 = cv.take<double2>(exact_fwd_y_elems(p->enc, F));
        s.xadj = xadj;
        s.xfwd = xfwd;
        s.dfw = w ? cv.take<float4>(w) : nullptr;
    }
    if (sc) *sc = s;
    return cv.used;
}

pinv_status apply_check(const pinv_plan* p, const void* d_data, void* d_image, int64_t F, int dtype) {
    if (!p) return set_error(PINV_ERR_INVALID_ARG, "null plan");
    if (F < 0) return set_error(PINV_ERR_INVALID_ARG, "n_frames < 0");
    if (dtype != PINV_C64 && dtype != PINV_C128) return set_error(PINV_ERR_INVALID_ARG, "dtype");
    if (!p->built) return set_error(PINV_ERR_NOT_BUILT, "plan not built");
    if (F > 0 && (!d_data || !d_image)) return set_error(PINV_ERR_INVALID_ARG, "null data or image");
    return PINV_OK;
}

pinv_status apply_impl(pinv_plan* p, const void* d_data, void* d_image, int64_t F, int dtype, cudaStream_t s,
                       const ApplyScratch& sc) {
    if (F == 0) return PINV_OK;
    const int64_t N = p->N, M = p->M;
    const ApplyModes md = apply_modes(p);
    p->last_refine_iters = 0;
    p->last_refine_resid = 0;
    p->last_refine_bound = 0;

    // FP64 view of the data
    const double2* D = nullptr;
    if (dtype == PINV_C128) {
        D = (const double2*)d_data;
    } else if (sc.d128) {
        CKA(launch_c64_to_c128((const float2*)d_data, sc.d128, F * M, s));
        D = sc.d128;
    }
    double2* X = dtype == PINV_C128 ? (double2*)d_image : sc.x128;
    if (sc.sched) CKA(cudaMemsetAsync(sc.sched, 0, sizeof(DevStatus), s));
    // x += W^H (W r) with the FP32 W: on the tensor cores (correct_tc_ok), else SIMT
    auto correct = [&](const double2* r) -> cudaError_t {
        if (sc.cw) return launch_correct_tc(p->W32, N, r, F, sc.x64, X, sc.cw, p->slices(), sc.sched, s);
        return launch_correct32(p->W32, N, r, F, sc.x64, X, s);
    };

    if (md.need_b) {  // b = E^H d, exactly on the tensor cores where possible
        if (sc.xadj) CKA(launch_adjoint_exact(p->enc, D, F, sc.fexp, sc.xbd, sc.b128, sc.dfw, p->st, s, p->Ad));
        else CKA(launch_adjoint_df(p->enc, D, F, 0.0, nullptr, sc.b128, s, sc.dfw));
    }
    if (!md.mixed) {
        if (p->recon) {
            CKA(launch_apply64((const double2*)p->R, N, M, D, F, X, s));
        } else {
            CKA(launch_adjoint64(p->enc, D, F, 0.0, nullptr, sc.r128, s));
            CKA(launch_hemv64(p->Ginv, N, N, sc.r128, F, nullptr, X, s));
        }
    } else if (p->recon) {
        // initial image from the mixed-precision Recon
        const float2* D32 = (const float2*)d_data;
        if (dtype == PINV_C128) {
            CKA(launch_c128_to_c64((const double2*)d_data, sc.d64, F * M, s));
            D32 = sc.d64;
        }
        // the refinement removes this product's rounding: split-BF16 on the tensor cores
        if (sc.apw) {
            CKA(launch_apply_tc((const float2*)p->R, N, M, D32, F, sc.x64, sc.apw, p->slices(), sc.sched, s));
        }
        else CKA(launch_apply32((const float2*)p->R, N, M, D32, F, sc.x64, s));
        CKA(launch_c64_to_c128(sc.x64, X, F * N, s));
    } else if (md.fpres) {
        // factor-only, FP64 throughout: x = W^H (W (E^H d))
        CKA(launch_adjoint64(p->enc, D, F, 0.0, nullptr, sc.r128, s));
        CKA(launch_trmv64(p->W, N, sc.r128, F, sc.u128, s));
        CKA(launch_trmv_h64(p->W, N, sc.u128, F, nullptr, X, s));
    } else {
        // factor-only: x = W^H (W b) with b = E^H d in double-float
        CKA(cudaMemsetAsync(X, 0, sizeof(double2) * F * N, s));
        CKA(correct(sc.b128));
    }

    // Residual refinement: r = E^H (d - E x) - lambda x (= E^H d - G x), then
    // x += G^-1 r. Mixed plans need it to reach FP64-level accuracy; FP64 plans
    // may use it to remove the explicit inverse's extra rounding (kappa(G) u).
    // With refine_tol == 0 a fixed number of steps runs without host reads.
    if (md.refine) {
        if (md.stop_rule) {
            if (md.need_b) {
                CKA(launch_frame_norms(sc.b128, F, N, sc.norms + F, s));
            } else {
                CKA(launch_adjoint64(p->enc, D, F, 0.0, nullptr, sc.r128, s));  // b = E^H d
                CKA(launch_frame_norms(sc.r128, F, N, sc.norms + F, s));
            }
        }
        // r = E^H (d - E x) - lambda x (= b - G x) of the current x into sc.r128
        auto residual = [&]() -> cudaError_t {
            cudaError_t e;
            if (md.toep && p->Gd)  // r = b - G x, exactly on the tensor cores
                return launch_gram_resid_exact(p->Gd, p->eG, N, sc.b128, X, F, sc.fexp, sc.xbd, sc.r128, sc.dfw,
                                               p->st, s);
            if (md.toep) return launch_gram_resid_df(p->Gx, N, sc.b128, X, F, sc.r128, s, sc.dfw);  // r = b - G x
            if (md.dfres && sc.xfwd) {  // u = d - E x, r = E^H u - lambda x, exact digit products
                if ((e = launch_forward_exact(p->enc, X, F, D, sc.u128, p->Af, sc.y128, sc.fexp, sc.xbd, sc.dfw,
                                              p->st, s)) != cudaSuccess)
                    return e;
                if ((e = launch_adjoint_exact(p->enc, sc.u128, F, sc.fexp, sc.xbd, sc.r128, sc.dfw, p->st, s,
                                              p->Ad)) != cudaSuccess)
                    return e;
                return launch_minus_lambda(sc.r128, X, p->lambda_abs, F * N, s);
            }
            if (md.dfres) {
                if ((e = launch_forward_df(p->enc, X, F, D, sc.u128, s, sc.dfw)) != cudaSuccess) return e;  // u = d - E x
                return launch_adjoint_df(p->enc, sc.u128, F, p->lambda_abs, X, sc.r128, s, sc.dfw);
            }
            if ((e = launch_forward64(p->enc, X, F, D, sc.u128, s)) != cudaSuccess) return e;
            return launch_adjoint64(p->enc, sc.u128, F, p->lambda_abs, X, sc.r128, s);
        };
        // stopping rule: per-frame ||r|| / ||E^H d|| read back in fixed-size chunks (no
        // allocation); with `bound`, also the certified error bound of x (below)
        auto check = [&](bool bound, double* worst_out, double* bound_out) -> pinv_status {
            CKA(launch_frame_norms(sc.r128, F, N, sc.norms, s));
            if (bound) CKA(launch_frame_norms(X, F, N, sc.norms + 2 * F, s));
            double worst = 0.0, wb = 0.0, hn[128], hb[128], hx[128];
            for (int64_t f0 = 0; f0 < F; f0 += 128) {
                const int64_t nf = std::min<int64_t>(128, F - f0);
                CKA(cudaMemcpyAsync(hn, sc.norms + f0, sizeof(double) * nf, cudaMemcpyDeviceToHost, s));
                CKA(cudaMemcpyAsync(hb, sc.norms + F + f0, sizeof(double) * nf, cudaMemcpyDeviceToHost, s));
                if (bound)
                    CKA(cudaMemcpyAsync(hx, sc.norms + 2 * F + f0, sizeof(double) * nf, cudaMemcpyDeviceToHost, s));
                CKA(cudaStreamSynchronize(s));
                for (int64_t f = 0; f < nf; ++f) {
                    // a residual or image that is not finite (data with NaN or Inf, or a
                    // factor that lost them) ends the refinement with an error
                    if (!std::isfinite(hn[f]) || !std::isfinite(hb[f]) || (bound && !std::isfinite(hx[f])))
                        return set_error(PINV_ERR_INVALID_ARG, "non-finite residual or image in frame " +
                                                                   std::to_string(f0 + f));
                    worst = std::max(worst, std::sqrt(hn[f] / std::max(hb[f], 1e-300)));
                    if (bound) wb = std::max(wb, std::sqrt(hn[f] / std::max(hx[f], 1e-300)) / p->lambda_abs);
                }
            }
            *worst_out = worst;
            if (bound_out) *bound_out = wb;
            return PINV_OK;
        };
        bool converged = false;
        for (int it = 0; it < p->refine_iters; ++it) {
            CKA(residual());
            if (md.stop_rule) {
                // with the stopping rule the residual is checked before the correction:
                // an x whose residual is already below the tolerance is kept as it is
                double worst = 0.0, wb = 0.0;
                const pinv_status cs = check(true, &worst, &wb);
                if (cs != PINV_OK) return cs;
                p->last_refine_resid = worst;
                p->last_refine_bound = wb;
                if (worst <= p->refine_tol) {
                    converged = true;
                    break;
                }
            }
            if (md.dfres || md.toep) {
                // the correction only preconditions the next residual: FP32 W suffices
                CKA(correct(sc.r128));
            } else if (md.mixed) {
                // x += W^H (W r) in FP64: never through an explicitly formed low-precision
                // G^-1, whose error the correction would amplify by kappa(G)
                CKA(launch_trmv64(p->W, N, sc.r128, F, sc.u128, s));
                CKA(launch_trmv_h64(p->W, N, sc.u128, F, X, X, s));
            } else {
                CKA(launch_hemv64(p->Ginv, N, N, sc.r128, F, X, X, s));
            }
            p->last_refine_iters = it + 1;
        }
        if (md.stop_rule && !converged) {
            // the residual of the x returned, so the recorded ratio and bound describe it
            CKA(residual());
            double worst = 0.0, wb = 0.0;
            const pinv_status cs = check(true, &worst, &wb);
            if (cs != PINV_OK) return cs;
            p->last_refine_resid = worst;
            p->last_refine_bound = wb;
        }
    }
    if (dtype == PINV_C64) CKA(launch_c128_to_c64(X, (float2*)d_image, F * N, s));
    return PINV_OK;
}

}  // namespace pinv

using namespace pinv;

extern "C" pinv_status pinv_apply(pinv_plan* p, const void* d_data, void* d_image, int64_t F, int dtype,
                                  void* stream) {
    pinv_status st = apply_check(p, d_data, d_image, F, dtype);
    if (st != PINV_OK || F == 0) return st;
    const size_t need = apply_scratch_layout(p, F, dtype, nullptr, nullptr);
    if (need > p->scratch_bytes) {
        // grow the plan-owned scratch, from the library's pool: the old region after
        // every earlier apply (on any stream) is done, the new one complete before
        // any stream uses it
        if (p->scratch_buf) {
            cudaError_t e = cudaDeviceSynchronize();
            if (e == cudaSuccess) e = cudaFreeAsync(p->scratch_buf, 0);
            p->scratch_buf = nullptr;
            p->scratch_bytes = 0;
            if (e != cudaSuccess) return cuda_err(e, "free(apply scratch)");
        }
        cudaError_t e = work_alloc(&p->scratch_buf, need, 0);
        if (e == cudaSuccess) e = cudaStreamSynchronize(0);
        if (e != cudaSuccess) {
            p->scratch_buf = nullptr;
            return cuda_err(e, "alloc(apply scratch)");
        }
        p->scratch_bytes = need;
    }
    ApplyScratch sc;
    apply_scratch_layout(p, F, dtype, p->scratch_buf, &sc);
    return apply_impl(p, d_data, d_image, F, dtype, (cudaStream_t)stream, sc);
}
