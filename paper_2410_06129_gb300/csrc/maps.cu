// Per-voxel image-quality maps from a built plan (Section 2.5).
//
// SRF = Recon x Encode (Eq. 9). With Recon = G^-1 E^H and E^H E = G - lambda I
// this is I - lambda G^-1, so the SRF map is 1 - lambda diag(G^-1).
// Noise matrix X = Recon Psi Recon^H (Eq. 10). For white noise (Psi = I) it is
// G^-1 (G - lambda I) G^-1 = G^-1 - lambda G^-2, so the noise map is
// diag(G^-1) - lambda diag(G^-2); diag(G^-2)[n] is the squared norm of column n
// of G^-1. With a coil noise covariance psi (C x C, the same for every sample)
// the map is formed from the stored Recon rows: X[n][n] = sum_m sum_{c,c'}
// Recon[n][(c,m)] psi[c][c'] conj(Recon[n][(c',m)]).
//
// Which G^-1: FP64 plans use their FP64 G^-1. Mixed plans with the exact Gram
// (TOEPLITZ residual) refine G^-1 itself: Y = W^H W, then Y += W^H W (I - G Y)
// for refine_iters steps with the double-float residual, the columns of the
// identity taking the place of frames. Other mixed plans use W^H W formed in
// FP64 from their split-precision W, so their maps carry that factor's error.
#include <algorithm>
#include <vector>

#include "plan_impl.h"

namespace pinv {
namespace {

pinv_status cuda_err(cudaError_t e, const char* where) {
    return set_error(e == cudaErrorMemoryAllocation ? PINV_ERR_OOM : PINV_ERR_CUDA,
                     std::string(where) + ": " + cudaGetErrorString(e));
}
#define CKM(call)                                              \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_err(e_, #call);     \
    } while (0)

// out[n] = srf ? 1 - lam * Y[n][n] : Y[n][n] - lam * norm2[n]   (Y Hermitian)
__global__ void k_map_from_ginv(const double2* Y, int64_t N, const double* norm2, double lam, int srf,
                                double* out) {
    const int64_t n = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= N) return;
    const double d = Y[n * N + n].x;
    out[n] = srf ? 1.0 - lam * d : d - lam * norm2[n];
}

// frame layout: row f of the array is column f of G^-1, the conjugate of row f
__global__ void k_conj(double2* a, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i].y = -a[i].y;
}

// X[n][n] for Recon rows (c128 or c64) and a C x C coil covariance; one block per voxel
template <class T>
__global__ void k_noise_recon(const T* R, int64_t N, int64_t Mk, int C, const double2* psi, double* out) {
    __shared__ double part[256];
    const int64_t n = blockIdx.x;
    const T* row = R + n * Mk * C;
    double acc = 0.0;
    for (int64_t m = threadIdx.x; m < Mk; m += blockDim.x) {
        for (int c = 0; c < C; ++c) {
            const T a = row[(int64_t)c * Mk + m];
            double2 t = make_double2(0.0, 0.0);  // sum_c' psi[c][c'] conj(R[c'])
            for (int c2 = 0; c2 < C; ++c2) {
                const T b = row[(int64_t)c2 * Mk + m];
                const double2 p = psi[c * C + c2];
                t.x += p.x * (double)b.x + p.y * (double)b.y;
                t.y += p.y * (double)b.x - p.x * (double)b.y;
            }
            acc += (double)a.x * t.x - (double)a.y * t.y;  // real part of a * t
        }
    }
    part[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[n] = part[0];
}

}  // namespace
}  // namespace pinv

using namespace pinv;

extern "C" pinv_status pinv_plan_map(pinv_plan* p, int what, const double* psi, double* d_out, void* stream) {
    if (!p || !d_out) return set_error(PINV_ERR_INVALID_ARG, "null plan or output");
    if (what != PINV_MAP_SRF && what != PINV_MAP_NOISE) return set_error(PINV_ERR_INVALID_ARG, "unknown map");
    if (!p->built) return set_error(PINV_ERR_NOT_BUILT, "plan not built");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = p->N;
    if (!p->Ginv && !p->W && !(what == PINV_MAP_NOISE && psi))
        return set_error(PINV_ERR_UNSUPPORTED, "a lean mixed plan keeps no FP64 inverse for maps");
    if (what == PINV_MAP_NOISE && psi) {
        if (!p->recon) return set_error(PINV_ERR_UNSUPPORTED, "a coil-covariance noise map needs the stored Recon");
        double2* dpsi = nullptr;
        CKM(work_alloc((void**)&dpsi, sizeof(double2) * p->C * p->C, s));
        CKM(cudaMemcpyAsync(dpsi, psi, sizeof(double2) * p->C * p->C, cudaMemcpyHostToDevice, s));
        if (p->precision == PINV_FP64)
            k_noise_recon<<<(unsigned)N, 256, 0, s>>>((const double2*)p->R, N, p->Mk, p->C, dpsi, d_out);
        else
            k_noise_recon<<<(unsigned)N, 256, 0, s>>>((const float2*)p->R, N, p->Mk, p->C, dpsi, d_out);
        note_launch();
        CKM(cudaGetLastError());
        CKM(cudaFreeAsync(dpsi, s));  // a pageable copy is staged before cudaMemcpyAsync returns
        return PINV_OK;
    }
    // Y = G^-1 (full, Hermitian), Y[f][n] read as frames f of an [N][N] array
    double2* Y = p->Ginv;
    double2 *Yown = nullptr, *B = nullptr, *R = nullptr;
    float2* T = nullptr;
    float4* work = nullptr;
    double* norm2 = nullptr;
    auto release = [&]() {
        if (Yown) cudaFreeAsync(Yown, s);
        if (B) cudaFreeAsync(B, s);
        if (R) cudaFreeAsync(R, s);
        if (T) cudaFreeAsync(T, s);
        if (work) cudaFreeAsync(work, s);
        if (norm2) cudaFreeAsync(norm2, s);
    };
    auto fail_free = [&](cudaError_t e, const char* where) {
        release();
        return cuda_err(e, where);
    };
#define CKF(call)                                             \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return fail_free(e_, #call);   \
    } while (0)
    if (!Y) {
        CKF(work_alloc((void**)&Yown, sizeof(double2) * N * N, s));
        CKF(launch_lauum64(p->W, N, N, Yown, s));  // W^H W in FP64
        Y = Yown;
        if (p->Gx && p->refine_iters > 0) {
            // refine the columns of G^-1, held as frames (Y[f] = column f): R = I - G Y
            // in double-float, then Y += W^H W R
            k_conj<<<(unsigned)((N * N + 255) / 256), 256, 0, s>>>(Y, N * N);
            note_launch();
            const size_t wel = df_work_elems(N, N, N);
            CKF(work_alloc((void**)&B, sizeof(double2) * N * N, s));
            CKF(work_alloc((void**)&R, sizeof(double2) * N * N, s));
            CKF(work_alloc((void**)&T, sizeof(float2) * N * N, s));
            if (wel) CKF(work_alloc((void**)&work, sizeof(float4) * wel, s));
            CKF(launch_fill_identity(B, N, N, s));
            for (int it = 0; it < p->refine_iters; ++it) {
                CKF(launch_gram_resid_df(p->Gx, N, B, Y, N, R, s, work));
                CKF(launch_correct32(p->W32, N, R, N, T, Y, s));
            }
        }
    }
    if (what == PINV_MAP_NOISE) {
        CKF(work_alloc((void**)&norm2, sizeof(double) * N, s));
        CKF(launch_frame_norms(Y, N, N, norm2, s));  // squared norms of the columns of G^-1
    }
    k_map_from_ginv<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(Y, N, norm2, p->lambda_abs,
                                                                 what == PINV_MAP_SRF ? 1 : 0, d_out);
    note_launch();
    CKF(cudaGetLastError());
    release();
#undef CKF
    return PINV_OK;
}
