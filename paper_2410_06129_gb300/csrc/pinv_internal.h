// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <functional>
#include <string>

#include "pinv.h"

namespace pinv {

// Kernels launched by this library in this process (reported to callers).
extern std::atomic<unsigned long long> g_launches;
inline void note_launch(unsigned long long n = 1) { g_launches.fetch_add(n, std::memory_order_relaxed); }

// Programmatic dependent launch (the Cholesky chain): a kernel launched with
// launch_pdl may start while the kernel before it in its stream drains. Such a
// kernel calls griddep_wait() before it touches global memory, which returns
// once every earlier kernel of the stream has completed and its writes are
// visible; griddep_launch() lets the next kernel's CTAs start (they then wait
// in griddep_wait). In a kernel launched without the attribute both are no-ops.
__device__ inline void griddep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ inline void griddep_launch() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
template <class... KA, class... A>
inline cudaError_t launch_pdl(void (*k)(KA...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    note_launch();
    return cudaLaunchKernelEx(&cfg, k, args...);
}

// ---------------------------------------------------------------------------
// Device-side encoding description: everything a kernel needs to generate an
// element of the coil-independent encoding A[m][n] = exp(-i2pi(k_m.r_n + df_n t_m))
// and the coil factor s_c(n), without ever storing A or E.
// ---------------------------------------------------------------------------
struct EncodeDev {
    int64_t N;        // voxels
    int64_t Mk;       // samples per coil
    int C;            // coils
    int nx, ny, nz;   // separable table widths (1 for unused dimensions)
    const double2* ex;      // [Mk][nx] exp(-i2pi kx_m x_ix)
    const double2* ey;      // [Mk][ny]
    const double2* ez;      // [Mk][nz]
    const int* vox_ijk;     // [N][3] grid coordinates of voxel n
    const double2* b0tab;   // [T][N] exp(-i2pi df_n t_u) or nullptr
    const int* tidx;        // [Mk] index u of t_m in b0tab, or nullptr
    const double2* coils;   // [C][N] s_c(n) or nullptr (C == 1, s = 1)
    // single-precision copies for the tensor-core producers
    const float2* ex32;
    const float2* ey32;
    const float2* ez32;
    const float2* b0tab32;
    const float2* coils32;
    // sample-contiguous FP32 copies for the tensor-core producers:
    // ext32[ix][m] = ex32[m][ix] (rows padded with zeros to Mkp = 8 * ceil(Mk / 8)),
    // b0t32[n][u] = b0tab32[u][n] (T distinct sample times)
    const float2* ext32;
    const float2* eyt32;
    const float2* ezt32;
    const float2* b0t32;
    int64_t Mkp;
    int T;
    int full_grid;          // voxels are the whole grid in flat order (no voxel list)
    // double-float copies (re.hi, re.lo, im.hi, im.lo) for the refinement residual
    // sample-contiguous double-float tables extdf[ix][m] (rows of Mkp, zero
    // padded), for the exact tensor-core E^H d of plans without B0
    const float4* extdf;
    const float4* eytdf;
    const float4* eztdf;
    const float4* exdf;
    const float4* eydf;
    const float4* ezdf;
    const float4* b0df;
    const float4* coilsdf;
};

// Device status word of a plan.
struct DevStatus {
    int not_pd_pivot;   // smallest failing pivot index, INT_MAX if none
    int timeout_site;   // nonzero if a bounded wait gave up
    int error_code;     // other device-detected error
    int pad;
    double min_pivot;   // min diag(L) as ordered bits (set by panel kernels)
    double max_pivot;
    // tile counter of the persistent tensor-core kernel running on this plan's
    // stream (next item, CTAs finished); the last CTA of a launch zeroes both
    unsigned long long sched_next, sched_done;
    // condition estimate (cond.cu): ||G||_1 and kappa_1(G) = ||G||_1 ||G^-1||_1
    double norm1_g;
    double kappa_est;
    // bound of the tensor-core kernels' pipeline waits in SM clock cycles (0: the
    // default, about 2 s); set at every status reset from pinv_set_wait_limit
    long long wait_limit;
};
// the process-wide setting of DevStatus::wait_limit (pinv_set_wait_limit)
long long wait_limit_setting();

// ---------------------------------------------------------------------------
// complex helpers
// ---------------------------------------------------------------------------
__host__ __device__ inline double2 zmul(double2 a, double2 b) {
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ inline double2 zconj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ inline double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ inline double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ inline void zfma(double2& acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}

// Coil-independent encoding element A[m][n] in FP64.
__device__ inline double2 gen_a64(const EncodeDev& e, int64_t m, int64_t n) {
    const int* g = e.vox_ijk + 3 * n;
    double2 v = e.ex[m * e.nx + g[0]];
    if (e.ny > 1) v = zmul(v, e.ey[m * e.ny + g[1]]);
    if (e.nz > 1) v = zmul(v, e.ez[m * e.nz + g[2]]);
    if (e.b0tab) v = zmul(v, e.b0tab[(int64_t)e.tidx[m] * e.N + n]);
    return v;
}

// Encoding element E[(c, m)][n] = s_c(n) A[m][n] in FP64.
__device__ inline double2 gen_e64(const EncodeDev& e, int c, int64_t m, int64_t n) {
    double2 v = gen_a64(e, m, n);
    if (e.coils) v = zmul(v, e.coils[(int64_t)c * e.N + n]);
    return v;
}

// ---------------------------------------------------------------------------
// FP64 kernels (zgemm64.cu, chol64.cu, tables.cu)
// ---------------------------------------------------------------------------
cudaError_t launch_tables(const double* traj, int ndim, int64_t Mk, const int* dims,
                          const double* fov, double2* ex, double2* ey, double2* ez,
                          float2* ex32, float2* ey32, float2* ez32, cudaStream_t s);
cudaError_t launch_b0_table(const double* b0, const double* tuniq, int T, int64_t N,
                            double2* tab, float2* tab32, cudaStream_t s);
cudaError_t launch_to_f32(const double2* src, float2* dst, int64_t n, cudaStream_t s);
// dst[c][r] = src[r][c] for an FP32 [rows][cols] matrix; dst rows have stride ldd >= rows,
// the padding columns rows..ldd-1 are zero-filled.
cudaError_t launch_transpose32(const float2* src, int64_t rows, int64_t cols, float2* dst, int64_t ldd,
                               cudaStream_t s);
cudaError_t launch_fill_identity(double2* W, int64_t N, int64_t ld, cudaStream_t s);
// The identity in double-float storage.
cudaError_t launch_fill_identity_df(float4* W, int64_t N, int64_t ld, cudaStream_t s);
// A lower-triangular matrix in double-float storage to FP64 in place and its FP32
// rounding into W32 (ld N, zero above the diagonal). Above the diagonal W is
// written only inside the diagonal blocks of width blk: the rest must hold zeros
// already (launch_fill_identity_df writes them).
cudaError_t launch_df_finish(float4* W, int64_t N, int64_t ld, int64_t blk, float2* W32, cudaStream_t s);

// Gram G = (A^H A) o (S^H S) + lambda I, lower tiles, FP64.
cudaError_t launch_gram64(const EncodeDev& e, double lambda, double2* G, int64_t ld, cudaStream_t s);
// Cholesky in place on the lower triangle of G (FP64, blocked, nb = 64).
cudaError_t launch_potrf64(double2* G, int64_t N, int64_t ld, double2* Dinv, DevStatus* st,
                           cudaStream_t s);
// W = L^-1 (lower), using the diagonal-block inverses Dinv from the factorisation.
cudaError_t launch_trtri64(const double2* L, int64_t N, int64_t ld, const double2* Dinv,
                           double2* W, cudaStream_t s);
// Ginv = W^H W, full Hermitian matrix.
cudaError_t launch_lauum64(const double2* W, int64_t N, int64_t ld, double2* Ginv, cudaStream_t s);
// One 64x64 diagonal block of the blocked Cholesky (FP64, in shared memory):
// factor in place, check pivots, write the block inverse (and an FP32 copy).
// Launch-shape autotuner: run(c) launches candidate c of a kernel family on
// stream s; returns the fastest candidate for this size class (cached).
using TuneRun = std::function<cudaError_t(int)>;
int tune_pick(const char* family, int64_t rows, int64_t F, int ncand, const TuneRun& run, cudaStream_t s);

// Stream-ordered allocation of build and query temporaries from the library's
// per-device pool, which keeps its memory between builds (free with cudaFreeAsync).
cudaError_t work_alloc(void** ptr, size_t bytes, cudaStream_t s);

// mixed path: the same diagonal block in double-float on the FP32 units, G in
// double-float storage (the block of L written back in place)
cudaError_t launch_potrf_diag_df(float4* G, int64_t ld, int64_t N, int64_t k0, double2* Dinv, float2* Dinv32,
                                 float2* L32, int64_t ldl,
                                 DevStatus* st, cudaStream_t s);
cudaError_t launch_potrf_diag(double2* G, int64_t ld, int64_t N, int64_t k0, double2* Dinv,
                              float2* Dinv32, DevStatus* st, cudaStream_t s);
// Recon[n][(c,m)] = sum_n' Ginv[n][n'] conj(E[(c,m)][n']), FP64.
cudaError_t launch_recon64(const EncodeDev& e, const double2* Ginv, int64_t ld, double2* R,
                           cudaStream_t s);
// X[f][n] = sum_j R[n][j] D[f][j] (R row-major [N][M], D [F][M]), FP64.
cudaError_t launch_apply64(const double2* R, int64_t N, int64_t M, const double2* D, int64_t F,
                           double2* X, cudaStream_t s);
// Y[f][n] = sum_j conj(E[j][n]) D[f][j] - lam * Xsub[f][n] (Xsub may be null), FP64.
cudaError_t launch_adjoint64(const EncodeDev& e, const double2* D, int64_t F, double lam,
                             const double2* Xsub, double2* Y, cudaStream_t s);
// U[f][j] = Dsub[f][j] - sum_n E[j][n] X[f][n] (Dsub may be null: U = -E X), FP64.
cudaError_t launch_forward64(const EncodeDev& e, const double2* X, int64_t F, const double2* Dsub,
                             double2* U, cudaStream_t s);
// Y[f][n] = Yadd[f][n] + sum_n' H[n][n'] X[f][n'] (H full [N][N]), FP64.
cudaError_t launch_hemv64(const double2* H, int64_t N, int64_t ld, const double2* X, int64_t F,
                          const double2* Yadd, double2* Y, cudaStream_t s);
// Copy the lower triangle of G (incl. diagonal) to L, zeroing the upper triangle;
// the _df forms read double-float storage.
cudaError_t launch_copy_lower(const double2* G, int64_t N, int64_t ld, double2* L, cudaStream_t s);
cudaError_t launch_copy_lower_df(const float4* G, int64_t N, int64_t ld, double2* L, cudaStream_t s);
// FP64 copy of n double-float entries (integer-pipe conversion).
cudaError_t launch_df_to_f64(const float4* a, int64_t n, double2* b, cudaStream_t s);
// Pivot extrema of diag(L) into st->min_pivot / max_pivot.
cudaError_t launch_pivot_stats(const double2* L, int64_t N, int64_t ld, DevStatus* st,
                               cudaStream_t s);
cudaError_t launch_pivot_stats_df(const float4* L, int64_t N, int64_t ld, DevStatus* st, cudaStream_t s);
// Conversions between c64 and c128 frame buffers.
cudaError_t launch_c64_to_c128(const float2* a, double2* b, int64_t n, cudaStream_t s);
cudaError_t launch_c128_to_c64(const double2* a, float2* b, int64_t n, cudaStream_t s);
// Per-frame squared norms: out[f] = sum_n |X[f][n]|^2 (FP64).
cudaError_t launch_frame_norms(const double2* X, int64_t F, int64_t n, double* out, cudaStream_t s);
// X += Y (FP64, n elements)
cudaError_t launch_zaxpy(double2* X, const double2* Y, int64_t n, cudaStream_t s);

// ---------------------------------------------------------------------------
// Mixed-precision (tcgen05, split BF16) kernels (tc_gemm.cu)
// ---------------------------------------------------------------------------
// Gram in split BF16 on tcgen05 tensor cores; result written as double-float
// lower tiles (float4 per entry, the storage of mixed plans' G while it is factored).
cudaError_t launch_gram_tc(const EncodeDev& e, double lambda, int slices, float4* G, int64_t ld,
                           DevStatus* st, cudaStream_t s);
// Bulk-fed Gram: the split encoding table (and, for a split sample range, the
// partial sums) in `work` of gram_bulk_bytes(); same result layout as launch_gram_tc.
size_t gram_bulk_bytes(const EncodeDev& e, int slices);
cudaError_t launch_gram_bulk(const EncodeDev& e, double lambda, int slices, float4* G, int64_t ld, void* work,
                             DevStatus* st, cudaStream_t s);
// Recon = W^H (W E^H) in split BF16 on tcgen05 (W = L^-1 in FP32, T = W E^H
// scratch [N][M] c64), c64 out.
cudaError_t launch_recon_tc(const EncodeDev& e, const float2* W32, const float2* WT32, float2* T, int slices,
                            float2* R, DevStatus* st, cudaStream_t s);
// Bulk-fed Recon from split operand tables in `work` of recon_bulk_bytes()
// (processed in chunks of samples); same result as launch_recon_tc.
size_t recon_bulk_bytes(const EncodeDev& e, int slices);
cudaError_t launch_recon_bulk(const EncodeDev& e, const float2* W32, int slices, float2* R, void* work,
                              DevStatus* st, cudaStream_t s);
// Y[f] = W X[f] (lower W), and Y[f] = Yadd[f] + W^H X[f], FP64.
cudaError_t launch_trmv64(const double2* W, int64_t N, const double2* X, int64_t F, double2* Y,
                          cudaStream_t s);
cudaError_t launch_trmv_h64(const double2* W, int64_t N, const double2* X, int64_t F, const double2* Yadd,
                            double2* Y, cudaStream_t s);
// X[f][n] = sum_j R[n][j] D[f][j], c64 (R c64 [N][M], D c64 [F][M]).
cudaError_t launch_apply32(const float2* R, int64_t N, int64_t M, const float2* D, int64_t F,
                           float2* X, cudaStream_t s);
// Blocked Cholesky with double-float diagonal blocks, FP32 panel solves and
// tensor-core trailing updates; L32 receives an FP32 copy of L ([N][N], lower
// part), Dinv32 the FP32 inverses of the diagonal blocks and Dinv (or nullptr)
// their FP64 copies.
// tab (factor_table_bytes(), or nullptr): operand tables of the bulk-fed
// panel trailing updates; without it the updates generate their operands.
size_t factor_table_bytes(int64_t N, int slices);
// ev_panel (or nullptr): one event per 256-wide panel, recorded by the Cholesky once
// the panel's columns of L32 and its diagonal inverses are final, and waited on by
// the inverse before that panel
// la (or nullptr): a second stream with its own status block and two events, on
// which all but the next panel's columns of each trailing update run (lookahead);
// and (s2 non-null) a third stream with two events for the solves and updates inside
// a panel beyond the next diagonal block (block lookahead)
struct TrailLookahead {
    cudaStream_t s;
    DevStatus* st;
    cudaEvent_t ev_tab, ev_done;
    cudaStream_t s2;
    cudaEvent_t ev_next, ev_side;
};
cudaError_t launch_potrf_tc(float4* G, int64_t N, int64_t ld, double2* Dinv, float2* Dinv32, float2* L32,
                            int slices, DevStatus* st, cudaStream_t s, void* tab = nullptr,
                            const cudaEvent_t* ev_panel = nullptr, const TrailLookahead* la = nullptr);
// W = L^-1 (double-float storage while it is formed, FP64 on return; tensor-core
// updates) and its FP32 copy W32.
cudaError_t launch_trtri_tc(const float2* L32, int64_t N, const float2* Dinv32, float4* W, float2* W32,
                            int slices, DevStatus* st, cudaStream_t s, void* tab = nullptr,
                            const cudaEvent_t* ev_panel = nullptr);
bool tc_available();

// ---------------------------------------------------------------------------
// Double-float refinement residual and FP32 correction (dfgemm.cu)
// ---------------------------------------------------------------------------
cudaError_t launch_to_df(const double2* src, float4* dst, int64_t n, cudaStream_t s);
// U[f] = D[f] - E X[f], double-float arithmetic, FP64 in/out
cudaError_t launch_reset_status(DevStatus* st, cudaStream_t s);
cudaError_t launch_merge_timeout(DevStatus* dst, const DevStatus* src, cudaStream_t s);

// Several plans' tensor-core Gram or Recon in one persistent launch. The
// problem descriptors are uploaded once (tc_multi_create) and stay valid
// while the plans and buffers they point to live.
struct TcPlanArgs {
    const EncodeDev* e;
    double lam;
    float4* G;            // Gram output (lower tiles, double-float), ld = N
    const float2* W32;    // W = L^-1, FP32 [N][N]
    float2* R;            // Recon [N][M]
    void* work;           // operand tables: gram_bulk_bytes() for the Gram, recon_bulk_bytes() for Recon
};
enum TcMultiKind { TC_MULTI_GRAM = 0, TC_MULTI_RECON1 = 1, TC_MULTI_RECON2 = 2 };
struct TcMulti {
    void* buf = nullptr;
    int kind = 0, n = 0;
    int64_t items = 0;
    size_t off_start = 0, off_gx = 0;
};
// Shared persistent launches of bulk-fed problems over several plans: every
// plan's Gram, or the two Recon steps over sample chunk `chunk` of every plan
// that has it. The per-plan stages around them (tables, split sums) are the
// gram_bulk_* / recon_bulk_* calls.
cudaError_t tc_multi_create(int kind, const TcPlanArgs* args, int n, int slices, int64_t chunk, TcMulti* out);
cudaError_t tc_multi_launch(const TcMulti& m, int slices, DevStatus* st, cudaStream_t s);
cudaError_t gram_bulk_table(const EncodeDev& e, int slices, void* work, cudaStream_t s);
cudaError_t gram_bulk_finish(const EncodeDev& e, double lambda, int slices, float4* G, int64_t ld, void* work,
                             cudaStream_t s);
int64_t recon_bulk_chunks(const EncodeDev& e, int slices);
cudaError_t recon_bulk_wtables(const EncodeDev& e, const float2* W32, int slices, void* work, cudaStream_t s);
cudaError_t recon_bulk_et(const EncodeDev& e, int slices, void* work, int64_t chunk, cudaStream_t s);
void tc_multi_free(TcMulti* m);

// ||G||_1 into st->norm1_g, from the lower triangle of G before the Cholesky
// overwrites it (FP64 G, or Gdf in double-float storage) or from the full
// double-float exact Gram Gx; exactly one of the three is non-null
cudaError_t launch_gram_norm1(const double2* G, const float4* Gdf, const float4* Gx, int64_t N, int64_t ld,
                              DevStatus* st, cudaStream_t s);

// double-float frame products split their k range over CTAs; `work` holds
// df_work_elems() partials (float4) when the split count is above one
size_t df_work_elems(int64_t rows, int64_t F, int64_t K);

// E^H d exactly on the tensor cores (fixed-point digits; F >= 16; plans with B0
// only with the per-build table of conj(A), table = true).
// fexp: [F] per-frame exponents (written here); Bd: exact_bdigit_bytes() for the
// data's digit tiles (written here); work: partials.
bool exact_adjoint_ok(const EncodeDev& e, int64_t F, bool table);
size_t exact_work_elems(const EncodeDev& e, int64_t F);
size_t exact_bdigit_bytes(const EncodeDev& e, int64_t F);
// Ad (or nullptr): the digits of conj(A) in tile layout (adj_digit_bytes(), written
// by launch_adj_digits), copied instead of formed in every CTA.
size_t adj_digit_bytes(const EncodeDev& e);
cudaError_t launch_adj_digits(const EncodeDev& e, uint8_t* Ad, cudaStream_t s);
cudaError_t launch_adjoint_exact(const EncodeDev& e, const double2* D, int64_t F, int* fexp, uint8_t* Bd,
                                 double2* B, float4* work, DevStatus* st, cudaStream_t s,
                                 const uint8_t* Ad = nullptr);
cudaError_t launch_transpose_df(const float4* src, int64_t rows, int64_t cols, float4* dst, int64_t ldd,
                                cudaStream_t s);

// U = D - E X exactly on the tensor cores (D may be null: U = -E X), from the
// per-build digit table of A (fwd_digit_bytes(), launch_fwd_digits; rows of 128
// samples, k = voxels); Y: exact_fwd_y_elems() FP64 scratch for s_c o x, fexp [F],
// Bd: exact_fwd_bdigit_bytes(), work: exact_fwd_work_elems() partials (F >= 16,
// as exact_adjoint_ok).
size_t fwd_digit_bytes(const EncodeDev& e);
cudaError_t launch_fwd_digits(const EncodeDev& e, uint8_t* Af, cudaStream_t s);
size_t exact_fwd_work_elems(const EncodeDev& e, int64_t F);
size_t exact_fwd_bdigit_bytes(const EncodeDev& e, int64_t F);
size_t exact_fwd_y_elems(const EncodeDev& e, int64_t F);
cudaError_t launch_forward_exact(const EncodeDev& e, const double2* X, int64_t F, const double2* D, double2* U,
                                 const uint8_t* Af, double2* Y, int* fexp, uint8_t* Bd, float4* work,
                                 DevStatus* st, cudaStream_t s);
// R -= lam X over n entries (FP64)
cudaError_t launch_minus_lambda(double2* R, const double2* X, double lam, int64_t n, cudaStream_t s);

// Recon x data (c64) on the tensor cores, split-BF16, for F >= 16 frames (in
// chunks of 128); the sample range is split over tiles with FP32 partials in `work`.
bool apply_tc_ok(int64_t F);
size_t apply_tc_work_elems(int64_t N, int64_t M, int64_t F);
cudaError_t launch_apply_tc(const float2* R, int64_t N, int64_t M, const float2* D, int64_t F, float2* X,
                            float2* work, int slices, DevStatus* st, cudaStream_t s);

// r = b - G x exactly on the tensor cores, from digit tiles of the exact Gram
// (gram_digit_bytes(N) bytes, written by launch_gram_digits at build time)
size_t gram_digit_bytes(int64_t N);
cudaError_t launch_gram_digits(const float4* G, int64_t N, int* eG, uint8_t* Gd, cudaStream_t s);
size_t resid_exact_work_elems(int64_t N, int64_t F);
size_t resid_bdigit_bytes(int64_t N, int64_t F);  // Bd of launch_gram_resid_exact
cudaError_t launch_gram_resid_exact(const uint8_t* Gd, const int* eG, int64_t N, const double2* Bv,
                                    const double2* X, int64_t F, int* fexp, uint8_t* Bd, double2* R,
                                    float4* work, DevStatus* st, cudaStream_t s);

// exact Gram of B0-free grid plans (Toeplitz table summed in double-float, kept
// FP64; the Gram itself stored double-float). launch_toeplitz needs the
// double-float phase tables (exdf, eydf, ezdf).
size_t toeplitz_work_bytes(const EncodeDev& e);
cudaError_t launch_toeplitz(const EncodeDev& e, float4* work, double2* T, cudaStream_t s);
cudaError_t launch_gram_exact(const EncodeDev& e, const double2* T, double lam, float4* G, cudaStream_t s);
cudaError_t launch_gram_resid_df(const float4* G, int64_t N, const double2* B, const double2* X, int64_t F,
                                 double2* R, cudaStream_t s, float4* work);
cudaError_t launch_from_df(const float4* a, int64_t n, double2* b, cudaStream_t s);
cudaError_t launch_forward_df(const EncodeDev& e, const double2* X, int64_t F, const double2* D, double2* U,
                              cudaStream_t s, float4* work);
// R[f] = E^H U[f] - lam X[f] (X may be null), double-float arithmetic, FP64 in/out
cudaError_t launch_adjoint_df(const EncodeDev& e, const double2* U, int64_t F, double lam, const double2* X,
                              double2* R, cudaStream_t s, float4* work);
// X[f] += W^H (W R[f]) in FP32 with scratch T [F][N]
cudaError_t launch_correct32(const float2* W32, int64_t N, const double2* R, int64_t F, float2* T, double2* X,
                             cudaStream_t s);
// The same correction on the tensor cores (split-BF16, split-K with ordered
// partial sums; `work` of correct_tc_work_elems() float2), for 16 or more frames.
bool correct_tc_ok(int64_t F);
size_t correct_tc_work_elems(int64_t N, int64_t F);
cudaError_t launch_correct_tc(const float2* W32, int64_t N, const double2* R, int64_t F, float2* T, double2* X,
                              float2* work, int slices, DevStatus* sched, cudaStream_t s);

}  // namespace pinv
