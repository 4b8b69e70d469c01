// Double-float residual kernels for the mixed-precision refinement.
//
// The refinement needs r = E^H (d - E x) - lambda x far more accurately than
// FP32 (about 1e-10 relative for an image NRMSE of 1e-4 at kappa(G) ~ 1e6), but
// FP64 on GB300 issues at 1/64 of the FP32 rate. These kernels carry every
// value as an unevaluated sum of two floats (hi + lo, about 44 significant
// bits): products use the exact FMA product error, sums use TwoSum, and the
// accumulator keeps a compensated (hi, lo) pair. One complex MAC costs 48 FP32
// instructions, about 5x less time than 4 DFMAs. Encoding elements are
// generated from double-float phase tables, as the FP64 kernels generate them
// from FP64 tables; inputs and outputs stay FP64 in memory.
//
// The correction step x += W^H (W r) only preconditions the next residual, so
// it runs in plain FP32 (tile engine k_ctile).
#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cstring>

#include <cooperative_groups.h>

#include "df.cuh"

namespace pinv {

// ------------------------------------------------------------------ double-float tile engine
// C[i][j] = sum_k a(i,k) b(k,j) over rows i, frames j. With a split of the k
// range over blockIdx.z (part != nullptr), each CTA writes its unreduced
// double-float partial to part[z][j][i] and k_df_reduce adds the partials in
// order z = 0, 1, ...; the split count depends only on the problem size, so a
// given problem always sums in the same order whatever tile shape runs it.
template <int BM, int BN, int TM, int TN, class P, int BK = 16>
__global__ void __launch_bounds__(256) k_dftile(P p, float4* part, int64_t chunk, int64_t rows, int64_t F) {
    constexpr int TX = BN / TN, TY = BM / TM;
    static_assert(TX * TY == 256, "256 threads");
    __shared__ float4 As[BK][BM];
    __shared__ float4 Bs[BK][BN];
    const int64_t i0 = (int64_t)blockIdx.y * BM, j0 = (int64_t)blockIdx.x * BN;
    const int64_t K = p.K();
    const int64_t kb = (int64_t)blockIdx.z * chunk;
    const int64_t ke = kb + chunk < K ? kb + chunk : K;
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    float4 acc[TM][TN];
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[r][c] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t k0 = kb; k0 < ke; k0 += BK) {
        for (int e = tid; e < BK * BM; e += 256) {
            const int ii = e % BM, kk = e / BM;
            const int64_t gi = i0 + ii, gk = k0 + kk;
            As[kk][ii] = (gk < ke && p.a_ok(gi)) ? p.a(gi, gk) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int e = tid; e < BK * BN; e += 256) {
            const int kk = e % BK, jj = e / BK;
            const int64_t gj = j0 + jj, gk = k0 + kk;
            Bs[kk][jj] = (gk < ke && p.b_ok(gj)) ? p.b(gk, gj) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncthreads();
#pragma unroll 2
        for (int kk = 0; kk < BK; ++kk) {
            float4 av[TM], bv[TN];
#pragma unroll
            for (int r = 0; r < TM; ++r) av[r] = As[kk][ty + TY * r];
#pragma unroll
            for (int c = 0; c < TN; ++c) bv[c] = Bs[kk][tx + TX * c];
#pragma unroll
            for (int r = 0; r < TM; ++r)
#pragma unroll
                for (int c = 0; c < TN; ++c) cacc(acc[r][c], av[r], bv[c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) {
            const int64_t gi = i0 + ty + TY * r, gj = j0 + tx + TX * c;
            if (!(p.a_ok(gi) && p.b_ok(gj))) continue;
            if (part) part[((int64_t)blockIdx.z * F + gj) * rows + gi] = acc[r][c];
            else p.store(gi, gj, from_df(acc[r][c]));
        }
}

template <class P>
__global__ void k_df_reduce(P p, const float4* part, int splits, int64_t rows, int64_t F) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= rows * F) return;
    const int64_t i = idx % rows, j = idx / rows;
    float4 a = part[j * rows + i];
    for (int z = 1; z < splits; ++z) {
        const float4 b = part[((int64_t)z * F + j) * rows + i];
        float rh, rl, ih, il;
        df_add(a.x, a.y, b.x, b.y, rh, rl);
        df_add(a.z, a.w, b.z, b.w, ih, il);
        a = make_float4(rh, rl, ih, il);
    }
    p.store(i, j, from_df(a));
}

// U[f][(c,m)] = D[f][(c,m)] - sum_n E[(c,m)][n] X[f][n]
struct ForwardDF {
    EncodeDev e;
    const double2* X;
    const double2* D;
    double2* U;
    int64_t F;
    __device__ int64_t K() const { return e.N; }
    __device__ bool a_ok(int64_t i) const { return i < e.Mk * e.C; }
    __device__ bool b_ok(int64_t j) const { return j < F; }
    __device__ float4 a(int64_t i, int64_t k) const {
        const int c = (int)(i / e.Mk);
        return gen_e_df(e, c, i - (int64_t)c * e.Mk, k);
    }
    __device__ float4 b(int64_t k, int64_t j) const { return to_df(X[j * e.N + k]); }
    __device__ void store(int64_t i, int64_t j, double2 v) const {
        const int64_t M = e.Mk * e.C;
        U[j * M + i] = zsub(D[j * M + i], v);
    }
};

// R[f][n] = sum_{(c,m)} conj(E[(c,m)][n]) U[f][(c,m)] - lam X[f][n]
struct AdjointDF {
    EncodeDev e;
    const double2* U;
    const double2* X;
    double2* R;
    double lam;
    int64_t F;
    __device__ int64_t K() const { return e.Mk * e.C; }
    __device__ bool a_ok(int64_t i) const { return i < e.N; }
    __device__ bool b_ok(int64_t j) const { return j < F; }
    __device__ float4 a(int64_t i, int64_t k) const {
        const int c = (int)(k / e.Mk);
        return cdf_conj(gen_e_df(e, c, k - (int64_t)c * e.Mk, i));
    }
    __device__ float4 b(int64_t k, int64_t j) const { return to_df(U[j * (e.Mk * e.C) + k]); }
    __device__ void store(int64_t i, int64_t j, double2 v) const {
        if (X) {
            const double2 x = X[j * e.N + i];
            v.x -= lam * x.x;
            v.y -= lam * x.y;
        }
        R[j * e.N + i] = v;
    }
};

// Split count of the k range for a double-float frame product of `rows` rows,
// F frames and length K: about four CTAs per SM on a reference tiling of
// 16 x 64 (independent of the tuned shape), chunks of at least 512.
int df_splits(int64_t rows, int64_t F, int64_t K) {
    const int64_t tiles = ((rows + 15) / 16) * ((F + 63) / 64);
    int64_t sp = (600 + tiles - 1) / tiles;
    sp = std::min<int64_t>(sp, K / 512);
    sp = std::min<int64_t>(std::max<int64_t>(sp, 1), 32);
    return (int)sp;
}

size_t df_work_elems(int64_t rows, int64_t F, int64_t K) {
    const int sp = df_splits(rows, F, K);
    return sp > 1 ? (size_t)sp * (size_t)rows * (size_t)F : 0;
}

template <int BM, int BN, int TM, int TN, class P>
static cudaError_t df_shape(const P& p, int64_t rows, int64_t F, int sp, int64_t chunk, float4* work,
                            cudaStream_t s) {
    dim3 grid((unsigned)((F + BN - 1) / BN), (unsigned)((rows + BM - 1) / BM), (unsigned)sp);
    k_dftile<BM, BN, TM, TN, P><<<grid, 256, 0, s>>>(p, sp > 1 ? work : nullptr, chunk, rows, F);
    note_launch();
    return cudaGetLastError();
}

// Tile shape per frame-count class, chosen by the autotuner among candidates
// that all sum over k in the same order (same split, same chunks).
template <class P>
static cudaError_t launch_df(P p, int64_t rows, int64_t F, int64_t K, cudaStream_t s, const char* family,
                             float4* work) {
    const int sp = df_splits(rows, F, K);
    if (sp > 1 && !work) return cudaErrorInvalidValue;
    const int64_t chunk = ((K + sp - 1) / sp + 15) / 16 * 16;
    cudaError_t err;
    if (F >= 48) {
        auto run = [&](int c) -> cudaError_t {
            switch (c) {
                case 1: return df_shape<32, 64, 2, 4>(p, rows, F, sp, chunk, work, s);
                case 2: return df_shape<64, 64, 4, 4>(p, rows, F, sp, chunk, work, s);
                case 3: return df_shape<32, 32, 2, 2>(p, rows, F, sp, chunk, work, s);
                case 4: return df_shape<64, 32, 4, 2>(p, rows, F, sp, chunk, work, s);
                default: return df_shape<16, 64, 1, 4>(p, rows, F, sp, chunk, work, s);
            }
        };
        err = run(tune_pick(family, rows, F, 5, run, s));
    } else if (F >= 8) {
        auto run = [&](int c) -> cudaError_t {
            switch (c) {
                case 1: return df_shape<32, 16, 2, 1>(p, rows, F, sp, chunk, work, s);
                case 2: return df_shape<64, 16, 4, 1>(p, rows, F, sp, chunk, work, s);
                case 3: return df_shape<32, 32, 2, 2>(p, rows, F, sp, chunk, work, s);
                default: return df_shape<16, 16, 1, 1>(p, rows, F, sp, chunk, work, s);
            }
        };
        err = run(tune_pick(family, rows, F, 4, run, s));
    } else {
        auto run = [&](int c) -> cudaError_t {
            switch (c) {
                case 1: return df_shape<128, 4, 2, 1>(p, rows, F, sp, chunk, work, s);
                case 2: return df_shape<128, 2, 1, 1>(p, rows, F, sp, chunk, work, s);
                default: return df_shape<64, 4, 1, 1>(p, rows, F, sp, chunk, work, s);
            }
        };
        err = run(tune_pick(family, rows, F, 3, run, s));
    }
    if (err != cudaSuccess || sp == 1) return err;
    const int64_t n = rows * F;
    k_df_reduce<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, work, sp, rows, F);
    note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------ Toeplitz table
// (A^H A)[n][n'] depends only on the index offset (i_n - i_n') per axis for voxels
// on the grid without B0, so
//   T[dz][dy][dx] = sum_m q_x(m, dx) q_y(m, dy) q_z(m, dz),
//   q(m, d) = exp(+i 2 pi k_m d fov / n_axis),
// over offsets -(n-1)..(n-1) per axis ((2n-1) entries, dx fastest). q comes from the
// double-float phase table as conj(e[m][d]) e[m][0] (d >= 0) or conj(e[m][0])
// e[m][-d] (d < 0), i.e. from the same pair of encoding elements the Gram entry
// multiplies. The double-float tile engine sums over the samples, split over
// blockIdx.z into partials that k_df_reduce adds in split order (deterministic).
// T[-d] = conj(T[d]): the engine forms the columns d_yz >= 0 and the store writes
// each canonical entry and the conjugate of its mirror, so T is Hermitian to the bit.
__device__ inline float4 toep_q_df(const float4* tab, int n, int64_t m, int d) {
    if (n == 1) return make_float4(1.f, 0.f, 0.f, 0.f);
    const float4* row = tab + m * n;
    return d >= 0 ? cdf_mul(cdf_conj(row[d]), row[0]) : cdf_mul(cdf_conj(row[0]), row[-d]);
}
struct ToeplitzDF {
    EncodeDev e;
    double2* T;
    int64_t Tx, Ty, Tyz, jm;  // columns jm .. Tyz - 1 of T[d_yz][d_x]
    __device__ int64_t K() const { return e.Mk; }
    __device__ bool a_ok(int64_t i) const { return i < Tx; }
    __device__ bool b_ok(int64_t j) const { return j < Tyz - jm; }
    __device__ float4 a(int64_t i, int64_t m) const { return toep_q_df(e.exdf, e.nx, m, (int)i - (e.nx - 1)); }
    __device__ float4 b(int64_t m, int64_t j) const {
        const int64_t jj = j + jm;
        const int dy = (int)(jj % Ty) - (e.ny - 1), dz = (int)(jj / Ty) - (e.nz - 1);
        const float4 qy = toep_q_df(e.eydf, e.ny, m, dy);
        return e.nz > 1 ? cdf_mul(qy, toep_q_df(e.ezdf, e.nz, m, dz)) : qy;
    }
    // canonical entries (d_yz > 0, or d_yz = 0 and d_x >= 0) and their mirrors
    __device__ void store(int64_t i, int64_t j, double2 v) const {
        const int64_t jj = j + jm;
        if (jj == jm && i < (Tx - 1) / 2) return;
        T[jj * Tx + i] = v;
        const int64_t mi = Tx - 1 - i, mj = Tyz - 1 - jj;
        if (mi != i || mj != jj) T[mj * Tx + mi] = zconj(v);
    }
};

size_t toeplitz_work_bytes(const EncodeDev& e) {
    const int64_t Tx = 2 * e.nx - 1, Tyz = (2 * e.ny - 1) * (2 * e.nz - 1), jm = (Tyz - 1) / 2;
    return (size_t)64 * Tx * (Tyz - jm) * sizeof(float4);  // at most 64 partial tables
}

cudaError_t launch_toeplitz(const EncodeDev& e, float4* work, double2* T, cudaStream_t s) {
    if (!e.exdf || !e.eydf || !e.ezdf) return cudaErrorInvalidValue;
    const int64_t Tx = 2 * e.nx - 1, Ty = 2 * e.ny - 1, Tyz = Ty * (2 * e.nz - 1), jm = (Tyz - 1) / 2;
    const int64_t rows = Tx, F = Tyz - jm, K = e.Mk;
    // sample splits of about 128 samples (short CTAs: the table forms beside the
    // Cholesky, whose launches need the SMs back quickly), at most 64
    const int sp = (int)std::max<int64_t>(1, std::min<int64_t>(64, (K + 127) / 128));
    const int64_t chunk = ((K + sp - 1) / sp + 15) / 16 * 16;
    const ToeplitzDF p{e, T, Tx, Ty, Tyz, jm};
    cudaError_t err = df_shape<64, 64, 4, 4>(p, rows, F, sp, chunk, work, s);
    if (err != cudaSuccess || sp == 1) return err;
    const int64_t n = rows * F;
    k_df_reduce<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(p, work, sp, rows, F);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_forward_df(const EncodeDev& e, const double2* X, int64_t F, const double2* D, double2* U,
                              cudaStream_t s, float4* work) {
    if (F == 0) return cudaSuccess;
    return launch_df(ForwardDF{e, X, D, U, F}, e.Mk * e.C, F, e.N, s, "forward_df", work);
}

cudaError_t launch_adjoint_df(const EncodeDev& e, const double2* U, int64_t F, double lam, const double2* X,
                              double2* R, cudaStream_t s, float4* work) {
    if (F == 0) return cudaSuccess;
    return launch_df(AdjointDF{e, U, X, R, lam, F}, e.N, F, e.Mk * e.C, s, "adjoint_df", work);
}

// ------------------------------------------------------------------ exact Gram residual
// Exact Gram for B0-free plans, G[n][n'] = T[i_n - i_n'] sum_c conj(s_c(n)) s_c(n')
// + lambda delta, formed in double-float from the Toeplitz table and the
// double-float coil table (about 2^-45 relative; the FP64 pipe took six times as
// long) and stored as double-float pairs [N][N] (both triangles: the thread of
// n' <= n also writes the conjugate to G[n'][n], so G is Hermitian to the bit).
// The residual of the normal equations is then r = E^H d - G x with E^H d formed
// once per apply.
__global__ void k_gram_exact(EncodeDev e, const double2* T, double lam, float4* G) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // n'
    const int64_t i = blockIdx.y;                                         // n
    if (j > i) return;
    const int* gi = e.vox_ijk + 3 * i;
    const int* gj = e.vox_ijk + 3 * j;
    const int64_t Tx = 2 * e.nx - 1, Ty = 2 * e.ny - 1;
    const int64_t t = ((int64_t)(gi[2] - gj[2] + e.nz - 1) * Ty + (gi[1] - gj[1] + e.ny - 1)) * Tx +
                      (gi[0] - gj[0] + e.nx - 1);
    float4 v = to_df_i(T[t]);
    if (e.coilsdf) {
        float4 sc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int c = 0; c < e.C; ++c)
            cacc(sc, cdf_conj(e.coilsdf[(int64_t)c * e.N + i]), e.coilsdf[(int64_t)c * e.N + j]);
        v = cdf_mul(v, sc);
    } else if (e.coils) {
        double2 sc = make_double2(0.0, 0.0);
        for (int c = 0; c < e.C; ++c)
            zfma(sc, zconj(e.coils[(int64_t)c * e.N + i]), e.coils[(int64_t)c * e.N + j]);
        v = to_df_i(zmul(T[t], sc));
    }
    if (i == j) {
        const float2 l = f64_to_df_rn(lam);
        float rh, rl;
        df_add(v.x, v.y, l.x, l.y, rh, rl);
        v.x = rh;
        v.y = rl;
    }
    G[i * e.N + j] = v;
    if (j != i) G[j * e.N + i] = cdf_conj(v);
}

cudaError_t launch_gram_exact(const EncodeDev& e, const double2* T, double lam, float4* G, cudaStream_t s) {
    dim3 grid((unsigned)((e.N + 255) / 256), (unsigned)e.N);
    k_gram_exact<<<grid, 256, 0, s>>>(e, T, lam, G);
    note_launch();
    return cudaGetLastError();
}

// R[f][n] = B[f][n] - sum_n' G[n][n'] X[f][n'], G Hermitian (read as conj(G[n'][n]))
struct GramResidDF {
    const float4* G;
    const double2* B;
    const double2* X;
    double2* R;
    int64_t N, F;
    __device__ int64_t K() const { return N; }
    __device__ bool a_ok(int64_t i) const { return i < N; }
    __device__ bool b_ok(int64_t j) const { return j < F; }
    __device__ float4 a(int64_t i, int64_t k) const { return cdf_conj(G[k * N + i]); }
    __device__ float4 b(int64_t k, int64_t j) const { return to_df(X[j * N + k]); }
    __device__ void store(int64_t i, int64_t j, double2 v) const { R[j * N + i] = zsub(B[j * N + i], v); }
};

cudaError_t launch_gram_resid_df(const float4* G, int64_t N, const double2* B, const double2* X, int64_t F,
                                 double2* R, cudaStream_t s, float4* work) {
    if (F == 0) return cudaSuccess;
    return launch_df(GramResidDF{G, B, X, R, N, F}, N, F, N, s, "gram_resid_df", work);
}

__global__ void k_from_df(const float4* a, int64_t n, double2* b) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = from_df(a[i]);
}

cudaError_t launch_from_df(const float4* a, int64_t n, double2* b, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_from_df<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(a, n, b);
    note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------ diagonal Cholesky blocks
// The mixed path's 64 x 64 diagonal blocks: G_kk = L_kk L_kk^H and
// Dinv = L_kk^-1, in double-float (about 44 significant bits) on the FP32
// units. GB300 issues about 2 DFMA per clock per SM, so the same block in FP64
// takes ~5x longer, and these blocks are the sequential chain of the blocked
// Cholesky. G is in double-float storage throughout the mixed factorisation
// (df_of_f32 / df_sub_f32), so the block enters and leaves as it is.
namespace {
constexpr int NBD = 64;
constexpr int NBDP = NBD + 1;  // padded row stride of the shared-memory blocks
constexpr int DIAG_THREADS = 1024;
__device__ inline float4 df_scale(float4 a, float rh, float rl) {  // complex DF times real DF
    float xh, xl, yh, yl;
    df_mul(a.x, a.y, rh, rl, xh, xl);
    df_mul(a.z, a.w, rh, rl, yh, yl);
    return make_float4(xh, xl, yh, yl);
}
__device__ inline float4 df_norm(float4 a) {  // renormalise both (hi, lo) pairs
    float h, l;
    fast_two_sum(a.x, a.y, h, l);
    a.x = h;
    a.y = l;
    fast_two_sum(a.z, a.w, h, l);
    a.z = h;
    a.w = l;
    return a;
}
}  // namespace

// 1 / sqrt(d) for a positive double-float d: FP32 estimate and one Newton
// step in double-float (error about the square of the estimate's, ~2^-44)
__device__ inline float2 df_rsqrt(float dh, float dl) {
    const float r0 = rsqrtf(dh);
    float sh, sl, th, tl, uh, ul;
    df_mul(r0, 0.f, r0, 0.f, sh, sl);          // r0^2
    df_mul(dh, dl, sh, sl, th, tl);            // d r0^2
    df_add(1.f, 0.f, -th, -tl, uh, ul);        // 1 - d r0^2
    df_mul(uh, ul, 0.5f * r0, 0.f, th, tl);    // r0 (1 - d r0^2) / 2
    df_add(r0, 0.f, th, tl, uh, ul);
    return make_float2(uh, ul);
}

// Column sweep over the 64 x 64 block, factor and inverse together (both
// right-looking). Step j:
//  (a) the 64 threads of the first two warps each form r = 1 / sqrt(A_jj) from
//      the broadcast pivot (the same value in every thread, so no barrier);
//      thread i > j scales L_ij = A_ij r, thread c <= j scales row j of
//      X = L^-1 (X_jc *= r: row j of X is then final);
//  (b) thread j writes L_jj (nothing reads A_jj any more), and the threads
//      update every entry (i, c), c <= i, of the rows i > j: c <= j is
//      X_ic -= L_ij X_jc, c > j is A_ic -= L_ij conj(L_cj). Row j + 1 + p is
//      paired with row 63 - p, so each pair holds j + 66 entries and the
//      threads run over pairs without idle lanes.
// Two barriers per column. Rows are NBDP = 65 entries apart, so row and column
// reads are free of bank conflicts. The block is read from and L written back to
// G in double-float storage. Dinv may be null (the FP32 inverse alone); L32 (or
// null) receives the block of L rounded to FP32.
__global__ void __launch_bounds__(DIAG_THREADS) k_potrf_diag_df(float4* G, int64_t ld, int64_t N, int64_t k0,
                                                             double2* Dinv, float2* Dinv32, float2* L32,
                                                             int64_t ldl, DevStatus* st) {
    extern __shared__ float4 smd[];
    float4* A = smd;               // [NBD][NBDP]
    float4* X = smd + NBD * NBDP;  // [NBD][NBDP] inverse
    __shared__ int bad;
    const int tid = threadIdx.x;
    const int nb = (int)((N - k0) < NBD ? (N - k0) : NBD);
    if (tid == 0) bad = (st->not_pd_pivot != INT_MAX) ? 1 : 0;
#pragma unroll
    for (int e = tid; e < NBD * NBD; e += DIAG_THREADS) {
        const int i = e / NBD, j = e % NBD;
        float4 v = make_float4(i == j ? 1.f : 0.f, 0.f, 0.f, 0.f);
        if (i < nb && j < nb && j <= i) v = G[(k0 + i) * ld + k0 + j];
        A[i * NBDP + j] = v;
        X[i * NBDP + j] = make_float4(i == j ? 1.f : 0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();

    for (int j = 0; j < NBD; ++j) {
        float lh = 0.f, ll = 0.f;  // L_jj in thread j
        if (tid < NBD) {
            const float4 a = A[j * NBDP + j];
            float dh = a.x, dl = a.y;
            const bool fail = !(dh > 0.f) || !isfinite(dh);  // a normalised pair has the sign of dh
            if (fail) {
                dh = 1.f;
                dl = 0.f;
            }
            const float2 r = df_rsqrt(dh, dl);
            if (tid > j) {
                A[tid * NBDP + j] = df_norm(df_scale(A[tid * NBDP + j], r.x, r.y));
            } else {
                X[j * NBDP + tid] = df_norm(df_scale(X[j * NBDP + tid], r.x, r.y));
                if (tid == j) {
                    if (fail && !bad) {
                        atomicMin(&st->not_pd_pivot, (int)(k0 + j));
                        bad = 1;
                    }
                    df_mul(dh, dl, r.x, r.y, lh, ll);  // L_jj = d / sqrt(d)
                }
            }
        }
        __syncthreads();
        if (tid == j) A[j * NBDP + j] = make_float4(lh, ll, 0.f, 0.f);
        const int rows = NBD - 1 - j, w = j + 66;  // rows below; entries per row pair
        const int slots = ((rows + 1) >> 1) * w;
        const unsigned wm = ((1u << 20) + (unsigned)w - 1u) / (unsigned)w;  // e / w = (e wm) >> 20 for e < 2^20 / w
        for (int e = tid; e < slots; e += DIAG_THREADS) {
            const int p = (int)(((unsigned)e * wm) >> 20);
            const int q = e - p * w;
            const int ia = j + 1 + p, ib = NBD - 1 - p;
            const bool first = q <= ia;
            const int i = first ? ia : ib, c = first ? q : q - ia - 1;
            if (!first && ib <= ia) continue;  // the middle row of an odd count has no partner
            const bool xs = c <= j;
            float4* t = (xs ? X : A) + i * NBDP + c;
            float4 b = xs ? X[j * NBDP + c] : A[c * NBDP + j];
            if (!xs) b = cdf_conj(b);
            const float4 l = A[i * NBDP + j];
            float4 v = *t;
            cacc(v, make_float4(-l.x, -l.y, -l.z, -l.w), b);
            *t = df_norm(v);
        }
        __syncthreads();
    }
#pragma unroll
    for (int e = tid; e < NBD * NBD; e += DIAG_THREADS) {
        const int i = e / NBD, j = e % NBD;
        const float4 x = j <= i ? X[i * NBDP + j] : make_float4(0.f, 0.f, 0.f, 0.f);
        if (Dinv) Dinv[e] = make_double2(join_f64(x.x, x.y), join_f64(x.z, x.w));
        if (Dinv32) Dinv32[e] = make_float2(x.x + x.y, x.z + x.w);
        if (i < nb && j < nb && j <= i) {
            const float4 a = A[i * NBDP + j];
            G[(k0 + i) * ld + k0 + j] = a;
            if (L32) L32[(k0 + i) * ldl + k0 + j] = df_to_f32(a);
        } else if (L32 && i < nb && j < nb) {
            L32[(k0 + i) * ldl + k0 + j] = make_float2(0.f, 0.f);
        }
    }
}

// The same block on a cluster of two CTAs with a one-column lookahead: rank 0
// factors, rank 1 forms the inverse X = L^-1 behind it. Each rank splits its
// 32 warps: the first two finish the next column (rank 0) or row (rank 1), the
// critical path; the next 28 apply the current column's term to everything
// beyond it, each thread to the two or three entries it keeps in registers;
// on rank 0 the last two warps take turns to raise rank 1's flags after the
// barriers (a release at cluster scope takes about 450 cycles, which the
// barrier would otherwise wait for). One block barrier per column.
//
// Rank 0, step j (columns 0..j of L final, column j + 1 holding the terms of
// columns 0..j-1): every thread i of the first two warps forms the pivot
// d = A_{j+1,j+1} - |L_{j+1,j}|^2 and r = 1 / sqrt(d) (the same value in each,
// so no barrier), and thread i > j + 1 finishes its entry of column j + 1,
// L_{i,j+1} = r (A_{i,j+1} - L_ij conj(L_{j+1,j})), and stores it also into rank
// 1's shared memory (posted remote stores; thread j + 1 stores r). Meanwhile
// the other warps subtract column j's term from the entries (i, c), c >= j + 2,
// and store an entry to shared memory after its last such term (c = j + 2),
// where step c - 1 reads it. After the barrier one of the last two warps raises
// a flag in rank 1 (release at cluster scope): columns 0..j+1 have arrived.
//
// Rank 1, step j (rows 0..j of X final): thread c <= j + 1 of the first two
// warps waits for column j + 1 (acquire; bounded, about 2 s, past the limit it
// records timeout site DIAG_SITE and the rank stops, still meeting rank 0 at the
// final cluster barrier) and forms X_{j+1,c} = r_{j+1} (Y_{j+1,c} - L_{j+1,j}
// X_jc), Y = I minus the terms applied so far; the other warps subtract row j's
// term from the rows below row j + 1, Y_ic -= L_ij X_jc.
//
// Every entry takes the same operations in the same order as in the one-CTA
// sweep above (right-looking, one term per column, renormalised after each),
// only spread differently over threads.
constexpr int DIAG_SITE = 20;
constexpr long long DIAG_WAIT_LIMIT = 4000000000LL;
constexpr int DCW = 64;                          // critical threads: the first two warps
constexpr int DUT = DIAG_THREADS - DCW - 64;     // update threads: the next 28 warps (896)
constexpr int DSIG = DIAG_THREADS - 64;          // rank 0: flag raisers, DSIG (even counts), DSIG + 32 (odd)
constexpr int DUE = 3;                           // entries per update thread
constexpr int DNE = (NBD - 2) * (NBD - 1) / 2;   // 1953 entries updated off the critical path
static_assert(DNE <= DUE * DUT, "update entries per thread");
// A (rank 0) or X (rank 1); Lb[j][i] = L_ij and r_j received by rank 1; L_jj on rank 0
constexpr size_t DIAG2_SMEM = (size_t)(NBD * NBDP + NBD * NBD) * sizeof(float4) + 2 * NBD * sizeof(float2);

__device__ inline void st_release_cluster(unsigned* p, unsigned v) {
    asm volatile("st.release.cluster.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ inline unsigned ld_acquire_cluster(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.cluster.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// rank 1: wait until rank 0 has published `need` columns (the larger of the two
// flags; `seen` keeps the count this thread has acquired, so most steps need no
// load); false on timeout
__device__ inline bool diag_wait(const unsigned* flag, unsigned need, unsigned& seen, DevStatus* st) {
    if (seen >= need) return true;
    const long long t0 = clock64();
    for (;;) {
        const unsigned a = ld_acquire_cluster(flag), b = ld_acquire_cluster(flag + 1);
        seen = a > b ? a : b;
        if (seen >= need) return true;
        if (clock64() - t0 > DIAG_WAIT_LIMIT) {
            atomicMax(&st->timeout_site, DIAG_SITE);
            return false;
        }
    }
}
// e = r (r + 1) / 2 + q with 0 <= q <= r (row r, column q of a lower triangle)
__device__ inline void tri_index(int e, int& r, int& q) {
    r = (int)((sqrtf(8.f * (float)e + 1.f) - 1.f) * 0.5f);
    while (r * (r + 1) / 2 > e) --r;
    while ((r + 1) * (r + 2) / 2 <= e) ++r;
    q = e - r * (r + 1) / 2;
}
__device__ inline float4 cdf_neg(float4 a) { return make_float4(-a.x, -a.y, -a.z, -a.w); }

__global__ void __cluster_dims__(2, 1, 1) __launch_bounds__(DIAG_THREADS)
    k_potrf_diag_df2(float4* G, int64_t ld, int64_t N, int64_t k0, double2* Dinv, float2* Dinv32, float2* L32,
                     int64_t ldl, DevStatus* st) {
    namespace cg = cooperative_groups;
    cg::cluster_group cl = cg::this_cluster();
    extern __shared__ float4 smd[];
    float4* A = smd;                                        // rank 0: the block, then L; rank 1: Y, then X
    float4* Lb = smd + NBD * NBDP;                          // rank 1: Lb[j][i] = L_ij
    float2* rb = reinterpret_cast<float2*>(Lb + NBD * NBD);  // rank 1: r_j
    float2* Ld = rb + NBD;                                  // rank 0: L_jj
    __shared__ unsigned flag[2];  // rank 1: columns of L published by rank 0 (even, odd counts)
    __shared__ int stop;
    const int tid = threadIdx.x;
    const unsigned rank = cl.block_rank();
    const int nb = (int)((N - k0) < NBD ? (N - k0) : NBD);
    griddep_wait();    // the block's updates have landed
    griddep_launch();  // the next kernel's CTAs may take their SMs and wait for this one
    if (tid == 0) {
        flag[0] = flag[1] = 0;
        stop = 0;
    }
    {  // the block's lower triangle (rank 0) or I (rank 1); all loads issued before the stores
        constexpr int PER = NBD * NBD / DIAG_THREADS;
        float4 g[PER];
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            const int e = tid + t * DIAG_THREADS, i = e / NBD, j = e % NBD;
            g[t] = (rank == 0 && i < nb && j < nb && j <= i) ? G[(k0 + i) * ld + k0 + j]
                                                              : make_float4(i == j ? 1.f : 0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int t = 0; t < PER; ++t) {
            const int e = tid + t * DIAG_THREADS, i = e / NBD, j = e % NBD;
            A[i * NBDP + j] = g[t];
        }
    }
    // the entries this thread updates off the critical path; rank 0: (i, c), 2 <= c <= i,
    // numbered from the last column; rank 1: (i, c), c <= i - 2, numbered by row from row 2
    const int u = tid - DCW;
    int ui[DUE], uc[DUE];
#pragma unroll
    for (int k = 0; k < DUE; ++k) {
        const int e = u + k * DUT;
        ui[k] = -1;
        uc[k] = -1;
        if (u >= 0 && u < DUT && e < DNE) {
            int r, q;
            tri_index(e, r, q);
            if (rank == 0) {
                uc[k] = NBD - 1 - r;
                ui[k] = uc[k] + q;
            } else {
                ui[k] = r + 2;
                uc[k] = q;
            }
        }
    }
    cl.sync();  // the blocks are loaded and rank 1's flag is zero before rank 0 may raise it
    float4 uv[DUE];
#pragma unroll
    for (int k = 0; k < DUE; ++k) uv[k] = ui[k] >= 0 ? A[ui[k] * NBDP + uc[k]] : make_float4(0.f, 0.f, 0.f, 0.f);
    if (rank == 0) {
        unsigned* rflag = cl.map_shared_rank(flag, 1);
        float4* rLb = cl.map_shared_rank(Lb, 1);
        float2* rrb = cl.map_shared_rank(rb, 1);
        // column 0
        if (tid < DCW) {
            const float4 a = A[0];
            float dh = a.x, dl = a.y;
            const bool fail = !(dh > 0.f) || !isfinite(dh);  // a normalised pair has the sign of dh
            if (fail) {
                dh = 1.f;
                dl = 0.f;
            }
            const float2 r = df_rsqrt(dh, dl);
            if (tid > 0) {
                const float4 l = df_norm(df_scale(A[tid * NBDP], r.x, r.y));
                A[tid * NBDP] = l;
                rLb[tid] = l;
            } else {
                if (fail) atomicMin(&st->not_pd_pivot, (int)k0);
                float lh, ll;
                df_mul(dh, dl, r.x, r.y, lh, ll);
                Ld[0] = make_float2(lh, ll);
                rrb[0] = r;
            }
        }
        __syncthreads();
        if (tid == DSIG + 32) st_release_cluster(rflag + 1, 1u);
        for (int j = 0; j + 1 < NBD; ++j) {
            if (tid < DCW) {
                if (tid > j) {  // rows j + 1 .. 63 of column j + 1
                    // the entry's update first: it does not wait for the pivot, and the
                    // two chains interleave (thread j + 1's entry is the pivot itself)
                    const float4 lj = A[(j + 1) * NBDP + j];  // L_{j+1,j}
                    float4 v = A[tid * NBDP + j + 1];
                    float4 dd = A[(j + 1) * NBDP + j + 1];
                    cacc(v, cdf_neg(A[tid * NBDP + j]), cdf_conj(lj));
                    cacc(dd, cdf_neg(lj), cdf_conj(lj));
                    v = df_norm(v);
                    dd = df_norm(dd);
                    float dh = dd.x, dl = dd.y;
                    const bool fail = !(dh > 0.f) || !isfinite(dh);
                    if (fail) {
                        dh = 1.f;
                        dl = 0.f;
                    }
                    const float2 r = df_rsqrt(dh, dl);
                    if (tid > j + 1) {
                        const float4 l = df_norm(df_scale(v, r.x, r.y));
                        A[tid * NBDP + j + 1] = l;
                        rLb[(j + 1) * NBD + tid] = l;
                    } else {
                        if (fail) atomicMin(&st->not_pd_pivot, (int)(k0 + j + 1));
                        float lh, ll;
                        df_mul(dh, dl, r.x, r.y, lh, ll);
                        Ld[j + 1] = make_float2(lh, ll);
                        rrb[j + 1] = r;
                    }
                }
            } else {
#pragma unroll
                for (int k = 0; k < DUE; ++k) {
                    if (uc[k] >= j + 2) {
                        cacc(uv[k], cdf_neg(A[ui[k] * NBDP + j]), cdf_conj(A[uc[k] * NBDP + j]));
                        uv[k] = df_norm(uv[k]);
                        if (uc[k] == j + 2) A[ui[k] * NBDP + uc[k]] = uv[k];
                    }
                }
            }
            __syncthreads();
            // columns 0..j+1; each raiser has two steps for its release
            if (tid == DSIG + 32 * (j & 1)) st_release_cluster(rflag + (j & 1), (unsigned)(j + 2));
        }
        for (int e = tid; e < NBD * NBD; e += DIAG_THREADS) {
            const int i = e / NBD, j = e % NBD;
            if (i < nb && j < nb && j <= i) {
                const float4 a = i == j ? make_float4(Ld[j].x, Ld[j].y, 0.f, 0.f) : A[i * NBDP + j];
                G[(k0 + i) * ld + k0 + j] = a;
                if (L32) L32[(k0 + i) * ldl + k0 + j] = df_to_f32(a);
            } else if (L32 && i < nb && j < nb) {
                L32[(k0 + i) * ldl + k0 + j] = make_float2(0.f, 0.f);
            }
        }
        cl.sync();
    } else {
        float4* X = A;
        float4 xp = make_float4(0.f, 0.f, 0.f, 0.f);  // thread c < 64: X_jc of the current step
        unsigned seen = 0;
        if (tid < DCW) {
            if (!diag_wait(flag, 1u, seen, st)) {
                stop = 1;
            } else if (tid == 0) {
                const float2 r = rb[0];
                xp = df_norm(df_scale(X[0], r.x, r.y));
                X[0] = xp;
            }
        }
        __syncthreads();
        for (int j = 0; j + 1 < NBD; ++j) {
            if (stop) break;  // set before the last barrier: the same in every thread
            if (tid < DCW) {
                if (tid <= j + 1) {  // row j + 1, columns 0 .. j + 1
                    if (!diag_wait(flag, (unsigned)(j + 2), seen, st)) {
                        stop = 1;
                    } else {
                        const float2 r = rb[j + 1];
                        float4 y = X[(j + 1) * NBDP + tid];
                        if (tid <= j) {
                            cacc(y, cdf_neg(Lb[j * NBD + j + 1]), xp);
                            y = df_norm(y);
                        }
                        xp = df_norm(df_scale(y, r.x, r.y));
                        X[(j + 1) * NBDP + tid] = xp;
                    }
                }
            } else {
#pragma unroll
                for (int k = 0; k < DUE; ++k) {
                    if (uc[k] >= 0 && uc[k] <= j && ui[k] >= j + 2) {
                        cacc(uv[k], cdf_neg(Lb[j * NBD + ui[k]]), X[j * NBDP + uc[k]]);
                        uv[k] = df_norm(uv[k]);
                        if (ui[k] == j + 2) X[ui[k] * NBDP + uc[k]] = uv[k];
                    }
                }
            }
            __syncthreads();
        }
        cl.sync();  // rank 0 has published everything and may exit
        for (int e = tid; e < NBD * NBD; e += DIAG_THREADS) {
            const int i = e / NBD, j = e % NBD;
            const float4 x = j <= i ? X[i * NBDP + j] : make_float4(0.f, 0.f, 0.f, 0.f);
            if (Dinv) Dinv[e] = make_double2(join_f64(x.x, x.y), join_f64(x.z, x.w));
            if (Dinv32) Dinv32[e] = make_float2(x.x + x.y, x.z + x.w);
        }
    }
}

cudaError_t launch_potrf_diag_df(float4* G, int64_t ld, int64_t N, int64_t k0, double2* Dinv, float2* Dinv32,
                                 float2* L32, int64_t ldl, DevStatus* st, cudaStream_t s) {
    // PINV_DIAG_CLUSTER=0: the one-CTA sweep (same results)
    const char* env = std::getenv("PINV_DIAG_CLUSTER");
    const bool cluster = !(env && std::strcmp(env, "0") == 0);
    static bool attr = false, attr2 = false;
    if (cluster) {
        const size_t smem2 = DIAG2_SMEM;
        if (!attr2) {
            cudaError_t err =
                cudaFuncSetAttribute(k_potrf_diag_df2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2);
            if (err != cudaSuccess) return err;
            attr2 = true;
        }
        cudaError_t err = launch_pdl(k_potrf_diag_df2, dim3(2), dim3(DIAG_THREADS), smem2, s, G, ld, N, k0, Dinv,
                                     Dinv32, L32, ldl, st);
        return err != cudaSuccess ? err : cudaGetLastError();
    }
    const size_t smem = 2 * NBD * NBDP * sizeof(float4);
    if (!attr) {
        cudaError_t err =
            cudaFuncSetAttribute(k_potrf_diag_df, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (err != cudaSuccess) return err;
        attr = true;
    }
    k_potrf_diag_df<<<1, DIAG_THREADS, smem, s>>>(G, ld, N, k0, Dinv, Dinv32, L32, ldl, st);
    note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------ FP32 correction x += W^H (W r)
template <int BM, int BN, int TM, int TN, class P, int BK = 16>
__global__ void __launch_bounds__(256) k_ctile(P p) {
    constexpr int TX = BN / TN, TY = BM / TM;
    static_assert(TX * TY == 256, "256 threads");
    __shared__ float2 As[BK][BM + 1];
    __shared__ float2 Bs[BK][BN + 1];
    const int64_t i0 = (int64_t)blockIdx.y * BM, j0 = (int64_t)blockIdx.x * BN;
    int64_t kb, ke;
    p.krange(i0, BM, kb, ke);
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    float2 acc[TM][TN];
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[r][c] = make_float2(0.f, 0.f);
    for (int64_t k0 = kb; k0 < ke; k0 += BK) {
        for (int e = tid; e < BK * BM; e += 256) {
            int ii, kk;
            if (P::A_KFAST) { kk = e % BK; ii = e / BK; } else { ii = e % BM; kk = e / BM; }
            const int64_t gi = i0 + ii, gk = k0 + kk;
            As[kk][ii] = (gk < ke && p.a_ok(gi)) ? p.a(gi, gk) : make_float2(0.f, 0.f);
        }
        for (int e = tid; e < BK * BN; e += 256) {
            const int kk = e % BK, jj = e / BK;
            const int64_t gj = j0 + jj, gk = k0 + kk;
            Bs[kk][jj] = (gk < ke && p.b_ok(gj)) ? p.b(gk, gj) : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < BK; ++kk) {
            float2 av[TM], bv[TN];
#pragma unroll
            for (int r = 0; r < TM; ++r) av[r] = As[kk][ty + TY * r];
#pragma unroll
            for (int c = 0; c < TN; ++c) bv[c] = Bs[kk][tx + TX * c];
#pragma unroll
            for (int r = 0; r < TM; ++r)
#pragma unroll
                for (int c = 0; c < TN; ++c) {
                    acc[r][c].x = fmaf(av[r].x, bv[c].x, fmaf(-av[r].y, bv[c].y, acc[r][c].x));
                    acc[r][c].y = fmaf(av[r].x, bv[c].y, fmaf(av[r].y, bv[c].x, acc[r][c].y));
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) {
            const int64_t gi = i0 + ty + TY * r, gj = j0 + tx + TX * c;
            if (p.a_ok(gi) && p.b_ok(gj)) p.store(gi, gj, acc[r][c]);
        }
}

// T[f][n] = sum_{k <= n} W[n][k] Rin[f][k]   (W lower, FP32; Rin FP64)
struct Trmv32 {
    static constexpr bool A_KFAST = true;
    const float2* W;
    const double2* Rin;
    float2* T;
    int64_t N, F;
    __device__ void krange(int64_t i0, int bm, int64_t& kb, int64_t& ke) const {
        kb = 0;
        ke = i0 + bm < N ? i0 + bm : N;
    }
    __device__ bool a_ok(int64_t i) const { return i < N; }
    __device__ bool b_ok(int64_t j) const { return j < F; }
    __device__ float2 a(int64_t i, int64_t k) const { return W[i * N + k]; }
    __device__ float2 b(int64_t k, int64_t j) const {
        const double2 v = Rin[j * N + k];
        return make_float2((float)v.x, (float)v.y);
    }
    __device__ void store(int64_t i, int64_t j, float2 v) const { T[j * N + i] = v; }
};

// X[f][n] += sum_{k >= n} conj(W[k][n]) T[f][k]
struct TrmvH32 {
    static constexpr bool A_KFAST = false;
    const float2* W;
    const float2* T;
    double2* X;
    int64_t N, F;
    __device__ void krange(int64_t i0, int bm, int64_t& kb, int64_t& ke) const {
        kb = i0;
        ke = N;
    }
    __device__ bool a_ok(int64_t i) const { return i < N; }
    __device__ bool b_ok(int64_t j) const { return j < F; }
    __device__ float2 a(int64_t i, int64_t k) const {
        const float2 w = W[k * N + i];
        return make_float2(w.x, -w.y);
    }
    __device__ float2 b(int64_t k, int64_t j) const { return T[j * N + k]; }
    __device__ void store(int64_t i, int64_t j, float2 v) const {
        double2 x = X[j * N + i];
        X[j * N + i] = make_double2(x.x + (double)v.x, x.y + (double)v.y);
    }
};

template <int BM, int BN, int TM, int TN, class P>
static cudaError_t c_shape(const P& p, int64_t rows, int64_t F, cudaStream_t s) {
    dim3 grid((unsigned)((F + BN - 1) / BN), (unsigned)((rows + BM - 1) / BM));
    k_ctile<BM, BN, TM, TN><<<grid, 256, 0, s>>>(p);
    note_launch();
    return cudaGetLastError();
}

// family != nullptr: autotuned (only for problems whose launches can be
// repeated, i.e. that overwrite their output)
template <class P>
static cudaError_t launch_c(P p, int64_t rows, int64_t F, cudaStream_t s, const char* family = nullptr) {
    if (F >= 48) {
        auto run = [&](int c) -> cudaError_t {
            switch (c) {
                case 1: return c_shape<32, 64, 2, 4>(p, rows, F, s);
                case 2: return c_shape<128, 64, 8, 4>(p, rows, F, s);
                default: return c_shape<64, 64, 4, 4>(p, rows, F, s);
            }
        };
        return run(family ? tune_pick(family, rows, F, 3, run, s) : 0);
    }
    if (F >= 8) {
        auto run = [&](int c) -> cudaError_t {
            switch (c) {
                case 1: return c_shape<32, 16, 2, 1>(p, rows, F, s);
                case 2: return c_shape<64, 16, 4, 1>(p, rows, F, s);
                default: return c_shape<16, 16, 1, 1>(p, rows, F, s);
            }
        };
        return run(family ? tune_pick(family, rows, F, 3, run, s) : 0);
    }
    auto run = [&](int c) -> cudaError_t {
        switch (c) {
            case 1: return c_shape<128, 4, 2, 1>(p, rows, F, s);
            default: return c_shape<64, 4, 1, 1>(p, rows, F, s);
        }
    };
    return run(family ? tune_pick(family, rows, F, 2, run, s) : 0);
}

cudaError_t launch_correct32(const float2* W32, int64_t N, const double2* R, int64_t F, float2* T, double2* X,
                             cudaStream_t s) {
    if (F == 0) return cudaSuccess;
    cudaError_t e = launch_c(Trmv32{W32, R, T, N, F}, N, F, s, "trmv32");
    if (e != cudaSuccess) return e;
    return launch_c(TrmvH32{W32, T, X, N, F}, N, F, s);
}

// ------------------------------------------------------------------ double-float tables
__global__ void k_to_df(const double2* __restrict__ a, float4* __restrict__ b, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = to_df(a[i]);
}
cudaError_t launch_to_df(const double2* src, float4* dst, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_to_df<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, dst, n);
    note_launch();
    return cudaGetLastError();
}

}  // namespace pinv
