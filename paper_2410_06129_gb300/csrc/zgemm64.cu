// FP64 complex tile engine and the FP64 path's contraction kernels.
//
// GB300 has few FP64 units (no FP64 tensor-core kind in tcgen05), so every
// FP64 contraction here is a SIMT DFMA kernel. One engine serves all of them:
// a CTA of 256 threads computes a BM x BN tile of C[i][j] = sum_k a(i,k) b(k,j)
// where a() and b() are operand functors that either read memory or generate
// encoding-matrix elements on the fly (the encoding matrix is never stored).
// Tiles are staged through shared memory BK = 16 at a time; each thread owns a
// TM x TN block of complex accumulators. The FP64 path is bound by the DFMA
// rate, not by memory, so the engine favours simplicity and zero waste on
// ragged edges (operands out of range load as zero, stores are predicated).
#include <algorithm>
#include <climits>

#include "pinv_internal.h"

namespace pinv {

constexpr int NB = 64;  // Cholesky / inverse block size

// lower-triangular tile enumeration: bid -> (ti, tj) with ti >= tj
__device__ inline void tri_index(int64_t bid, int& ti, int& tj) {
    int t = (int)((sqrt(8.0 * (double)bid + 1.0) - 1.0) * 0.5);
    while ((int64_t)(t + 1) * (t + 2) / 2 <= bid) ++t;
    while ((int64_t)t * (t + 1) / 2 > bid) --t;
    ti = t;
    tj = (int)(bid - (int64_t)t * (t + 1) / 2);
}

template <int BM, int BN, int TM, int TN, class P, int BK = 16>
__global__ void __launch_bounds__(256) k_ztile(P p) {
    constexpr int TX = BN / TN;
    constexpr int TY = BM / TM;
    static_assert(TX * TY == 256, "256 threads");
    __shared__ double2 As[BK][BM];
    __shared__ double2 Bs[BK][BN];
    int64_t i0, j0, kb, ke;
    if (!p.tile(i0, j0, kb, ke)) return;
    const int tid = threadIdx.x;
    const int tx = tid % TX, ty = tid / TX;
    double2 acc[TM][TN];
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[r][c] = make_double2(0.0, 0.0);

    for (int64_t k0 = kb; k0 < ke; k0 += BK) {
        for (int e = tid; e < BK * BM; e += 256) {
            int ii, kk;
            if (P::A_KFAST) { kk = e % BK; ii = e / BK; } else { ii = e % BM; kk = e / BM; }
            int64_t gi = i0 + ii, gk = k0 + kk;
            As[kk][ii] = (gk < ke && p.a_ok(gi)) ? p.a(gi, gk) : make_double2(0.0, 0.0);
        }
        for (int e = tid; e < BK * BN; e += 256) {
            int jj, kk;
            if (P::B_KFAST) { kk = e % BK; jj = e / BK; } else { jj = e % BN; kk = e / BN; }
            int64_t gj = j0 + jj, gk = k0 + kk;
            Bs[kk][jj] = (gk < ke && p.b_ok(gj)) ? p.b(gk, gj) : make_double2(0.0, 0.0);
        }
        __syncthreads();
#pragma unroll 4
        for (int kk = 0; kk < BK; ++kk) {
            double2 av[TM], bv[TN];
#pragma unroll
            for (int r = 0; r < TM; ++r) av[r] = As[kk][ty + TY * r];
#pragma unroll
            for (int c = 0; c < TN; ++c) bv[c] = Bs[kk][tx + TX * c];
#pragma unroll
            for (int r = 0; r < TM; ++r)
#pragma unroll
                for (int c = 0; c < TN; ++c) zfma(acc[r][c], av[r], bv[c]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) {
            int64_t gi = i0 + ty + TY * r, gj = j0 + tx + TX * c;
            if (p.a_ok(gi) && p.b_ok(gj)) p.store(gi, gj, acc[r][c]);
        }
}

// ---------------------------------------------------------------------------
// Gram: C[i][j] = sum_m conj(A[m][i]) A[m][j], lower tiles; epilogue multiplies
// by the coil Gram sum_c conj(s_c(i)) s_c(j) and adds lambda on the diagonal.
// ---------------------------------------------------------------------------
struct GramP {
    static constexpr bool A_KFAST = false, B_KFAST = false;
    EncodeDev e;
    double lam;
    double2* G;
    int64_t ld;
    __device__ bool tile(int64_t& i0, int64_t& j0, int64_t& kb, int64_t& ke) const {
        int ti, tj;
        tri_index(blockIdx.x, ti, tj);
        i0 = (int64_t)ti * 64;
        j0 = (int64_t)tj * 64;
        kb = 0;
        ke = e.Mk;
        return true;
    }
    __device__ bool a_ok(int64_t i) const { return i < e.N; }
    __device__ bool b_ok(int64_t j) const { return j < e.N; }
    __device__ double2 a(int64_t i, int64_t k) const { return zconj(gen_a64(e, k, i)); }
    __device__ double2 b(int64_t k, int64_t j) const { return gen_a64(e, k, j); }
    __device__ void store(int64_t i, int64_t j, double2 v) const {
        if (e.coils) {
            double2 sc = make_double2(0.0, 0.0);
            for (int c = 0; c < e.C; ++c)
                zfma(sc, zconj(e.coils[(int64_t)c * e.N + i]), e.coils[(int64_t)c * e.N + j]);
            v = zmul(v, sc);
        }
        if (i == j) v.x += lam;
        G[i * ld + j] = v;
    }
};

cudaError_t launch_gram64(const EncodeDev& e, double lambda, double2* G, int64_t ld, cudaStream_t s) {
    int64_t nt = (e.N + 63) / 64;
    GramP p{e, lambda, G, ld};
    k_ztile<64, 64, 4, 4><<<(unsigned)(nt * (nt + 1) / 2), 256, 0, s>>>(p);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Blocked Cholesky pieces
// ---------------------------------------------------------------------------
// panel solve: L[i][k0+j] = sum_k G[i][k0+k] conj(Dinv[j][k]) for rows i >= k0+NB
struct TrsmP {
    static constexpr bool A_KFAST = true, B_KFAST = true;
    double2* G;
    int64_t ld, N, k0, nbk;   // nbk = width of this panel
    const double2* Dinv;      // [NB][NB]
    __device__ bool tile(int64_t& i0, int64_t& j0, int64_t& kb, int64_t& ke) const {
        i0 = k0 + nbk + (int64_t)blockIdx.x * 64;
        j0 = 0;
        kb = 0;
        ke = nbk;
        return true;
    }
    __device__ bool a_ok(int64_t i) const { return i < N; }
    __device__ bool b_ok(int64_t j) const { return j < nbk; }
    __device__ double2 a(int64_t i, int64_t k) const { return G[i * ld + k0 + k]; }
    __device__ double2 b(int64_t k, int64_t j) const { return zconj(Dinv[j * NB + k]); }
    __device__ void store(int64_t i, int64_t j, double2 v) const { G[i * ld + k0 + j] = v; }
};

// trailing update: G[i][j] -= sum_k L[i][k0+k] conj(L[j][k0+k]) for lower tiles i,j >= t0
struct HerkP {
    static constexpr bool A_KFAST = true, B_KFAST = true;
    double2* G;
    int64_t ld, N, k0, nbk, t0;
    __device__ bool tile(int64_t& i0, int64_t& j0, int64_t& kb, int64_t& ke) const {
        int ti, tj;
        tri_index(blockIdx.x, ti, tj);
        i0 = t0 + (int64_t)ti * 64;
        j0 = t0 + (int64_t)tj * 64;
        kb = 0;
        ke = nbk;
        return true;
    }
    __device__ bool a_ok(int64_t i) const { return i < N; }
    __device__ bool b_ok(int64_t j) const { return j < N; }
    __device__ double2 a(int64_t i, int64_t k) const { return G[i * ld + k0 + k]; }
    __device__ double2 b(int64_t k, int64_t j) const { return zconj(G[j * ld + k0 + k]); }
    __device__ void store(int64_t i, int64_t j, double2 v) const {
        if (j <= i) G[i * ld + j] = zsub(G[i * ld + j], v);
    }
};

// Unblocked Cholesky of one diagonal block in shared memory, plus the inverse
// of the resulting triangular block (used by the panel solve and the inverse).
__global__ void __launch_bounds__(256) k_potrf_diag(double2* G, int64_t ld, int64_t N, int64_t k0,
                                                    double2* Dinv, float2* Dinv32, DevStatus* st) {
    extern __shared__ double2 sm[];
    double2* A = sm;               // [NB][NB]
    double2* X = sm + NB * NB;     // [NB][NB] inverse
    __shared__ int bad;
    const int tid = threadIdx.x;
    const int nb = (int)((N - k0) < NB ? (N - k0) : NB);
    if (tid == 0) bad = (st->not_pd_pivot != INT_MAX) ? 1 : 0;
    for (int e = tid; e < NB * NB; e += 256) {
        int i = e / NB, j = e % NB;
        double2 v = make_double2(i == j ? 1.0 : 0.0, 0.0);
        if (i < nb && j < nb && j <= i) v = G[(k0 + i) * ld + k0 + j];
        A[e] = v;
    }
    __syncthreads();
    // Right-looking, two barriers per column. Phase 1: thread 0 takes the
    // pivot (one rsqrt, no division) while the other threads scale the
    // previous column by its reciprocal pivot. Phase 2: the trailing update
    // uses the still unscaled column j with the factor 1 / d_j.
    __shared__ double rdiag[NB];  // 1 / L_jj
    for (int j = 0; j < NB; ++j) {
        if (tid == 0) {
            double d = A[j * NB + j].x;
            if (!(d > 0.0) || !isfinite(d)) {
                if (!bad) atomicMin(&st->not_pd_pivot, (int)(k0 + j));
                bad = 1;
                d = 1.0;
            }
            const double r = rsqrt(d);
            A[j * NB + j] = make_double2(d * r, 0.0);
            rdiag[j] = r;
        } else if (j > 0) {
            const double r = rdiag[j - 1];
            for (int i = j + tid - 1; i < NB; i += 255) {
                const double2 v = A[i * NB + j - 1];
                A[i * NB + j - 1] = make_double2(v.x * r, v.y * r);
            }
        }
        __syncthreads();
        const double r2 = rdiag[j] * rdiag[j];
        const int rem = NB - j - 1;
        for (int e = tid; e < rem * rem; e += 256) {
            const int i = j + 1 + e / rem, k = j + 1 + e % rem;
            if (k <= i) {
                const double2 a = A[i * NB + j];
                double2 v = A[i * NB + k];
                zfma(v, make_double2(-a.x * r2, -a.y * r2), zconj(A[k * NB + j]));
                A[i * NB + k] = v;
            }
        }
        __syncthreads();
    }
    // X = A^-1 by forward substitution down each column. Four lanes of one
    // warp share a column: each sums every fourth term of the row's dot
    // product (independent FMA chains), a shuffle combines them, and the
    // column's X values stay visible inside the warp.
    {
        const int c = tid >> 2, q = tid & 3;
        for (int i = 0; i < NB; ++i) {
            double2 part = make_double2(0.0, 0.0);
            if (i > c) {
                for (int k = c + q; k < i; k += 4) {
                    const double2 l = A[i * NB + k];
                    zfma(part, l, X[k * NB + c]);
                }
            }
            part.x += __shfl_xor_sync(0xffffffffu, part.x, 1);
            part.y += __shfl_xor_sync(0xffffffffu, part.y, 1);
            part.x += __shfl_xor_sync(0xffffffffu, part.x, 2);
            part.y += __shfl_xor_sync(0xffffffffu, part.y, 2);
            if (q == 0) {
                double2 v = make_double2(0.0, 0.0);
                if (i >= c) {
                    const double ri = rdiag[i];
                    v = make_double2(((i == c ? 1.0 : 0.0) - part.x) * ri, -part.y * ri);
                }
                X[i * NB + c] = v;
            }
            __syncwarp();
        }
    }
    __syncthreads();
    for (int e = tid; e < NB * NB; e += 256) {
        int i = e / NB, j = e % NB;
        Dinv[e] = X[e];
        if (Dinv32) Dinv32[e] = make_float2((float)X[e].x, (float)X[e].y);
        if (i < nb && j < nb && j <= i) G[(k0 + i) * ld + k0 + j] = A[e];
    }
}

cudaError_t launch_potrf_diag(double2* G, int64_t ld, int64_t N, int64_t k0, double2* Dinv,
                              float2* Dinv32, DevStatus* st, cudaStream_t s) {
    static bool attr = false;
    size_t smem = 2 * NB * NB * sizeof(double2);
    if (!attr) {
        cudaError_t err = cudaFuncSetAttribute(k_potrf_diag, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
        if (err != cudaSuccess) return err;
        attr = true;
    }
    k_potrf_diag<<<1, 256, smem, s>>>(G, ld, N, k0, Dinv, Dinv32, st);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_potrf64(double2* G, int64_t N, int64_t ld, double2* Dinv, DevStatus* st,
                           cudaStream_t s) {
    for (int64_t k0 = 0; k0 < N; k0 += NB) {
        int64_t nbk = std::min<int64_t>(NB, N - k0);
        double2* Dk = Dinv + (k0 / NB) * NB * NB;
        cudaError_t err = launch_potrf_diag(G, ld, N, k0, Dk, nullptr, st, s);
        if (err != cudaSuccess) return err;
        int64_t rest = N - k0 - nbk;
        if (rest <= 0) break;
        TrsmP tp{G, ld, N, k0, nbk, Dk};
        k_ztile<64, 64, 4, 4><<<(unsigned)((rest + 63) / 64), 256, 0, s>>>(tp);
        note_launch();
        int64_t nt = (rest + 63) / 64;
        HerkP hp{G, ld, N, k0, nbk, k0 + nbk};
        k_ztile<64, 64, 4, 4><<<(unsigned)(nt * (nt + 1) / 2), 256, 0, s>>>(hp);
        note_launch();
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Triangular inverse W = L^-1 by right-looking block forward substitution on
// the identity: W[kb] = Dinv[kb] W[kb]; then W[i] -= L[i][kb] W[kb] for i > kb.
// ---------------------------------------------------------------------------
struct TrtriDiagP {   // W[k0+i][j] = sum_k Dinv[i][k] W[k0+k][j], j < k0 + nbk
    static constexpr bool A_KFAST = true, B_KFAST = false;
    double2* W;
    int64_t ld, N, k0, nbk;
    const double2* Dinv;
    __device__ bool tile(int64_t& i0, int64_t& j0, int64_t& kb, int64_t& ke) const {
        i0 = 0;
        j0 = (int64_t)blockIdx.x * 64;
        kb = 0;
        ke = nbk;
        return true;
    }
    __device__ bool a_ok(int64_t i) const { return i < nbk; }
    __device__ bool b_ok(int64_t j) const { return j < k0 + nbk; }
    __device__ double2 a(int64_t i, int64_t k) const { return Dinv[i * NB + k]; }
    __device__ double2 b(int64_t k, int64_t j) const { return W[(k0 + k) * ld + j]; }
    __device__ void store(int64_t i, int64_t j, double2 v) const { W[(k0 + i) * ld + j] = v; }
};

struct TrtriUpdP {    // W[i][j] -= sum_k L[i][k0+k] W[k0+k][j], i >= k0+nbk, j < k0+nbk
    static constexpr bool A_KFAST = true, B_KFAST = false;
    double2* W;
    const double2* L;
    int64_t ld, N, k0, nbk;
    __device__ bool tile(int64_t& i0, int64_t& j0, int64_t& kb, int64_t& ke) const {
        i0 = k0 + nbk + (int64_t)blockIdx.y * 64;
        j0 = (int64_t)blockIdx.x * 64;
        kb = 0;
        ke = nbk;
        return true;
    }
    __device__ bool a_ok(int64_t i) const { return i < N; }
    __device__ bool b_ok(int64_t j) const { return j < k0 + nbk; }
    __device__ double2 a(int64_t i, int64_t k) const { return L[i * ld + k0 + k]; }
    __device__ double2 b(int64_t k, int64_t j) const { return W[(k0 + k) * ld + j]; }
    __device__ void store(int64_t i, int64_t j, double2 v) const {
        W[i * ld + j] = zsub(W[i * ld + j], v);
    }
};

cudaError_t launch_trtri64(const double2* L, int64_t N, int64_t ld, const double2* Dinv, double2* W,
                           cudaStream_t s) {
    cudaError_t err = launch_fill_identity(W, N, ld, s);
    if (err != cudaSuccess) return err;
    for (int64_t k0 = 0; k0 < N; k0 += NB) {
        int64_t nbk = std::min<int64_t>(NB, N - k0);
        const double2* Dk = Dinv + (k0 / NB) * NB * NB;
        int64_t ncol = k0 + nbk;
        TrtriDiagP dp{W, ld, N, k0, nbk, Dk};
        k_ztile<64, 64, 4, 4><<<(unsigned)((ncol + 63) / 64), 256, 0, s>>>(dp);
        note_launch();
        int64_t rest = N - k0 - nbk;
        if (rest <= 0) break;
        TrtriUpdP up{W, L, ld, N, k0, nbk};
        dim3 grid((unsigned)((ncol + 63) / 64), (unsigned)((rest + 63) / 64));
        k_ztile<64, 64, 4, 4><<<grid, 256, 0, s>>>(up);
        note_launch();
    }
    return cudaGetLastError();
}

// Ginv[i][j] = sum_{k >= max(i,j)} conj(W[k][i]) W[k][j], lower tiles, mirrored.
struct LauumP {
    static constexpr bool A_KFAST = false, B_KFAST = false;
    const double2* W;
    double2* Gi;
    int64_t ld, N;
    __device__ bool tile(int64_t& i0, int64_t& j0, int64_t& kb, int64_t& ke) const {
        int ti, tj;
        tri_index(blockIdx.x, ti, tj);
        i0 = (int64_t)ti * 64;
        j0 = (int64_t)tj * 64;
        kb = i0;
        ke = N;
        return true;
    }
    __device__ bool a_ok(int64_t i) const { return i < N; }
    __device__ bool b_ok(int64_t j) const { return j < N; }
    __device__ double2 a(int64_t i, int64_t k) const { return zconj(W[k * ld + i]); }
    __device__ double2 b(int64_t k, int64_t j) const { return W[k * ld + j]; }
    __device__ void store(int64_t i, int64_t j, double2 v) const {
        if (j <= i) {
            Gi[i * ld + j] = v;
            Gi[j * ld + i] = zconj(v);
        }
    }
};

cudaError_t launch_lauum64(const double2* W, int64_t N, int64_t ld, double2* Ginv, cudaStream_t s) {
    int64_t nt = (N + 63) / 64;
    LauumP p{W, Ginv, ld, N};
    k_ztile<64, 64, 4, 4><<<(unsigned)(nt * (nt + 1) / 2), 256, 0, s>>>(p);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Recon[n][(c,m)] = sum_n' Ginv[n][n'] conj(s_c(n') A[m][n'])   (Eq. 8)
// ---------------------------------------------------------------------------
struct ReconP {
    static constexpr bool A_KFAST = true, B_KFAST = true;
    EncodeDev e;
    const double2* Gi;
    int64_t ld;
    double2* R;
    __device__ bool tile(int64_t& i0, int64_t& j0, int64_t& kb, int64_t& ke) const {
        i0 = (int64_t)blockIdx.y * 64;
        j0 = (int64_t)blockIdx.x * 64;
        kb = 0;
        ke = e.N;
        return true;
    }
    __device__ bool a_ok(int64_t i) const { return i < e.N; }
    __device__ bool b_ok(int64_t j) const { return j < e.Mk * e.C; }
    __device__ double2 a(int64_t i, int64_t k) const { return Gi[i * ld + k]; }
    __device__ double2 b(int64_t k, int64_t j) const {
        int c = (int)(j / e.Mk);
        return zconj(gen_e64(e, c, j % e.Mk, k));
    }
    __device__ void store(int64_t i, int64_t j, double2 v) const { R[i * (e.Mk * e.C) + j] = v; }
};

cudaError_t launch_recon64(const EncodeDev& e, const double2* Ginv, int64_t ld, double2* R,
                           cudaStream_t s) {
    int64_t M = e.Mk * e.C;
    ReconP p{e, Ginv, ld, R};
    dim3 grid((unsigned)((M + 63) / 64), (unsigned)((e.N + 63) / 64));
    k_ztile<64, 64, 4, 4><<<grid, 256, 0, s>>>(p);
    note_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Batched products with frames: tile width chosen from the frame count so a
// single frame does not pay for 64 (FP64 units are the bottleneck).
// ---------------------------------------------------------------------------
template <class P>
static cudaError_t launch_frames(P p, int64_t rows, int64_t F, cudaStream_t s) {
    // 16-row tiles: the FP64 units, not shared memory, bound these kernels, so
    // narrow tiles cost nothing per flop and give N / 16 CTAs instead of N / 64
    if (F >= 48) {
        dim3 grid((unsigned)((F + 63) / 64), (unsigned)((rows + 15) / 16));
        k_ztile<16, 64, 1, 4><<<grid, 256, 0, s>>>(p);
        note_launch();
    } else if (F >= 8) {
        dim3 grid((unsigned)((F + 15) / 16), (unsigned)((rows + 15) / 16));
        k_ztile<16, 16, 1, 1><<<grid, 256, 0, s>>>(p);
        note_launch();
    } else {
        dim3 grid((unsigned)F, (unsigned)((rows + 255) / 256));
        k_ztile<256, 1, 1, 1, P, 8><<<grid, 256, 0, s>>>(p);
        note_launch();
    }
    return cudaGetLastError();
}

// tile(): rows from blockIdx.y * bm, frames from blockIdx.x * bn, where
// (bm, bn) is the shape frame_shape() picked for the launch.
__device__ inline void frame_tile(int64_t rows_per_tile, int64_t cols_per_tile, int64_t& i0,
                                  int64_t& j0) {
    i0 = (int64_t)blockIdx.y * rows_per_tile;
    j0 = (int64_t)blockIdx.x * cols_per_tile;
}

// X[f][n] = sum_j R[n][j] D[f][j]
struct ApplyP {
    static constexpr bool A_KFAST = true, B_KFAST = true;
    const double2* R;
    const double2* D;
    double2* X;
    int64_t N, M, F, bm, bn;
    __device__ bool tile(int64_t& i0, int64_t& j0, int64_t& kb, int64_t& ke) const {
        frame_tile(bm, bn, i0, j0);
        kb = 0;
        ke = M;
        return true;
    }
    __device__ bool a_ok(int64_t i) const { return i < N; }
    __device__ bool b_ok(int64_t j) const { return j < F; }
    __device__ double2 a(int64_t i, int64_t k) const { return R[i * M + k]; }
    __device__ double2 b(int64_t k, int64_t j) const { return D[j * M + k]; }
    __device__ void store(int64_t i, int64_t j, double2 v) const { X[j * N + i] = v; }
};

static void frame_shape(int64_t F, int64_t& bm, int64_t& bn) {
    if (F >= 48) { bm = 16; bn = 64; }
    else if (F >= 8) { bm = 16; bn = 16; }
    else { bm = 256; bn = 1; }
}

cudaError_t launch_apply64(const double2* R, int64_t N, int64_t M, const double2* D, int64_t F,
                           double2* X, cudaStream_t s) {
    if (F == 0) return cudaSuccess;
    int64_t bm, bn;
    frame_shape(F, bm, bn);
    ApplyP p{R, D, X, N, M, F, bm, bn};
    return launch_frames(p, N, F, s);
}

// Y[f][n] = sum_{(c,m)} conj(s_c(n) A[m][n]) D[f][(c,m)] - lam * Xs[f][n]
struct AdjointP {
    static constexpr bool A_KFAST = false, B_KFAST = true;
    EncodeDev e;
    const double2* D;
    const double2* Xs;
    double2* Y;
    double lam;
    int64_t F, bm, bn;
    __device__ bool tile(int64_t& i0, int64_t& j0, int64_t& kb, int64_t& ke) const {
        frame_tile(bm, bn, i0, j0);
        kb = 0;
        ke = e.Mk * e.C;
        return true;
    }
    __device__ bool a_ok(int64_t i) const { return i < e.N; }
    __device__ bool b_ok(int64_t j) const { return j < F; }
    __device__ double2 a(int64_t i, int64_t k) const {
        int c = (int)(k / e.Mk);
        return zconj(gen_e64(e, c, k % e.Mk, i));
    }
    __device__ double2 b(int64_t k, int64_t j) const { return D[j * (e.Mk * e.C) + k]; }
    __device__ void store(int64_t i, int64_t j, double2 v) const {
        if (Xs) {
            double2 x = Xs[j * e.N + i];
            v.x -= lam * x.x;
            v.y -= lam * x.y;
        }
        Y[j * e.N + i] = v;
    }
};

cudaError_t launch_adjoint64(const EncodeDev& e, const double2* D, int64_t F, double lam,
                             const double2* Xsub, double2* Y, cudaStream_t s) {
    if (F == 0) return cudaSuccess;
    int64_t bm, bn;
    frame_shape(F, bm, bn);
    AdjointP p{e, D, Xsub, Y, lam, F, bm, bn};
    return launch_frames(p, e.N, F, s);
}

// U[f][(c,m)] = Dsub[f][(c,m)] - sum_n s_c(n) A[m][n] X[f][n]
struct ForwardP {
    static constexpr bool A_KFAST = true, B_KFAST = true;
    EncodeDev e;
    const double2* X;
    const double2* Dsub;
    double2* U;
    int64_t F, bm, bn;
    __device__ bool tile(int64_t& i0, int64_t& j0, int64_t& kb, int64_t& ke) const {
        frame_tile(bm, bn, i0, j0);
        kb = 0;
        ke = e.N;
        return true;
    }
    __device__ bool a_ok(int64_t i) const { return i < e.Mk * e.C; }
    __device__ bool b_ok(int64_t j) const { return j < F; }
    __device__ double2 a(int64_t i, int64_t k) const {
        int c = (int)(i / e.Mk);
        return gen_e64(e, c, i % e.Mk, k);
    }
    __device__ double2 b(int64_t k, int64_t j) const { return X[j * e.N + k]; }
    __device__ void store(int64_t i, int64_t j, double2 v) const {
        int64_t M = e.Mk * e.C;
        double2 d = Dsub ? Dsub[j * M + i] : make_double2(0.0, 0.0);
        U[j * M + i] = zsub(d, v);
    }
};

cudaError_t launch_forward64(const EncodeDev& e, const double2* X, int64_t F, const double2* Dsub,
                             double2* U, cudaStream_t s) {
    if (F == 0) return cudaSuccess;
    int64_t bm, bn;
    frame_shape(F, bm, bn);
    ForwardP p{e, X, Dsub, U, F, bm, bn};
    return launch_frames(p, e.Mk * e.C, F, s);
}

// Y[f][n] = Yadd[f][n] + sum_n' H[n][n'] X[f][n']
struct HemvP {
    static constexpr bool A_KFAST = true, B_KFAST = true;
    const double2* H;
    const double2* X;
    const double2* Yadd;
    double2* Y;
    int64_t N, ld, F, bm, bn;
    __device__ bool tile(int64_t& i0, int64_t& j0, int64_t& kb, int64_t& ke) const {
        frame_tile(bm, bn, i0, j0);
        kb = 0;
        ke = N;
        return true;
    }
    __device__ bool a_ok(int64_t i) const { return i < N; }
    __device__ bool b_ok(int64_t j) const { return j < F; }
    __device__ double2 a(int64_t i, int64_t k) const { return H[i * ld + k]; }
    __device__ double2 b(int64_t k, int64_t j) const { return X[j * N + k]; }
    __device__ void store(int64_t i, int64_t j, double2 v) const {
        if (Yadd) v = zadd(v, Yadd[j * N + i]);
        Y[j * N + i] = v;
    }
};

cudaError_t launch_hemv64(const double2* H, int64_t N, int64_t ld, const double2* X, int64_t F,
                          const double2* Yadd, double2* Y, cudaStream_t s) {
    if (F == 0) return cudaSuccess;
    int64_t bm, bn;
    frame_shape(F, bm, bn);
    HemvP p{H, X, Yadd, Y, N, ld, F, bm, bn};
    return launch_frames(p, N, F, s);
}

// Y[f][n] = sum_{k <= n} W[n][k] X[f][k] for lower-triangular W (zeros above stored)
struct TrmvP {
    static constexpr bool A_KFAST = true, B_KFAST = true;
    const double2* W;
    const double2* X;
    double2* Y;
    int64_t N, F, bm, bn;
    __device__ bool tile(int64_t& i0, int64_t& j0, int64_t& kb, int64_t& ke) const {
        frame_tile(bm, bn, i0, j0);
        kb = 0;
        ke = i0 + bm < N ? i0 + bm : N;
        return true;
    }
    __device__ bool a_ok(int64_t i) const { return i < N; }
    __device__ bool b_ok(int64_t j) const { return j < F; }
    __device__ double2 a(int64_t i, int64_t k) const { return W[i * N + k]; }
    __device__ double2 b(int64_t k, int64_t j) const { return X[j * N + k]; }
    __device__ void store(int64_t i, int64_t j, double2 v) const { Y[j * N + i] = v; }
};

// Y[f][n] = Yadd[f][n] + sum_{k >= n} conj(W[k][n]) X[f][k]
struct TrmvHP {
    static constexpr bool A_KFAST = false, B_KFAST = true;
    const double2* W;
    const double2* X;
    const double2* Yadd;
    double2* Y;
    int64_t N, F, bm, bn;
    __device__ bool tile(int64_t& i0, int64_t& j0, int64_t& kb, int64_t& ke) const {
        frame_tile(bm, bn, i0, j0);
        kb = i0;
        ke = N;
        return true;
    }
    __device__ bool a_ok(int64_t i) const { return i < N; }
    __device__ bool b_ok(int64_t j) const { return j < F; }
    __device__ double2 a(int64_t i, int64_t k) const { return zconj(W[k * N + i]); }
    __device__ double2 b(int64_t k, int64_t j) const { return X[j * N + k]; }
    __device__ void store(int64_t i, int64_t j, double2 v) const {
        if (Yadd) v = zadd(v, Yadd[j * N + i]);
        Y[j * N + i] = v;
    }
};

cudaError_t launch_trmv64(const double2* W, int64_t N, const double2* X, int64_t F, double2* Y,
                          cudaStream_t s) {
    if (F == 0) return cudaSuccess;
    int64_t bm, bn;
    frame_shape(F, bm, bn);
    TrmvP p{W, X, Y, N, F, bm, bn};
    return launch_frames(p, N, F, s);
}

cudaError_t launch_trmv_h64(const double2* W, int64_t N, const double2* X, int64_t F, const double2* Yadd,
                            double2* Y, cudaStream_t s) {
    if (F == 0) return cudaSuccess;
    int64_t bm, bn;
    frame_shape(F, bm, bn);
    TrmvHP p{W, X, Yadd, Y, N, F, bm, bn};
    return launch_frames(p, N, F, s);
}

}  // namespace pinv
