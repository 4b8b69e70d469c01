// Mixed-precision stages of the build on the tcgen05 split-BF16 engine
// (tc_engine.cuh): Gram, blocked-Cholesky panel solves and trailing updates,
// the triangular inverse and Recon = (L^-1)^H L^-1 E^H (Eq. 8), plus the c64
// SIMT apply used when frames are few.
//
// Every problem supplies tile(); row_a()/row_b(), a per-thread context built
// once per tile (a row pointer, or the phase-table rows of one voxel or one
// sample); a8()/b8(), 8 consecutive k of that row of A or column of B, zero
// outside the problem; row_ok()/col_ok() and store().
#include <algorithm>
#include <cstring>
#include <cstdlib>
#include <vector>

#include "df.cuh"
#include "tc_engine.cuh"

namespace pinv {
namespace tc {

// ------------------------------------------------------------------ FP32 helpers
__device__ inline float2 cmulf(float2 a, float2 b) {
    return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
__device__ inline float2 conjf2(float2 a) { return make_float2(a.x, -a.y); }

// 8 consecutive values from a 16-byte aligned address
__device__ inline void ld8a(const float2* p, float2 (&v)[8]) {
    const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const float4 w = __ldg(q + t);
        v[2 * t] = make_float2(w.x, w.y);
        v[2 * t + 1] = make_float2(w.z, w.w);
    }
}

// 8 consecutive FP32 complex values p[0..7] (zero past `avail`)
__device__ inline void load8f(const float2* p, int avail, float2 (&v)[8]) {
    if (avail >= 8 && (((uintptr_t)p) & 15) == 0) {
        ld8a(p, v);
        return;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) v[t] = t < avail ? __ldg(p + t) : make_float2(0.f, 0.f);
}

// 8 values down a column: p[0], p[ld], ..., p[7 ld] (zero past `avail`)
__device__ inline void load8col(const float2* p, int64_t ld, int avail, float2 (&v)[8]) {
#pragma unroll
    for (int t = 0; t < 8; ++t) v[t] = t < avail ? __ldg(p + t * ld) : make_float2(0.f, 0.f);
}

// A row of a memory operand: pointer to its first element and a validity flag.
struct RowPtr {
    const float2* p;
    int ok;
};

// ------------------------------------------------------------------ generated encoding
// Phase-table rows of one voxel n, for 8 consecutive samples m at a time:
// A[m][n] = ex[m][ix] ey[m][iy] ez[m][iz] b0[u(m)][n] from the sample-contiguous tables.
struct VoxRow {
    const float2* x;
    const float2* y;
    const float2* z;
    const float2* b;
    int ok;
};
__device__ inline VoxRow vox_row(const EncodeDev& e, int64_t n) {
    VoxRow r;
    r.ok = n < e.N;
    const int64_t nn = r.ok ? n : 0;
    const int* g = e.vox_ijk + 3 * nn;
    r.x = e.ext32 + (int64_t)__ldg(g) * e.Mkp;
    r.y = e.ny > 1 ? e.eyt32 + (int64_t)__ldg(g + 1) * e.Mkp : nullptr;
    r.z = e.nz > 1 ? e.ezt32 + (int64_t)__ldg(g + 2) * e.Mkp : nullptr;
    r.b = e.b0t32 ? e.b0t32 + nn * e.T : nullptr;
    return r;
}
// A[m0 .. m0+7][n] (m0 a multiple of 8, ke <= M_k; table rows are padded to a
// multiple of 8, so m0 < ke keeps all eight reads inside the row)
__device__ inline void gen_a8_samples(const EncodeDev& e, const VoxRow& r, int64_t m0, int64_t ke,
                                      float2 (&v)[8]) {
    if (!r.ok || m0 >= ke) {
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = make_float2(0.f, 0.f);
        return;
    }
    ld8a(r.x + m0, v);
    if (r.y) {
        float2 w[8];
        ld8a(r.y + m0, w);
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = cmulf(v[t], w[t]);
    }
    if (r.z) {
        float2 w[8];
        ld8a(r.z + m0, w);
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = cmulf(v[t], w[t]);
    }
    if (r.b) {
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            const int u = m0 + t < ke ? __ldg(e.tidx + m0 + t) : 0;
            v[t] = cmulf(v[t], __ldg(r.b + u));
        }
    }
#pragma unroll
    for (int t = 0; t < 8; ++t)
        if (!r.ok || m0 + t >= ke) v[t] = make_float2(0.f, 0.f);
}

// One column j = (c, m) of E^H, for 8 consecutive voxels at a time:
// conj(s_c(n) A[m][n]) from the voxel-contiguous tables ex32[m][ix] etc.
struct EhCol {
    const float2* x;
    const float2* y;
    const float2* z;
    const float2* c;
    const float2* b;
    int ok;
};
__device__ inline EhCol eh_col(const EncodeDev& e, int64_t j) {
    EhCol r;
    const int64_t M = e.Mk * e.C;
    r.ok = j < M;
    const int64_t jj = r.ok ? j : 0;
    const int c = (int)(jj / e.Mk);
    const int64_t m = jj - (int64_t)c * e.Mk;
    r.x = e.ex32 + m * e.nx;
    r.y = e.ey32 + m * e.ny;
    r.z = e.ez32 + m * e.nz;
    r.c = e.coils32 ? e.coils32 + (int64_t)c * e.N : nullptr;
    r.b = e.b0tab32 ? e.b0tab32 + (int64_t)__ldg(e.tidx + m) * e.N : nullptr;
    return r;
}
__device__ inline void gen_eh8_voxels(const EncodeDev& e, const EhCol& r, int64_t n0, int64_t ke,
                                      float2 (&v)[8]) {
    if (!r.ok) {
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = make_float2(0.f, 0.f);
        return;
    }
    if (e.full_grid && (e.nx & 7) == 0 && n0 + 8 <= ke) {
        // 8 voxels on one grid line: contiguous ix, shared iy and iz
        const int64_t ix0 = n0 % e.nx, rest = n0 / e.nx;
        ld8a(r.x + ix0, v);
        float2 sc = make_float2(1.f, 0.f);
        if (e.ny > 1) sc = __ldg(r.y + rest % e.ny);
        if (e.nz > 1) sc = cmulf(sc, __ldg(r.z + rest / e.ny));
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = cmulf(v[t], sc);
        if (r.b) {
            float2 w[8];
            ld8a(r.b + n0, w);
#pragma unroll
            for (int t = 0; t < 8; ++t) v[t] = cmulf(v[t], w[t]);
        }
        if (r.c) {
            float2 w[8];
            ld8a(r.c + n0, w);
#pragma unroll
            for (int t = 0; t < 8; ++t) v[t] = cmulf(v[t], w[t]);
        }
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = conjf2(v[t]);
        return;
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int64_t n = n0 + t;
        if (n < ke) {
            const int* g = e.vox_ijk + 3 * n;
            float2 a = __ldg(r.x + __ldg(g));
            if (e.ny > 1) a = cmulf(a, __ldg(r.y + __ldg(g + 1)));
            if (e.nz > 1) a = cmulf(a, __ldg(r.z + __ldg(g + 2)));
            if (r.b) a = cmulf(a, __ldg(r.b + n));
            if (r.c) a = cmulf(a, __ldg(r.c + n));
            v[t] = conjf2(a);
        } else {
            v[t] = make_float2(0.f, 0.f);
        }
    }
}

// ------------------------------------------------------------------ Gram (Eq. 6, Eq. 11)
// G[i][j] = (sum_m conj(A[m][i]) A[m][j]) * (sum_c conj(s_c(i)) s_c(j)) + lam delta_ij, lower part,
// in double-float storage (df_of_f32). v is the sample sum (A^H A)_ij; j > i is not stored.
__device__ inline void gram_store(const EncodeDev& e, double lam, float4* G, int64_t ld, int64_t i, int64_t j,
                                  float2 v) {
    if (j > i) return;
    if (i == j) {
        // every encoding element is a unit phasor, so (A^H A)_ii = M_k exactly;
        // the diagonal is written in FP64 rather than from the accumulator
        double s = 1.0;
        if (e.coils) {
            s = 0.0;
            for (int c = 0; c < e.C; ++c) {
                const double2 a = e.coils[(int64_t)c * e.N + i];
                s += a.x * a.x + a.y * a.y;
            }
        }
        G[i * ld + i] = to_df_i(make_double2((double)e.Mk * s + lam, 0.0));
        return;
    }
    if (e.coils32) {
        float2 sc = make_float2(0.f, 0.f);
        for (int c = 0; c < e.C; ++c) {
            const float2 a = conjf2(e.coils32[(int64_t)c * e.N + i]);
            const float2 b = e.coils32[(int64_t)c * e.N + j];
            sc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, sc.x));
            sc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, sc.y));
        }
        v = cmulf(v, sc);
    }
    G[i * ld + j] = df_of_f32(v);
}

struct GramTC {
    EncodeDev e;
    double lam;
    float4* G;
    int64_t ld;
    __device__ bool tile(int64_t bx, int64_t by, int64_t& i0, int64_t& j0, int64_t& kb, int64_t& ke) const {
        i0 = by * BM;
        j0 = bx * BN;
        kb = 0;
        ke = e.Mk;
        return j0 <= i0 + BM - 1;  // tile touches the lower triangle
    }
    __device__ VoxRow row_a(int64_t i) const { return vox_row(e, i); }
    __device__ VoxRow row_b(int64_t j) const { return vox_row(e, j); }
    __device__ void a8(const VoxRow& r, int64_t k0, int64_t ke, float2 (&v)[8]) const {
        gen_a8_samples(e, r, k0, ke, v);
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t].y = -v[t].y;
    }
    __device__ void b8(const VoxRow& r, int64_t k0, int64_t ke, float2 (&v)[8]) const {
        gen_a8_samples(e, r, k0, ke, v);
    }
    __device__ bool row_ok(int64_t i) const { return i < e.N; }
    __device__ bool col_ok(int64_t j) const { return j < e.N; }
    __device__ void store(int64_t i, int64_t j, float2 v) const { gram_store(e, lam, G, ld, i, j, v); }
};

// ------------------------------------------------------------------ Gram, bulk-fed
// The encoding A is generated once into a table of stage tiles, each split into
// S bf16 slices: block (row tile rt, sample chunk kc, slice s), 16 KiB, holds
// T1 = rows [Re A | -Im A] over the chunk's 16 samples (the A operand conj(A)
// and the first half of the B operand) and T2 = rows [Im A | Re A] (the second
// half of the B operand), both in the stage layout. The Gram kernel then only
// copies: per stage T1 of row tile i and T1|T2 of column tile j, per slice.
// Items are (split, i, j) with the sample range cut into `splits` parts (so
// that the last wave of tiles is not mostly idle), visited in bands of GBAND
// row tiles, column-major inside a band (the tiles running at one time share
// few rows and columns, which stay in L2). With one split the epilogue writes G
// directly; otherwise it writes FP32 partial sums that k_gram_finalize adds in
// split order.
constexpr int GBAND = 8;
constexpr int64_t TAB_BLOCK = B_SL;  // one B slice tile (the A slice tile is its first half)

// Operand tables hold stage tiles, one per (tile, 16-wide k chunk, slice):
// A tiles (A_SL bytes) rows [re | im] of a(i, k); B tiles (B_SL bytes) rows
// [re | -im] then [im | re] of b(k, j). A thread writes 8 consecutive k
// (group g = 0 or 1 of the chunk) of row r in every slice.
template <int S>
__device__ inline void tab_split(const float2 (&v)[8], uint32_t (&wr)[S][4], uint32_t (&wi)[S][4]) {
    float re[8], im[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
        re[u] = v[u].x;
        im[u] = v[u].y;
    }
    split8<S>(re, wr);
    split8<S>(im, wi);
}
__device__ inline void st16(uint8_t* p, const uint32_t (&w)[4], uint32_t flip) {
    *reinterpret_cast<uint4*>(p) = make_uint4(w[0] ^ flip, w[1] ^ flip, w[2] ^ flip, w[3] ^ flip);
}
template <int S>
__device__ inline void put_a(uint8_t* blk, int r, int g, const float2 (&v)[8]) {
    uint32_t wr[S][4], wi[S][4];
    tab_split<S>(v, wr, wi);
#pragma unroll
    for (int sl = 0; sl < S; ++sl) {
        st16(blk + sl * A_SL + koff(r, g), wr[sl], 0u);
        st16(blk + sl * A_SL + koff(r, g + 2), wi[sl], 0u);
    }
}
template <int S>
__device__ inline void put_b(uint8_t* blk, int r, int g, const float2 (&v)[8]) {
    uint32_t wr[S][4], wi[S][4];
    tab_split<S>(v, wr, wi);
#pragma unroll
    for (int sl = 0; sl < S; ++sl) {
        uint8_t* b = blk + sl * B_SL;
        st16(b + koff(r, g), wr[sl], 0u);
        st16(b + koff(r, g + 2), wi[sl], 0x80008000u);
        st16(b + A_SL + koff(r, g), wi[sl], 0u);
        st16(b + A_SL + koff(r, g + 2), wr[sl], 0u);
    }
}

// Item l of a rows x cols tile grid, in bands of GBAND row tiles and
// column-major inside a band: the tiles running at one time share few rows and
// columns, whose operand tiles then stay in L2.
__device__ inline void band_tile(int64_t l, int64_t rows, int64_t cols, int64_t& rt, int64_t& ct) {
    const int64_t band = l / (GBAND * cols), l2 = l - band * GBAND * cols;
    const int64_t hgt = rows - band * GBAND < GBAND ? rows - band * GBAND : GBAND;
    ct = l2 / hgt;
    rt = band * GBAND + l2 % hgt;
}

// Gram table: the B tiles of b(m, n) = A[m][n] over row tiles of voxels and
// chunks of 16 samples; their first halves are the A tiles of conj(A).
template <int S>
__global__ void __launch_bounds__(256) k_gram_tab(EncodeDev e, int64_t kcn, uint8_t* tab) {
    const int64_t kc = blockIdx.x, rt = blockIdx.y;
    const int r = threadIdx.x & (BM - 1), g = threadIdx.x >> 7;
    float2 v[8];
    gen_a8_samples(e, vox_row(e, rt * BM + r), kc * KC + 8 * g, e.Mk, v);
    put_b<S>(tab + (rt * kcn + kc) * S * B_SL, r, g, v);
}

struct GramBulk {
    static constexpr bool kBulk = true;
    EncodeDev e;
    double lam;
    float4* G;           // splits == 1: the lower part of G (double-float)
    int64_t ld;
    float2* part;        // splits > 1: partial sums [split][NP][NP], NP = nt * BM
    const uint8_t* tab;  // [nt][kcn][S] blocks
    int64_t nt, kcn, kcs;  // row tiles, sample chunks, chunks per split
    int S, splits;
    __device__ bool tile(int64_t bx, int64_t, int64_t& i0, int64_t& j0, int64_t& kb, int64_t& ke) const {
        const int64_t per = nt * nt;
        const int64_t sp = bx / per;
        int64_t it, jt;
        band_tile(bx - sp * per, nt, nt, it, jt);
        i0 = (sp * nt + it) * BM;  // the split rides on the row coordinate
        j0 = jt * BN;
        kb = sp * kcs * KC;
        ke = ((sp + 1) * kcs < kcn ? (sp + 1) * kcs : kcn) * KC;
        return jt <= it && kb < ke;
    }
    __device__ const uint8_t* bulk_a(int64_t i0, int64_t kc, int sl) const {
        return tab + ((((i0 / BM) % nt) * kcn + kc) * S + sl) * TAB_BLOCK;
    }
    __device__ const uint8_t* bulk_b(int64_t j0, int64_t kc, int sl) const {
        return tab + (((j0 / BN) * kcn + kc) * S + sl) * TAB_BLOCK;
    }
    // (A^H A)[i][j + 32 u], u = 0..3, lower part: partial sums, or G with the coil factor
    __device__ void store4(int64_t i, int64_t j, const float2 (&v)[4]) const {
        const int64_t np = nt * BM, il = i % np;
        if (il >= e.N) return;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if (j + 32 * u > il) continue;
            if (splits > 1)
                part[i * np + j + 32 * u] = v[u];
            else
                gram_store(e, lam, G, ld, il, j + 32 * u, v[u]);
        }
    }
    __device__ bool row_ok(int64_t i) const { return i % (nt * BM) < e.N; }
    __device__ bool col_ok(int64_t j) const { return j < e.N; }
    __device__ void store(int64_t, int64_t, float2) const {}
};

// ------------------------------------------------------------------ refinement correction
// x += W^H (W r) for a block of frames (F <= BN), in two split-K products whose
// partial sums (one per range of k, `chunk` wide) are added in order afterwards:
//   CorrW   T[f][i]  = sum_{k <= i} W[i][k] r[f][k]
//   CorrWH  X[f][n] += sum_{k >= n} conj(W[k][n]) T[f][k]
// The column coordinate carries the k range: column j is frame j % BN of split j / BN.
__device__ inline void load8d(const double2* p, int avail, float2 (&v)[8]) {
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const double2 a = t < avail ? p[t] : make_double2(0.0, 0.0);
        v[t] = make_float2((float)a.x, (float)a.y);
    }
}
struct CorrW {
    static constexpr bool kPrefetch = true;  // W streams from HBM
    const float2* W;
    const double2* R;  // [F][N]
    float2* part;      // [splits][F][N]
    int64_t N, F, chunk;
    __device__ bool tile(int64_t bx, int64_t by, int64_t& i0, int64_t& j0, int64_t& kb, int64_t& ke) const {
        i0 = by * BM;
        j0 = bx * BN;
        kb = bx * chunk;
        ke = kb + chunk;
        const int64_t kmax = i0 + BM < N ? i0 + BM : N;  // W is lower triangular
        if (ke > kmax) ke = kmax;
        return kb < ke;
    }
    __device__ RowPtr row_a(int64_t i) const { return RowPtr{W + (i < N ? i : 0) * N, i < N}; }
    __device__ int64_t row_b(int64_t j) const { return j % BN; }
    __device__ void a8(const RowPtr& r, int64_t k, int64_t ke, float2 (&v)[8]) const {
        load8f(r.p + k, r.ok ? (int)(ke - k) : 0, v);
    }
    __device__ void b8(int64_t f, int64_t k, int64_t ke, float2 (&v)[8]) const {
        load8d(R + (f < F ? f : 0) * N + k, f < F ? (int)(ke - k) : 0, v);
    }
    __device__ bool row_ok(int64_t i) const { return i < N; }
    __device__ bool col_ok(int64_t j) const { return j % BN < F; }
    __device__ void store(int64_t i, int64_t j, float2 v) const { part[((j / BN) * F + j % BN) * N + i] = v; }
};
struct CorrWH {
    static constexpr bool kPrefetch = true;  // W streams from HBM
    const float2* W;
    const float2* T;  // [F][N]
    float2* part;     // [splits][F][N]
    int64_t N, F, chunk;
    __device__ bool tile(int64_t bx, int64_t by, int64_t& i0, int64_t& j0, int64_t& kb, int64_t& ke) const {
        i0 = by * BM;
        j0 = bx * BN;
        kb = bx * chunk;
        if (kb < i0) kb = i0;  // W is lower triangular: k >= n
        ke = (bx + 1) * chunk < N ? (bx + 1) * chunk : N;
        return kb < ke;
    }
    __device__ int64_t row_a(int64_t i) const { return i; }
    __device__ int64_t row_b(int64_t j) const { return j % BN; }
    __device__ void a8(int64_t n, int64_t k, int64_t ke, float2 (&v)[8]) const {
        load8col(W + k * N + (n < N ? n : 0), N, n < N ? (int)(ke - k) : 0, v);
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t].y = -v[t].y;
    }
    __device__ void b8(int64_t f, int64_t k, int64_t ke, float2 (&v)[8]) const {
        load8f(T + (f < F ? f : 0) * N + k, f < F ? (int)(ke - k) : 0, v);
    }
    __device__ bool row_ok(int64_t i) const { return i < N; }
    __device__ bool col_ok(int64_t j) const { return j % BN < F; }
    __device__ void store(int64_t i, int64_t j, float2 v) const { part[((j / BN) * F + j % BN) * N + i] = v; }
};

// ------------------------------------------------------------------ Recon, bulk-fed
// Recon = W^H (W E^H) (Eq. 8) computed transposed, sample rows by voxel columns,
// over one range of samples (a chunk of row tiles) at a time:
//   step 1  T^T[j][i] = sum_k conj(E[j][k]) W[i][k]     (k < i0 + 128: W is lower)
//   step 2  Recon[n][j] = sum_k T^T[j][k] conj(W[k][n])  (k >= n0)
// Operand tables: ET (A tiles of conj(E), generated from the phase tables), WB1
// and WB2 (B tiles of W[i][k] and conj(W[k][n]), from the FP32 W) and TT (A
// tiles of T^T, written split by the step-1 epilogue: T never exists in FP32).
template <int S>
__global__ void __launch_bounds__(256) k_tab_et(EncodeDev e, int64_t kcn, int64_t j_off, uint8_t* tab) {
    const int64_t kc = blockIdx.x, rt = blockIdx.y;
    const int r = threadIdx.x & (BM - 1), g = threadIdx.x >> 7;
    float2 v[8];
    gen_eh8_voxels(e, eh_col(e, j_off + rt * BM + r), kc * KC + 8 * g, e.N, v);
    put_a<S>(tab + (rt * kcn + kc) * S * A_SL, r, g, v);
}

// WB1 (lower = 1): b(k, i) = W[i][k]; WB2 (lower = 0): b(k, n) = conj(W[k][n]).
// Only the chunks the triangular products read are written.
template <int S>
__global__ void __launch_bounds__(256) k_tab_w(const float2* __restrict__ W32, int64_t N, int64_t kcn, int lower,
                                               uint8_t* tab) {
    const int64_t kc = blockIdx.x, ct = blockIdx.y;
    if (lower ? kc * KC >= (ct + 1) * BN : (kc + 1) * KC <= ct * BN) return;
    const int r = threadIdx.x & (BM - 1), g = threadIdx.x >> 7;
    const int64_t col = ct * BN + r, k0 = kc * KC + 8 * g;
    const int avail = col < N && k0 < N ? (int)(N - k0) : 0;
    float2 v[8];
    if (lower) {
        load8f(W32 + (col < N ? col : 0) * N + (k0 < N ? k0 : 0), avail, v);
    } else {
        load8col(W32 + (k0 < N ? k0 : 0) * N + (col < N ? col : 0), N, avail, v);
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t].y = -v[t].y;
    }
    put_b<S>(tab + (ct * kcn + kc) * S * B_SL, r, g, v);
}

struct ReconB1 {
    static constexpr bool kBulk = true;
    static constexpr bool kHintB = true;
    const uint8_t* et;
    const uint8_t* wb;
    uint8_t* tt;
    int64_t rows, nt, kcn;  // sample tiles in the chunk, voxel tiles, voxel chunks
    int S;
    __device__ bool tile(int64_t bx, int64_t, int64_t& i0, int64_t& j0, int64_t& kb, int64_t& ke) const {
        int64_t rt, ct;
        band_tile(bx, rows, nt, rt, ct);
        ct = nt - 1 - ct;  // the longest tiles of a band first
        i0 = rt * BM;
        j0 = ct * BN;
        kb = 0;
        ke = (ct + 1) * BN;
        return true;
    }
    __device__ const uint8_t* bulk_a(int64_t i0, int64_t kc, int sl) const {
        return et + (((i0 / BM) * kcn + kc) * S + sl) * A_SL;
    }
    __device__ const uint8_t* bulk_b(int64_t j0, int64_t kc, int sl) const {
        return wb + (((j0 / BN) * kcn + kc) * S + sl) * B_SL;
    }
    // row i of T^T, voxels j0 .. j0 + 15 (one chunk of TT), split into S slices
    __device__ void store16(int64_t i, int64_t j0, const float (&re)[16], const float (&im)[16]) const {
        uint8_t* blk = tt + ((i / BM) * kcn + j0 / KC) * S * A_SL;
        const int r = (int)(i % BM);
#pragma unroll
        for (int g = 0; g < 2; ++g) {
            float2 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = make_float2(re[8 * g + u], im[8 * g + u]);
            if (S == 3)
                put_a<3>(blk, r, g, v);
            else
                put_a<2>(blk, r, g, v);
        }
    }
    __device__ bool row_ok(int64_t) const { return true; }
    __device__ bool col_ok(int64_t) const { return true; }
    __device__ void store(int64_t, int64_t, float2) const {}
};

struct ReconB2 {
    static constexpr bool kBulk = true;
    static constexpr bool kHintB = true;
    const uint8_t* tt;
    const uint8_t* wb;
    float2* R;
    int64_t rows, nt, kcn;
    int64_t N, M, j_off, mvalid;  // Recon is [N][M]; this chunk holds samples j_off .. j_off + mvalid - 1
    int S;
    __device__ bool tile(int64_t bx, int64_t, int64_t& i0, int64_t& j0, int64_t& kb, int64_t& ke) const {
        int64_t rt, ct;
        band_tile(bx, rows, nt, rt, ct);
        i0 = rt * BM;
        j0 = ct * BN;
        kb = ct * BN;
        ke = nt * BN;
        return true;
    }
    __device__ const uint8_t* bulk_a(int64_t i0, int64_t kc, int sl) const {
        return tt + (((i0 / BM) * kcn + kc) * S + sl) * A_SL;
    }
    __device__ const uint8_t* bulk_b(int64_t j0, int64_t kc, int sl) const {
        return wb + (((j0 / BN) * kcn + kc) * S + sl) * B_SL;
    }
    __device__ bool row_ok(int64_t i) const { return i < mvalid; }
    __device__ bool col_ok(int64_t j) const { return j < N; }
    __device__ void store(int64_t i, int64_t j, float2 v) const { R[j * M + j_off + i] = v; }
};

// ------------------------------------------------------------------ panel trailing updates, bulk-fed
// After a 256-wide panel p0 .. p0 + kw of the factor, both trailing updates
// have the panel L[i][p0 + k] (rows i >= r0) as their A operand:
//   HerkBulk   G[i][j] -= sum_k L[i][k] conj(L[j][k])   (i >= j >= r0)
//   TrtriBulk  W[i][j] -= sum_k L[i][k] W[p0 + k][j]     (i >= r0, j < r0)
// One table of B tiles of conj(L) serves as the HERK's A tiles (first halves)
// and B tiles; a second holds the B tiles of the panel's rows of W.
template <int S>
__global__ void __launch_bounds__(256) k_tab_panel(const float2* __restrict__ L32, int64_t ldl, int64_t N,
                                                   int64_t p0, int64_t kw, int64_t r0, uint8_t* tab) {
    const int64_t kc = blockIdx.x, rt = blockIdx.y, kcn = gridDim.x;
    const int r = threadIdx.x & (BM - 1), g = threadIdx.x >> 7;
    const int64_t i = r0 + rt * BM + r, k0 = kc * KC + 8 * g;
    griddep_wait();
    griddep_launch();
    float2 v[8];
    load8f(L32 + (i < N ? i : 0) * ldl + p0 + k0, i < N && k0 < kw ? (int)(kw - k0) : 0, v);
#pragma unroll
    for (int t = 0; t < 8; ++t) v[t].y = -v[t].y;
    put_b<S>(tab + (rt * kcn + kc) * S * B_SL, r, g, v);
}
template <int S>
__global__ void __launch_bounds__(256) k_tab_wrows(const float4* __restrict__ W, int64_t ld, int64_t p0, int64_t kw,
                                                   int64_t ncols, uint8_t* tab) {
    const int64_t kc = blockIdx.x, ct = blockIdx.y, kcn = gridDim.x;
    const int r = threadIdx.x & (BM - 1), g = threadIdx.x >> 7;
    griddep_wait();
    griddep_launch();
    const int64_t j = ct * BN + r, k0 = kc * KC + 8 * g;
    float2 v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const bool ok = j < ncols && k0 + t < kw;
        v[t] = ok ? df_to_f32(W[(p0 + k0 + t) * ld + j]) : make_float2(0.f, 0.f);
    }
    put_b<S>(tab + (ct * kcn + kc) * S * B_SL, r, g, v);
}

struct HerkBulk {
    static constexpr bool kBulk = true;
    const uint8_t* tab;
    float4* G;                   // double-float storage
    int64_t ld, N, r0, nt, kcn;  // trailing rows from r0 in nt tiles; panel chunks
    int S;
    int64_t jt0, ncols;          // column tiles jt0 .. jt0 + ncols - 1 of the trailing matrix (grid nt x ncols)
    __device__ bool tile(int64_t bx, int64_t, int64_t& i0, int64_t& j0, int64_t& kb, int64_t& ke) const {
        int64_t it, jt;
        band_tile(bx, nt, ncols, it, jt);
        jt += jt0;
        i0 = r0 + it * BM;
        j0 = r0 + jt * BN;
        kb = 0;
        ke = kcn * KC;
        return jt <= it;
    }
    __device__ const uint8_t* bulk_a(int64_t i0, int64_t kc, int sl) const {
        return tab + ((((i0 - r0) / BM) * kcn + kc) * S + sl) * B_SL;
    }
    __device__ const uint8_t* bulk_b(int64_t j0, int64_t kc, int sl) const {
        return tab + ((((j0 - r0) / BN) * kcn + kc) * S + sl) * B_SL;
    }
    // G[i][j] -= v: the entry to update (lower part), or null
    __device__ float4* rmw_ptr(int64_t i, int64_t j) const { return (i < N && j <= i) ? G + i * ld + j : nullptr; }
    // G[i][j .. j + n - 1] into L2, the lower part only
    __device__ void prefetch(int64_t i, int64_t j, int n) const {
        if (i >= N || j > i) return;
        bulk_prefetch_l2(G + i * ld + j, (uint32_t)(i - j + 1 < n ? i - j + 1 : n) * 16u);
    }
    __device__ bool row_ok(int64_t i) const { return i < N; }
    __device__ bool col_ok(int64_t j) const { return j < N; }
    __device__ void store(int64_t, int64_t, float2) const {}
};
struct TrtriBulk {
    static constexpr bool kBulk = true;
    const uint8_t* tabl;
    const uint8_t* tabw;
    float4* W;                          // double-float storage
    int64_t ld, N, r0, ntr, ntc, kcn;  // rows from r0 in ntr tiles; columns below r0 in ntc tiles
    int S;
    __device__ bool tile(int64_t bx, int64_t, int64_t& i0, int64_t& j0, int64_t& kb, int64_t& ke) const {
        int64_t rt, ct;
        band_tile(bx, ntr, ntc, rt, ct);
        i0 = r0 + rt * BM;
        j0 = ct * BN;
        kb = 0;
        ke = kcn * KC;
        return true;
    }
    __device__ const uint8_t* bulk_a(int64_t i0, int64_t kc, int sl) const {
        return tabl + ((((i0 - r0) / BM) * kcn + kc) * S + sl) * B_SL;
    }
    __device__ const uint8_t* bulk_b(int64_t j0, int64_t kc, int sl) const {
        return tabw + (((j0 / BN) * kcn + kc) * S + sl) * B_SL;
    }
    // W[i][j] -= v: the entry to update (columns below r0), or null
    __device__ float4* rmw_ptr(int64_t i, int64_t j) const { return (i < N && j < r0) ? W + i * ld + j : nullptr; }
    // W[i][j .. j + n - 1] into L2, the columns below r0 only
    __device__ void prefetch(int64_t i, int64_t j, int n) const {
        if (i >= N || j >= r0) return;
        bulk_prefetch_l2(W + i * ld + j, (uint32_t)(r0 - j < n ? r0 - j : n) * 16u);
    }
    __device__ bool row_ok(int64_t i) const { return i < N; }
    __device__ bool col_ok(int64_t j) const { return j < r0; }
    __device__ void store(int64_t, int64_t, float2) const {}
};

// ------------------------------------------------------------------ blocked Cholesky
// Trailing update G[i][j] -= sum_k P[i][k] conj(P[j][k]) on lower tiles, rows
// i >= t0 and columns t0 <= j < jmax (jmax < N restricts it to a panel).
struct HerkTC {
    const float2* P;
    int64_t ldp;
    float4* G;  // double-float storage
    int64_t ld, N, nbk, t0, jmax;
    __device__ bool tile(int64_t bx, int64_t by, int64_t& i0, int64_t& j0, int64_t& kb, int64_t& ke) const {
        i0 = t0 + by * BM;
        j0 = t0 + bx * BN;
        kb = 0;
        ke = nbk;
        return i0 < N && j0 < jmax && j0 <= i0 + BM - 1;
    }
    __device__ RowPtr row_a(int64_t i) const { return RowPtr{P + (i < N ? i : 0) * ldp, i < N}; }
    __device__ RowPtr row_b(int64_t j) const { return RowPtr{P + (j < N ? j : 0) * ldp, j < N}; }
    __device__ void a8(const RowPtr& r, int64_t k, int64_t ke, float2 (&v)[8]) const {
        load8f(r.p + k, r.ok ? (int)(ke - k) : 0, v);
    }
    __device__ void b8(const RowPtr& r, int64_t k, int64_t ke, float2 (&v)[8]) const {
        load8f(r.p + k, r.ok ? (int)(ke - k) : 0, v);
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t].y = -v[t].y;
    }
    __device__ bool row_ok(int64_t i) const { return i < N; }
    __device__ bool col_ok(int64_t j) const { return j < jmax; }
    __device__ void store(int64_t i, int64_t j, float2 v) const {
        if (j > i) return;
        G[i * ld + j] = df_sub_f32(G[i * ld + j], v);
    }
};

// ------------------------------------------------------------------ W = L^-1
// W[i][j] -= sum_k L[i][k0+k] W[k0+k][j] for k0 + nbk <= i < imax, j < k0 + nbk
// (W in double-float storage).
struct TrtriUpdTC {
    const float2* L32;
    int64_t ldl;
    float4* W;
    int64_t ld, N, k0, nbk, imax;
    __device__ bool tile(int64_t bx, int64_t by, int64_t& i0, int64_t& j0, int64_t& kb, int64_t& ke) const {
        i0 = k0 + nbk + by * BM;
        j0 = bx * BN;
        kb = 0;
        ke = nbk;
        return i0 < imax;
    }
    __device__ RowPtr row_a(int64_t i) const { return RowPtr{L32 + (i < imax ? i : 0) * ldl + k0, i < imax}; }
    __device__ int64_t row_b(int64_t j) const { return j; }
    __device__ void a8(const RowPtr& r, int64_t k, int64_t ke, float2 (&v)[8]) const {
        load8f(r.p + k, r.ok ? (int)(ke - k) : 0, v);
    }
    __device__ void b8(int64_t j, int64_t k, int64_t ke, float2 (&v)[8]) const {
#pragma unroll
        for (int t = 0; t < 8; ++t)
            v[t] = (j < k0 + nbk && k + t < ke) ? df_to_f32(W[(k0 + k + t) * ld + j]) : make_float2(0.f, 0.f);
    }
    __device__ bool row_ok(int64_t i) const { return i < imax; }
    __device__ bool col_ok(int64_t j) const { return j < k0 + nbk; }
    __device__ void store(int64_t i, int64_t j, float2 v) const { W[i * ld + j] = df_sub_f32(W[i * ld + j], v); }
};

// ------------------------------------------------------------------ Recon = W^H (W E^H)
// T[n][j] = sum_{k <= n} W[n][k] conj(E[j][k])     (j = c * M_k + m)
struct ReconStep1TC {
    EncodeDev e;
    const float2* W32;
    float2* T;
    __device__ bool tile(int64_t bx, int64_t by, int64_t& i0, int64_t& j0, int64_t& kb, int64_t& ke) const {
        j0 = bx * BN;
        i0 = by * BM;
        kb = 0;
        ke = i0 + BM < e.N ? i0 + BM : e.N;  // W is lower triangular
        return true;
    }
    __device__ RowPtr row_a(int64_t i) const { return RowPtr{W32 + (i < e.N ? i : 0) * e.N, i < e.N}; }
    __device__ EhCol row_b(int64_t j) const { return eh_col(e, j); }
    __device__ void a8(const RowPtr& r, int64_t k, int64_t ke, float2 (&v)[8]) const {
        load8f(r.p + k, r.ok ? (int)(ke - k) : 0, v);
    }
    __device__ void b8(const EhCol& c, int64_t k, int64_t ke, float2 (&v)[8]) const {
        gen_eh8_voxels(e, c, k, ke, v);
    }
    __device__ bool row_ok(int64_t i) const { return i < e.N; }
    __device__ bool col_ok(int64_t j) const { return j < e.Mk * e.C; }
    __device__ void store(int64_t i, int64_t j, float2 v) const { T[i * (e.Mk * e.C) + j] = v; }
};

// R[n][j] = sum_{k >= n} conj(W[k][n]) T[k][j] with WT = W^T (so W's column n is
// WT's row n, read contiguously); row tiles vary fastest so the CTAs in flight
// share one column panel of T in L2.
struct ReconStep2TC {
    const float2* WT32;
    const float2* T;
    float2* R;
    int64_t N, M;
    __device__ bool tile(int64_t bx, int64_t by, int64_t& i0, int64_t& j0, int64_t& kb, int64_t& ke) const {
        i0 = bx * BM;
        j0 = by * BN;
        kb = i0;  // W is lower triangular
        ke = N;
        return true;
    }
    __device__ RowPtr row_a(int64_t i) const { return RowPtr{WT32 + (i < N ? i : 0) * N, i < N}; }
    __device__ RowPtr row_b(int64_t j) const { return RowPtr{T + (j < M ? j : 0), j < M}; }
    __device__ void a8(const RowPtr& r, int64_t k, int64_t ke, float2 (&v)[8]) const {
        load8f(r.p + k, r.ok ? (int)(ke - k) : 0, v);
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t].y = -v[t].y;
    }
    __device__ void b8(const RowPtr& r, int64_t k, int64_t ke, float2 (&v)[8]) const {
        load8col(r.p + k * M, M, r.ok ? (int)(ke - k) : 0, v);
    }
    __device__ bool row_ok(int64_t i) const { return i < N; }
    __device__ bool col_ok(int64_t j) const { return j < M; }
    __device__ void store(int64_t i, int64_t j, float2 v) const { R[i * M + j] = v; }
};

}  // namespace tc

template <class P>
static cudaError_t run(const P& p, dim3 grid, int slices, DevStatus* st, int site, cudaStream_t s,
                       bool rev = false, int cap = 0, bool pdl = false) {
    return slices == 3 ? tc::launch<3>(p, grid, st, site, s, rev, cap, pdl)
                       : tc::launch<2>(p, grid, st, site, s, rev, cap, pdl);
}

static inline unsigned cdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

cudaError_t launch_gram_tc(const EncodeDev& e, double lambda, int slices, float4* G, int64_t ld,
                           DevStatus* st, cudaStream_t s) {
    tc::GramTC p{e, lambda, G, ld};
    return run(p, dim3(cdiv(e.N, tc::BN), cdiv(e.N, tc::BM)), slices, st, 1, s);
}

// G[i][j] (j <= i) from the partial sample sums of the bulk Gram, added in split order
__global__ void k_gram_finalize(EncodeDev e, double lam, const float2* __restrict__ part, int splits, int64_t np,
                                float4* G, int64_t ld) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= e.N * e.N) return;
    const int64_t i = idx / e.N, j = idx - i * e.N;
    if (j > i) return;
    float2 v = part[i * np + j];
    for (int sp = 1; sp < splits; ++sp) {
        const float2 w = part[(sp * np + i) * np + j];
        v.x += w.x;
        v.y += w.y;
    }
    tc::gram_store(e, lam, G, ld, i, j, v);
}

namespace {
struct GramBulkShape {
    int64_t nt, kcn, kcs;
    int splits;
    size_t tab_bytes, part_bytes;
};
// sample-range splits: the fewest (up to 4) that fill the last wave of tiles to 90 %
GramBulkShape gram_bulk_shape(const EncodeDev& e, int slices) {
    GramBulkShape g;
    g.nt = (e.N + tc::BM - 1) / tc::BM;
    g.kcn = (e.Mk + tc::KC - 1) / tc::KC;
    const int64_t tiles = g.nt * (g.nt + 1) / 2, sms = tc::sm_count();
    g.splits = 1;
    for (int sp = 1; sp <= 4; ++sp) {
        const int64_t items = tiles * sp, waves = (items + sms - 1) / sms;
        g.splits = sp;
        if ((double)items >= 0.9 * (double)(waves * sms) || g.kcn < 64 * (sp + 1)) break;
    }
    g.kcs = (g.kcn + g.splits - 1) / g.splits;
    const size_t np = (size_t)g.nt * tc::BM;
    g.tab_bytes = (size_t)g.nt * g.kcn * slices * tc::B_SL;
    g.part_bytes = g.splits > 1 ? g.splits * np * np * sizeof(float2) : 0;
    return g;
}
tc::GramBulk gram_bulk_problem(const EncodeDev& e, double lam, int slices, float4* G, int64_t ld, void* work,
                               int64_t* items) {
    const GramBulkShape g = gram_bulk_shape(e, slices);
    uint8_t* tab = (uint8_t*)work;
    float2* part = g.splits > 1 ? (float2*)(tab + g.tab_bytes) : nullptr;
    *items = g.splits * g.nt * g.nt;
    return tc::GramBulk{e, lam, G, ld, part, tab, g.nt, g.kcn, g.kcs, slices, g.splits};
}
}  // namespace

size_t gram_bulk_bytes(const EncodeDev& e, int slices) {
    const GramBulkShape g = gram_bulk_shape(e, slices);
    return g.tab_bytes + g.part_bytes;
}

cudaError_t gram_bulk_table(const EncodeDev& e, int slices, void* work, cudaStream_t s) {
    const GramBulkShape g = gram_bulk_shape(e, slices);
    const dim3 tg((unsigned)g.kcn, (unsigned)g.nt);
    if (slices == 3)
        tc::k_gram_tab<3><<<tg, 256, 0, s>>>(e, g.kcn, (uint8_t*)work);
    else
        tc::k_gram_tab<2><<<tg, 256, 0, s>>>(e, g.kcn, (uint8_t*)work);
    note_launch();
    return cudaGetLastError();
}

cudaError_t gram_bulk_finish(const EncodeDev& e, double lambda, int slices, float4* G, int64_t ld, void* work,
                             cudaStream_t s) {
    const GramBulkShape g = gram_bulk_shape(e, slices);
    if (g.splits <= 1) return cudaSuccess;
    const int64_t n = e.N * e.N;
    k_gram_finalize<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
        e, lambda, (const float2*)((uint8_t*)work + g.tab_bytes), g.splits, g.nt * tc::BM, G, ld);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_gram_bulk(const EncodeDev& e, double lambda, int slices, float4* G, int64_t ld, void* work,
                             DevStatus* st, cudaStream_t s) {
    cudaError_t err = gram_bulk_table(e, slices, work, s);
    if (err != cudaSuccess) return err;
    int64_t items = 0;
    const tc::GramBulk p = gram_bulk_problem(e, lambda, slices, G, ld, work, &items);
    if ((err = run(p, dim3((unsigned)items, 1), slices, st, 1, s)) != cudaSuccess) return err;
    return gram_bulk_finish(e, lambda, slices, G, ld, work, s);
}

// ------------------------------------------------------------------ panel-internal updates (FP32 SIMT)
// Inside a 256-wide panel the solves and updates have K = 64: work of a few
// microseconds that a tensor-core launch spends on setting up TMEM, barriers and
// its pipeline. These kernels stage the 64-wide operands in shared memory and
// accumulate in FP32 (the accuracy class of the split-BF16 products).
constexpr int PNL_ROWS = 16;

// Both kernels: 16 rows per CTA, and each thread holds 2 rows (warp w: rows w and
// w + 8) x CB columns (lane + 32 b) of accumulators, so one shared-memory read
// serves several products. The column operand is stored k-major, so a warp reads
// 32 consecutive columns. Every output sums its 64 (zero-padded) k terms in
// order, with the same two FMAs per term as a one-output-per-thread loop.
// Operands are staged 16 loads per thread at a time, all issued before their
// stores, so a CTA waits for a few memory latencies rather than one per element.
__device__ inline void cmac_conj(float2& acc, float2 a, float2 b) {  // acc += a * conj(b)
    acc.x = fmaf(a.x, b.x, fmaf(a.y, b.y, acc.x));
    acc.y = fmaf(a.y, b.x, fmaf(-a.x, b.y, acc.y));
}

// L[i][k0 + j] = sum_k A[i][k] conj(Dinv[j][k]) for rows i >= row0, A[i][k] the
// FP32 rounding of G[i][k0 + k]: written to G (double-float) and to P (FP32)
__global__ void __launch_bounds__(256) k_trsm_panel(float2* P, int64_t ldp, const float2* __restrict__ Dinv32,
                                                  float4* G, int64_t ldg, int64_t k0, int nbk, int64_t row0,
                                                  int64_t N) {
    __shared__ float2 Dt[64][65];  // Dt[k][j] = Dinv[j][k]
    __shared__ float2 A[PNL_ROWS][64];
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int64_t i0 = row0 + (int64_t)blockIdx.x * PNL_ROWS;
    griddep_wait();
    griddep_launch();
    {
        float2 v[16], u[4];
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const int e = tid + 256 * t, j = e / 64, k = e % 64;
            v[t] = (j < nbk && k < nbk) ? Dinv32[j * 64 + k] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int e = tid + 256 * t, r = e / 64, k = e % 64;
            const int64_t i = i0 + r;
            u[t] = (i < N && k < nbk) ? df_to_f32(G[i * ldg + k0 + k]) : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const int e = tid + 256 * t;
            Dt[e % 64][e / 64] = v[t];
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int e = tid + 256 * t;
            A[e / 64][e % 64] = u[t];
        }
    }
    __syncthreads();
    float2 acc[2][2];
#pragma unroll
    for (int ra = 0; ra < 2; ++ra) acc[ra][0] = acc[ra][1] = make_float2(0.f, 0.f);
#pragma unroll 8
    for (int k = 0; k < 64; ++k) {
        const float2 a0 = A[w][k], a1 = A[w + 8][k], d0 = Dt[k][lane], d1 = Dt[k][lane + 32];
        cmac_conj(acc[0][0], a0, d0);
        cmac_conj(acc[0][1], a0, d1);
        cmac_conj(acc[1][0], a1, d0);
        cmac_conj(acc[1][1], a1, d1);
    }
#pragma unroll
    for (int ra = 0; ra < 2; ++ra) {
        const int64_t i = i0 + w + 8 * ra;
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const int j = lane + 32 * b;
            if (i < N && j < nbk) {
                G[i * ldg + k0 + j] = df_of_f32(acc[ra][b]);
                P[i * ldp + j] = acc[ra][b];
            }
        }
    }
}

// G[i][j] -= sum_k P[i][k] conj(P[j][k]) for t0 <= j < jmax, j <= i, rows r0 <= i < N
// (K = nbk <= 64; jmax - t0 <= 32 CB; r0 >= t0). Dynamic shared memory: herk_panel_smem(CB).
constexpr size_t herk_panel_smem(int cb) { return sizeof(float2) * (PNL_ROWS * 64 + 64 * (32 * cb + 1)); }
template <int CB>
__global__ void __launch_bounds__(256) k_herk_panel(const float2* __restrict__ P, int64_t ldp, float4* G,
                                                  int64_t ldg, int nbk, int64_t t0, int64_t jmax, int64_t r0,
                                                  int64_t N) {
    constexpr int WP = 32 * CB + 1;  // padded row of Bt: transposed stores spread over the banks
    extern __shared__ float2 pnl_smem[];
    float2(*Ai)[64] = reinterpret_cast<float2(*)[64]>(pnl_smem);
    float2(*Bt)[WP] = reinterpret_cast<float2(*)[WP]>(pnl_smem + PNL_ROWS * 64);  // Bt[k][c] = P[t0 + c][k]
    const int tid = threadIdx.x, w = tid >> 5, lane = tid & 31;
    const int W = (int)(jmax - t0);
    const int64_t i0 = r0 + (int64_t)blockIdx.x * PNL_ROWS;
    griddep_wait();
    griddep_launch();
    {
        float2 u[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int e = tid + 256 * t, r = e / 64, k = e % 64;
            const int64_t i = i0 + r;
            u[t] = (i < N && k < nbk) ? P[i * ldp + k] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int e = tid + 256 * t;
            Ai[e / 64][e % 64] = u[t];
        }
    }
#pragma unroll 1
    for (int t0b = 0; t0b < 8 * CB; t0b += 16) {  // 8 CB loads per thread, 16 at a time
        float2 v[16];
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const int e = tid + 256 * (t0b + t), c = e / 64, k = e % 64;
            const int64_t j = t0 + c;
            v[t] = (t0b + t < 8 * CB && c < W && j < N && k < nbk) ? P[j * ldp + k] : make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int t = 0; t < 16; ++t) {
            const int e = tid + 256 * (t0b + t);
            if (t0b + t < 8 * CB) Bt[e % 64][e / 64] = v[t];
        }
    }
    __syncthreads();
    float2 acc[2][CB];
#pragma unroll
    for (int b = 0; b < CB; ++b) acc[0][b] = acc[1][b] = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int k = 0; k < 64; ++k) {
        const float2 a0 = Ai[w][k], a1 = Ai[w + 8][k];
#pragma unroll
        for (int b = 0; b < CB; ++b) {
            const float2 bv = Bt[k][lane + 32 * b];
            cmac_conj(acc[0][b], a0, bv);
            cmac_conj(acc[1][b], a1, bv);
        }
    }
#pragma unroll
    for (int ra = 0; ra < 2; ++ra) {
        const int64_t i = i0 + w + 8 * ra;
#pragma unroll
        for (int b = 0; b < CB; ++b) {
            const int c = lane + 32 * b;
            const int64_t j = t0 + c;
            if (i < N && c < W && j <= i) G[i * ldg + j] = df_sub_f32(G[i * ldg + j], acc[ra][b]);
        }
    }
}

template <int CB>
static cudaError_t launch_herk_panel(const float2* P, int64_t ldp, float4* G, int64_t ldg, int nbk, int64_t t0,
                                     int64_t jmax, int64_t r0, int64_t N, cudaStream_t s) {
    static bool attr = false;
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(k_herk_panel<CB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)herk_panel_smem(CB));
        if (e != cudaSuccess) return e;
        attr = true;
    }
    const int64_t rows = N - r0;
    cudaError_t e = launch_pdl(k_herk_panel<CB>, dim3((unsigned)((rows + PNL_ROWS - 1) / PNL_ROWS)), dim3(256),
                               herk_panel_smem(CB), s, P, ldp, G, ldg, nbk, t0, jmax, r0, N);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// G[i][j] -= sum_k P[i][k] conj(P[j][k]) for columns t0 <= j < jmax (at most 192), rows r0 <= i < N
static cudaError_t herk_panel(const float2* P, int64_t ldp, float4* G, int64_t ldg, int nbk, int64_t t0,
                              int64_t jmax, int64_t r0, int64_t N, cudaStream_t s) {
    const int64_t w = jmax - t0;
    return w <= 64    ? launch_herk_panel<2>(P, ldp, G, ldg, nbk, t0, jmax, r0, N, s)
           : w <= 128 ? launch_herk_panel<4>(P, ldp, G, ldg, nbk, t0, jmax, r0, N, s)
                      : launch_herk_panel<6>(P, ldp, G, ldg, nbk, t0, jmax, r0, N, s);
}
static cudaError_t trsm_panel(float2* P, int64_t ldp, const float2* Dinv32, float4* G, int64_t ldg, int64_t k0,
                              int nbk, int64_t row0, int64_t N, cudaStream_t s) {
    cudaError_t e = launch_pdl(k_trsm_panel, dim3(cdiv(N - row0, PNL_ROWS)), dim3(256), 0, s, P, ldp, Dinv32, G,
                               ldg, k0, nbk, row0, N);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// Panel table (B tiles of conj(L), rows from r0, kw panel columns from p0)
size_t panel_table_bytes(int64_t N, int slices) {
    return (size_t)cdiv(N, tc::BM) * cdiv(256, tc::KC) * slices * tc::B_SL;
}
size_t factor_table_bytes(int64_t N, int slices) { return 2 * panel_table_bytes(N, slices); }
static cudaError_t panel_table(const float2* L32, int64_t N, int64_t p0, int64_t kw, int64_t r0, int slices,
                               uint8_t* tab, cudaStream_t s) {
    const dim3 g(cdiv(kw, tc::KC), cdiv(N - r0, tc::BM));
    const int64_t ld = N;
    cudaError_t e = slices == 3 ? launch_pdl(tc::k_tab_panel<3>, g, dim3(256), 0, s, (const float2*)L32, ld, N, p0,
                                             kw, r0, tab)
                                : launch_pdl(tc::k_tab_panel<2>, g, dim3(256), 0, s, (const float2*)L32, ld, N, p0,
                                             kw, r0, tab);
    return e != cudaSuccess ? e : cudaGetLastError();
}

// Two-level blocking: 64-wide diagonal blocks inside 256-wide panels. Inside a
// panel each step updates only the panel's remaining columns (K = 64); the
// trailing matrix gets one update per panel with K = 256, so its tiles run
// 16 tensor-core stages instead of 4 and G is read and written a quarter as
// often. G is in double-float storage (float4 per entry) for the whole
// factorisation, and L is left there in the same form.
constexpr int NBK = 64, NBP = 256;

cudaError_t launch_potrf_tc(float4* G, int64_t N, int64_t ld, double2* Dinv, float2* Dinv32, float2* L32,
                            int slices, DevStatus* st, cudaStream_t s, void* tab, const cudaEvent_t* ev_panel,
                            const TrailLookahead* la) {
    // lookahead: after each panel only the next panel's columns (two column tiles)
    // are updated on the chain's stream; the rest of the trailing matrix on la->s,
    // beside the next panel's steps, and before the next panel's update
    // (PINV_CHOL_LOOKAHEAD=0: all of it on the chain's stream). Every tile is
    // computed the same way either way, so the factor is the same bit for bit.
    const char* lenv = std::getenv("PINV_CHOL_LOOKAHEAD");
    const bool ahead = la && la->s && tab && !(lenv && std::strcmp(lenv, "0") == 0);
    int cap = 0;
    if (ahead) {
        const char* cenv = std::getenv("PINV_TRAIL_SMS");
        cap = cenv ? std::atoi(cenv) : (N <= 16384 ? std::max(1, 2 * tc::sm_count() / 5) : 0);
    }
    bool pending = false;  // a side update of the previous panel may still run
    // block lookahead inside a panel: after diagonal block k only the next block's
    // 64 rows are solved, and its diagonal block updated, on the chain's stream; the
    // rows below and the rest of the panel's columns go to la->s2 and run beside
    // diagonal block k + 1, whose solve of the rows below waits for them. Each row of
    // the solves and each entry of the updates is computed as without the lookahead.
    const bool bla = ahead && la->s2;
    bool side = false;  // la->s2 holds in-panel work the chain has not waited for
    for (int64_t p0 = 0; p0 < N; p0 += NBP) {
        const int64_t pend = std::min<int64_t>(N, p0 + NBP);
        for (int64_t k0 = p0; k0 < pend; k0 += NBK) {
            const int64_t nbk = std::min<int64_t>(NBK, N - k0);
            const int64_t kb = k0 / NBK;
            // the diagonal block writes its FP32 copy to L32; the solve below reads
            // its right-hand sides from G
            cudaError_t e =
                launch_potrf_diag_df(G, ld, N, k0, Dinv ? Dinv + kb * NBK * NBK : nullptr,
                                     Dinv32 + kb * NBK * NBK, L32, N, st, s);
            if (e != cudaSuccess) return e;
            const int64_t rest = N - k0 - nbk;
            if (rest <= 0) break;
            const int64_t t0 = k0 + nbk;
            const float2* Dk = Dinv32 + kb * NBK * NBK;
            if (side) {  // the rows below were updated by the previous block's side work
                if ((e = cudaStreamWaitEvent(s, la->ev_side, 0)) != cudaSuccess) return e;
                side = false;
            }
            if (bla && t0 < pend) {
                const int64_t t1 = std::min<int64_t>(t0 + NBK, pend);  // the next diagonal block
                if ((e = trsm_panel(L32 + k0, N, Dk, G, ld, k0, (int)nbk, t0, t1, s)) != cudaSuccess) return e;
                if ((e = herk_panel(L32 + k0, N, G, ld, (int)nbk, t0, t1, t0, t1, s)) != cudaSuccess) return e;
                if (t1 < N) {
                    if ((e = cudaEventRecord(la->ev_next, s)) != cudaSuccess) return e;
                    if ((e = cudaStreamWaitEvent(la->s2, la->ev_next, 0)) != cudaSuccess) return e;
                    if ((e = trsm_panel(L32 + k0, N, Dk, G, ld, k0, (int)nbk, t1, N, la->s2)) != cudaSuccess)
                        return e;
                    if ((e = herk_panel(L32 + k0, N, G, ld, (int)nbk, t0, pend, t1, N, la->s2)) != cudaSuccess)
                        return e;
                    if ((e = cudaEventRecord(la->ev_side, la->s2)) != cudaSuccess) return e;
                    side = true;
                }
                continue;
            }
            // panel solve of every row below the block
            if ((e = trsm_panel(L32 + k0, N, Dk, G, ld, k0, (int)nbk, t0, N, s)) != cudaSuccess) return e;
            if (t0 < pend) {  // the panel's remaining columns, all rows below
                if ((e = herk_panel(L32 + k0, N, G, ld, (int)nbk, t0, pend, t0, N, s)) != cudaSuccess) return e;
            }
        }
        if (side) {
            cudaError_t e = cudaStreamWaitEvent(s, la->ev_side, 0);
            if (e != cudaSuccess) return e;
            side = false;
        }
        if (ev_panel) {
            cudaError_t e = cudaEventRecord(ev_panel[p0 / NBP], s);
            if (e != cudaSuccess) return e;
        }
        if (pend < N) {  // trailing matrix, K = panel width
            cudaError_t e;
            if (tab) {
                const int64_t nt = cdiv(N - pend, tc::BM), kcn = cdiv(pend - p0, tc::KC);
                if (pending) {  // the previous panel's side update also writes these columns, and reads the table
                    if ((e = cudaStreamWaitEvent(s, la->ev_done, 0)) != cudaSuccess) return e;
                    pending = false;
                }
                if ((e = panel_table(L32, N, p0, pend - p0, pend, slices, (uint8_t*)tab, s)) != cudaSuccess) return e;
                const int64_t near = ahead ? std::min<int64_t>(nt, NBP / tc::BN) : nt;
                tc::HerkBulk hp{(const uint8_t*)tab, G, ld, N, pend, nt, kcn, slices, 0, near};
                e = run(hp, dim3((unsigned)(nt * near), 1), slices, st, 4, s, false, 0, true);
                if (e == cudaSuccess && near < nt) {
                    if ((e = cudaEventRecord(la->ev_tab, s)) != cudaSuccess) return e;
                    if ((e = cudaStreamWaitEvent(la->s, la->ev_tab, 0)) != cudaSuccess) return e;
                    tc::HerkBulk fp{(const uint8_t*)tab, G, ld, N, pend, nt, kcn, slices, near, nt - near};
                    if ((e = run(fp, dim3((unsigned)(nt * (nt - near)), 1), slices, la->st, 4, la->s, false, cap)) !=
                        cudaSuccess)
                        return e;
                    if ((e = cudaEventRecord(la->ev_done, la->s)) != cudaSuccess) return e;
                    pending = true;
                }
            } else {
                tc::HerkTC hp{L32 + p0, N, G, ld, N, pend - p0, pend, N};
                e = run(hp, dim3(cdiv(N - pend, tc::BN), cdiv(N - pend, tc::BM)), slices, st, 4, s);
            }
            if (e != cudaSuccess) return e;
        }
    }
    if (pending) {
        cudaError_t e = cudaStreamWaitEvent(s, la->ev_done, 0);
        if (e != cudaSuccess) return e;
    }
    return cudaGetLastError();
}

// Inside a panel the inverse's steps have K = 64, too short for the tensor-core
// engine's set-up (tensor-core launches of these steps took 27 / 44 us against a
// few microseconds of products): these FP32 SIMT kernels stage the 64-wide operands
// in shared memory, as the Cholesky's panel kernels do, and accumulate in FP32.
__device__ inline void cmac(float2& acc, float2 a, float2 b) {  // acc += a * b
    acc.x = fmaf(a.x, b.x, fmaf(-a.y, b.y, acc.x));
    acc.y = fmaf(a.x, b.y, fmaf(a.y, b.x, acc.y));
}

// W[k0 + i][j] = sum_k Dinv[i][k] W[k0 + k][j] (W rounded to FP32) for i < nbk, j < ncol:
// one CTA per 64 columns, each thread 4 x 4 outputs (rows ty + 16 a, columns tx + 16 b)
__global__ void __launch_bounds__(256) k_trtri_diag(const float2* __restrict__ Dinv32, float4* W, int64_t ld,
                                                  int64_t k0, int nbk, int64_t ncol) {
    __shared__ float2 Ds[64][65];  // Ds[i][k] = Dinv[i][k]
    __shared__ float2 Bs[64][65];  // Bs[k][c] = W[k0 + k][j0 + c]
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t j0 = (int64_t)blockIdx.x * 64;
    griddep_wait();
    griddep_launch();
#pragma unroll 4
    for (int t = 0; t < 16; ++t) {
        const int e = tid + 256 * t, r = e / 64, c = e % 64;
        Ds[r][c] = (r < nbk && c < nbk) ? Dinv32[r * 64 + c] : make_float2(0.f, 0.f);
        const int64_t j = j0 + c;
        Bs[r][c] = (r < nbk && j < ncol) ? df_to_f32(W[(k0 + r) * ld + j]) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2 acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = make_float2(0.f, 0.f);
#pragma unroll 4
    for (int k = 0; k < 64; ++k) {
        float2 dv[4], bv[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) dv[a] = Ds[ty + 16 * a][k];
#pragma unroll
        for (int b = 0; b < 4; ++b) bv[b] = Bs[k][tx + 16 * b];
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
            for (int b = 0; b < 4; ++b) cmac(acc[a][b], dv[a], bv[b]);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) {
        const int r = ty + 16 * a;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int64_t j = j0 + tx + 16 * b;
            if (r < nbk && j < ncol) W[(k0 + r) * ld + j] = df_of_f32(acc[a][b]);
        }
    }
}

// W[i][j] -= sum_k L[i][k0 + k] W[k0 + k][j] for rows r0 <= i < imax, j < ncol (K = nbk):
// one CTA per 16 rows x 64 columns, each thread 1 row x 4 columns
__global__ void __launch_bounds__(256) k_trtri_upd(const float2* __restrict__ L32, int64_t ldl, float4* W,
                                                 int64_t ld, int64_t k0, int nbk, int64_t r0, int64_t imax,
                                                 int64_t ncol) {
    __shared__ float2 As[16][65];  // As[r][k] = L[i0 + r][k0 + k]
    __shared__ float2 Bs[64][65];  // Bs[k][c] = W[k0 + k][j0 + c]
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int64_t j0 = (int64_t)blockIdx.x * 64, i0 = r0 + (int64_t)blockIdx.y * 16;
    griddep_wait();
    griddep_launch();
#pragma unroll
    for (int t = 0; t < 4; ++t) {
        const int e = tid + 256 * t, r = e / 64, k = e % 64;
        const int64_t i = i0 + r;
        As[r][k] = (i < imax && k < nbk) ? L32[i * ldl + k0 + k] : make_float2(0.f, 0.f);
    }
#pragma unroll 4
    for (int t = 0; t < 16; ++t) {
        const int e = tid + 256 * t, k = e / 64, c = e % 64;
        const int64_t j = j0 + c;
        Bs[k][c] = (k < nbk && j < ncol) ? df_to_f32(W[(k0 + k) * ld + j]) : make_float2(0.f, 0.f);
    }
    __syncthreads();
    float2 acc[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[b] = make_float2(0.f, 0.f);
#pragma unroll 8
    for (int k = 0; k < 64; ++k) {
        const float2 av = As[ty][k];
#pragma unroll
        for (int b = 0; b < 4; ++b) cmac(acc[b], av, Bs[k][tx + 16 * b]);
    }
    const int64_t i = i0 + ty;
    if (i >= imax) return;
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const int64_t j = j0 + tx + 16 * b;
        if (j < ncol) W[i * ld + j] = df_sub_f32(W[i * ld + j], acc[b]);
    }
}

// W = L^-1 by blocked forward substitution on I, with the same two levels:
// inside a 256-row panel each 64-row step updates the panel's rows only; the
// rows below get one update per panel with K = 256.
cudaError_t launch_trtri_tc(const float2* L32, int64_t N, const float2* Dinv32, float4* W, float2* W32,
                            int slices, DevStatus* st, cudaStream_t s, void* tab, const cudaEvent_t* ev_panel) {
    // W is in double-float storage while it is formed; the last pass leaves it in FP64
    cudaError_t e = launch_fill_identity_df(W, N, N, s);
    if (e != cudaSuccess) return e;
    // the inverse runs beside the Cholesky chain (and its trailing updates). Up to
    // N = 16384, where the chain is a latency-bound sequence of small launches, the
    // inverse's persistent launches take at most half the SMs so that the chain's
    // launches find free SMs; the trailing updates beside the chain take two fifths.
    // Measured at 64x64 (inverse / trailing SMs -> build): 114 / 38 -> 8.78 ms,
    // 152 / 50 -> 8.77 ms, 76 / 50 -> 8.63 ms, 76 / 64 -> 8.57 ms, 64 / 64 -> 8.56 ms,
    // any / 24 -> 9.3 ms and more (the trailing updates fall behind). Above
    // N = 16384 all three are throughput-bound
    // and each takes every SM. PINV_INV_SMS: another count (0 all).
    const char* cenv = std::getenv("PINV_INV_SMS");
    const int cap = cenv ? std::atoi(cenv) : (N <= 16384 ? std::max(1, tc::sm_count() / 2) : 0);
    for (int64_t p0 = 0; p0 < N; p0 += NBP) {
        const int64_t pend = std::min<int64_t>(N, p0 + NBP);
        if (ev_panel && (e = cudaStreamWaitEvent(s, ev_panel[p0 / NBP], 0)) != cudaSuccess) return e;
        for (int64_t k0 = p0; k0 < pend; k0 += NBK) {
            const int64_t nbk = std::min<int64_t>(NBK, N - k0);
            const int64_t ncol = k0 + nbk;
            if ((e = launch_pdl(k_trtri_diag, dim3(cdiv(ncol, 64)), dim3(256), 0, s, Dinv32 + (k0 / NBK) * NBK * NBK,
                                W, N, k0, (int)nbk, ncol)) != cudaSuccess)
                return e;
            if (ncol >= pend) continue;
            if ((e = launch_pdl(k_trtri_upd, dim3(cdiv(ncol, 64), cdiv(pend - ncol, 16)), dim3(256), 0, s, L32, N, W,
                                N, k0, (int)nbk, ncol, pend, ncol)) != cudaSuccess)
                return e;
        }
        if (pend < N) {
            if (tab) {
                const int64_t ntr = cdiv(N - pend, tc::BM), ntc = cdiv(pend, tc::BN), kcn = cdiv(pend - p0, tc::KC);
                uint8_t* tabl = (uint8_t*)tab;
                uint8_t* tabw = tabl + panel_table_bytes(N, slices);
                if ((e = panel_table(L32, N, p0, pend - p0, pend, slices, tabl, s)) != cudaSuccess) return e;
                const dim3 wg((unsigned)kcn, (unsigned)ntc);
                const float4* Wc = W;
                e = slices == 3 ? launch_pdl(tc::k_tab_wrows<3>, wg, dim3(256), 0, s, Wc, N, p0, pend - p0, pend, tabw)
                                : launch_pdl(tc::k_tab_wrows<2>, wg, dim3(256), 0, s, Wc, N, p0, pend - p0, pend, tabw);
                if (e != cudaSuccess || (e = cudaGetLastError()) != cudaSuccess) return e;
                tc::TrtriBulk up{tabl, tabw, W, N, N, pend, ntr, ntc, kcn, slices};
                if ((e = run(up, dim3((unsigned)(ntr * ntc), 1), slices, st, 6, s, false, cap, true)) != cudaSuccess)
                    return e;
            } else {
                tc::TrtriUpdTC up{L32, N, W, N, N, p0, pend - p0, N};
                if ((e = run(up, dim3(cdiv(pend, tc::BN), cdiv(N - pend, tc::BM)), slices, st, 6, s, false, cap)) !=
                    cudaSuccess)
                    return e;
            }
        }
    }
    return launch_df_finish(W, N, N, NBK, W32, s);  // above the diagonal only k_trtri_diag writes
}

cudaError_t launch_recon_tc(const EncodeDev& e, const float2* W32, const float2* WT32, float2* T, int slices,
                            float2* R, DevStatus* st, cudaStream_t s) {
    const int64_t M = e.Mk * e.C;
    tc::ReconStep1TC p1{e, W32, T};
    // step-1 tiles get longer with the row (W is lower triangular): longest first
    cudaError_t err = run(p1, dim3(cdiv(M, tc::BN), cdiv(e.N, tc::BM)), slices, st, 2, s, true);
    if (err != cudaSuccess) return err;
    tc::ReconStep2TC p2{WT32, T, R, e.N, M};
    return run(p2, dim3(cdiv(e.N, tc::BM), cdiv(M, tc::BN)), slices, st, 8, s);
}

namespace {
struct ReconBulkShape {
    int64_t nt, kcn, mt, rows, chunks;  // voxel tiles, voxel chunks, sample tiles, sample tiles per chunk
    size_t wb_bytes, et_bytes;
};
// ET + TT of one chunk of samples: 4 GiB, or PINV_RECON_CHUNK_MB
size_t recon_chunk_bytes() {
    const char* v = std::getenv("PINV_RECON_CHUNK_MB");
    const long mb = v ? std::atol(v) : 0;
    return mb > 0 ? (size_t)mb << 20 : size_t(4) << 30;
}
ReconBulkShape recon_bulk_shape(const EncodeDev& e, int slices) {
    ReconBulkShape r;
    r.nt = (e.N + tc::BM - 1) / tc::BM;
    r.kcn = r.nt * (tc::BM / tc::KC);
    r.mt = (e.Mk * e.C + tc::BM - 1) / tc::BM;
    const size_t per_tile = 2 * (size_t)r.kcn * slices * tc::A_SL;
    int64_t cap = (int64_t)(recon_chunk_bytes() / per_tile);
    if (cap < 1) cap = 1;
    r.chunks = (r.mt + cap - 1) / cap;
    r.rows = (r.mt + r.chunks - 1) / r.chunks;
    r.wb_bytes = (size_t)r.nt * r.kcn * slices * tc::B_SL;
    r.et_bytes = (size_t)r.rows * r.kcn * slices * tc::A_SL;
    return r;
}
struct ReconWork {
    uint8_t *wb1, *wb2, *et, *tt;
};
ReconWork recon_work(const ReconBulkShape& r, void* work) {
    ReconWork w;
    w.wb1 = (uint8_t*)work;
    w.wb2 = w.wb1 + r.wb_bytes;
    w.et = w.wb2 + r.wb_bytes;
    w.tt = w.et + r.et_bytes;
    return w;
}
int64_t chunk_rows(const ReconBulkShape& r, int64_t c) {
    const int64_t t0 = c * r.rows;
    return t0 >= r.mt ? 0 : std::min(r.rows, r.mt - t0);
}
tc::ReconB1 recon_b1_problem(const EncodeDev& e, int slices, void* work, int64_t c, int64_t* items) {
    const ReconBulkShape r = recon_bulk_shape(e, slices);
    const ReconWork w = recon_work(r, work);
    const int64_t rows = chunk_rows(r, c);
    *items = rows * r.nt;
    return tc::ReconB1{w.et, w.wb1, w.tt, rows, r.nt, r.kcn, slices};
}
tc::ReconB2 recon_b2_problem(const EncodeDev& e, int slices, float2* R, void* work, int64_t c, int64_t* items) {
    const ReconBulkShape r = recon_bulk_shape(e, slices);
    const ReconWork w = recon_work(r, work);
    const int64_t rows = chunk_rows(r, c), M = e.Mk * e.C, j_off = c * r.rows * tc::BM;
    *items = rows * r.nt;
    return tc::ReconB2{w.tt, w.wb2, R, rows, r.nt, r.kcn, e.N, M, j_off, std::min(rows * tc::BM, M - j_off), slices};
}
}  // namespace

size_t recon_bulk_bytes(const EncodeDev& e, int slices) {
    const ReconBulkShape r = recon_bulk_shape(e, slices);
    return 2 * r.wb_bytes + 2 * r.et_bytes;
}

int64_t recon_bulk_chunks(const EncodeDev& e, int slices) { return recon_bulk_shape(e, slices).chunks; }

cudaError_t recon_bulk_wtables(const EncodeDev& e, const float2* W32, int slices, void* work, cudaStream_t s) {
    const ReconBulkShape r = recon_bulk_shape(e, slices);
    const ReconWork w = recon_work(r, work);
    const dim3 wg((unsigned)r.kcn, (unsigned)r.nt);
    for (int lower = 1; lower >= 0; --lower) {
        if (slices == 3)
            tc::k_tab_w<3><<<wg, 256, 0, s>>>(W32, e.N, r.kcn, lower, lower ? w.wb1 : w.wb2);
        else
            tc::k_tab_w<2><<<wg, 256, 0, s>>>(W32, e.N, r.kcn, lower, lower ? w.wb1 : w.wb2);
        note_launch();
    }
    return cudaGetLastError();
}

cudaError_t recon_bulk_et(const EncodeDev& e, int slices, void* work, int64_t c, cudaStream_t s) {
    const ReconBulkShape r = recon_bulk_shape(e, slices);
    const ReconWork w = recon_work(r, work);
    const int64_t rows = chunk_rows(r, c);
    if (rows <= 0) return cudaSuccess;
    const dim3 eg((unsigned)r.kcn, (unsigned)rows);
    const int64_t j_off = c * r.rows * tc::BM;
    if (slices == 3)
        tc::k_tab_et<3><<<eg, 256, 0, s>>>(e, r.kcn, j_off, w.et);
    else
        tc::k_tab_et<2><<<eg, 256, 0, s>>>(e, r.kcn, j_off, w.et);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_recon_bulk(const EncodeDev& e, const float2* W32, int slices, float2* R, void* work,
                              DevStatus* st, cudaStream_t s) {
    cudaError_t err = recon_bulk_wtables(e, W32, slices, work, s);
    if (err != cudaSuccess) return err;
    const int64_t chunks = recon_bulk_chunks(e, slices);
    for (int64_t c = 0; c < chunks; ++c) {
        if ((err = recon_bulk_et(e, slices, work, c, s)) != cudaSuccess) return err;
        int64_t items = 0;
        const tc::ReconB1 p1 = recon_b1_problem(e, slices, work, c, &items);
        if ((err = run(p1, dim3((unsigned)items, 1), slices, st, 2, s)) != cudaSuccess) return err;
        const tc::ReconB2 p2 = recon_b2_problem(e, slices, R, work, c, &items);
        if ((err = run(p2, dim3((unsigned)items, 1), slices, st, 8, s)) != cudaSuccess) return err;
    }
    return cudaSuccess;
}

// ------------------------------------------------------------------ refinement correction (host)
namespace {
// k ranges of the correction: about two tiles per SM, at least 256 wide
// k chunk of the correction's triangular products: row tile r holds the
// nonempty chunks below min((r + 1) BM, N); the chunk that minimises whole waves of
// those tiles x (chunk + per-tile overhead), at least 256 columns
int64_t correct_tc_chunk(int64_t N) {
    const int64_t rows = (N + tc::BM - 1) / tc::BM, sms = tc::sm_count();
    const int64_t hi = std::max<int64_t>(1, std::min<int64_t>(64, N / 256));
    int64_t best = 0;
    double bt = 0.0;
    for (int64_t sp = 1; sp <= hi; ++sp) {
        const int64_t chunk = ((N + sp - 1) / sp + tc::KC - 1) / tc::KC * tc::KC;
        int64_t tiles = 0;
        for (int64_t r = 0; r < rows; ++r) tiles += (std::min<int64_t>((r + 1) * tc::BM, N) + chunk - 1) / chunk;
        const double t = (double)((tiles + sms - 1) / sms) * (double)(chunk + 256);
        if (best == 0 || t < bt * (1.0 - 1e-9)) {
            bt = t;
            best = chunk;
        }
    }
    return best;
}
}  // namespace

// T[f][i] = sum of the nonempty splits (k range below the end of i's row tile), in order
__global__ void k_corr_reduce_w(const float2* __restrict__ part, int64_t N, int64_t F, int64_t chunk,
                                float2* __restrict__ T) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * F) return;
    const int64_t f = idx / N, i = idx - f * N;
    const int64_t kend = (i / tc::BM + 1) * tc::BM, kmax = kend < N ? kend : N;
    float2 a = make_float2(0.f, 0.f);
    for (int64_t sp = 0; sp * chunk < kmax; ++sp) {
        const float2 b = part[(sp * F + f) * N + i];
        a.x += b.x;
        a.y += b.y;
    }
    T[f * N + i] = a;
}
// X[f][n] += sum of the nonempty splits (k range reaching n's row tile), in order
__global__ void k_corr_reduce_wh(const float2* __restrict__ part, int64_t N, int64_t F, int64_t chunk,
                                 double2* __restrict__ X) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * F) return;
    const int64_t f = idx / N, n = idx - f * N;
    const int64_t n0 = n / tc::BM * tc::BM;
    double2 a = make_double2(0.0, 0.0);
    for (int64_t sp = n0 / chunk; sp * chunk < N; ++sp) {
        const float2 b = part[(sp * F + f) * N + n];
        a.x += (double)b.x;
        a.y += (double)b.y;
    }
    double2 x = X[f * N + n];
    X[f * N + n] = make_double2(x.x + a.x, x.y + a.y);
}

// the fewest frames for which the refinement's correction runs on the tensor cores:
// every count (a 64x64 apply of 1-6 frames: 5.4 ms with the SIMT W products, 1.8 ms
// here). PINV_CORR_TC_MIN_FRAMES: another count.
static int64_t correct_tc_min_frames() {
    static const int64_t v = [] {
        const char* e = std::getenv("PINV_CORR_TC_MIN_FRAMES");
        return e ? std::max<int64_t>(1, std::atoll(e)) : (int64_t)1;
    }();
    return v;
}
bool correct_tc_ok(int64_t F) { return F >= correct_tc_min_frames() && tc_available(); }

size_t correct_tc_work_elems(int64_t N, int64_t F) {
    const int64_t chunk = correct_tc_chunk(N), sp = (N + chunk - 1) / chunk;
    return (size_t)(sp * std::min<int64_t>(F, tc::BN) * N);
}

cudaError_t launch_correct_tc(const float2* W32, int64_t N, const double2* R, int64_t F, float2* T, double2* X,
                              float2* work, int slices, DevStatus* sched, cudaStream_t s) {
    const int64_t chunk = correct_tc_chunk(N), sp = (N + chunk - 1) / chunk;
    for (int64_t f0 = 0; f0 < F; f0 += tc::BN) {
        const int64_t Fc = std::min<int64_t>(tc::BN, F - f0);
        const int64_t n = N * Fc;
        const unsigned rb = (unsigned)((n + 255) / 256);
        tc::CorrW p1{W32, R + f0 * N, work, N, Fc, chunk};
        cudaError_t e = run(p1, dim3((unsigned)sp, cdiv(N, tc::BM)), slices, sched, 10, s);
        if (e != cudaSuccess) return e;
        k_corr_reduce_w<<<rb, 256, 0, s>>>(work, N, Fc, chunk, T + f0 * N);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        tc::CorrWH p2{W32, T + f0 * N, work, N, Fc, chunk};
        if ((e = run(p2, dim3((unsigned)sp, cdiv(N, tc::BM)), slices, sched, 11, s)) != cudaSuccess) return e;
        k_corr_reduce_wh<<<rb, 256, 0, s>>>(work, N, Fc, chunk, X + f0 * N);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// ------------------------------------------------------------------ batched launches
cudaError_t tc_multi_create(int kind, const TcPlanArgs* a, int n, int slices, int64_t chunk, TcMulti* out) {
    *out = TcMulti{};
    out->kind = kind;
    std::vector<int64_t> start(1, 0), gx;
    std::vector<unsigned char> probs;  // problem descriptors, stride sizeof(problem)
    // plans with the longest tiles first (K per tile: M_k for the Gram, up to N for Recon)
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        const int64_t kx = kind == TC_MULTI_GRAM ? a[x].e->Mk : a[x].e->N;
        const int64_t ky = kind == TC_MULTI_GRAM ? a[y].e->Mk : a[y].e->N;
        return kx > ky;
    });
    for (int ii = 0; ii < n; ++ii) {
        const int i = order[ii];
        const EncodeDev& e = *a[i].e;
        int64_t items = 0;
        if (kind == TC_MULTI_GRAM) {
            const tc::GramBulk p = gram_bulk_problem(e, a[i].lam, slices, a[i].G, e.N, a[i].work, &items);
            probs.insert(probs.end(), (const unsigned char*)&p, (const unsigned char*)&p + sizeof(p));
        } else {
            if (chunk >= recon_bulk_chunks(e, slices)) continue;
            if (kind == TC_MULTI_RECON1) {
                const tc::ReconB1 p = recon_b1_problem(e, slices, a[i].work, chunk, &items);
                probs.insert(probs.end(), (const unsigned char*)&p, (const unsigned char*)&p + sizeof(p));
            } else {
                const tc::ReconB2 p = recon_b2_problem(e, slices, a[i].R, a[i].work, chunk, &items);
                probs.insert(probs.end(), (const unsigned char*)&p, (const unsigned char*)&p + sizeof(p));
            }
        }
        gx.push_back(items);  // bulk problems decode their own tile from the item index
        start.push_back(start.back() + items);
    }
    out->n = (int)gx.size();
    out->items = start.back();
    if (out->n == 0) return cudaSuccess;
    out->off_start = (probs.size() + 255) & ~(size_t)255;
    out->off_gx = out->off_start + ((sizeof(int64_t) * (out->n + 1) + 255) & ~(size_t)255);
    const size_t bytes = out->off_gx + sizeof(int64_t) * out->n;
    cudaError_t e = cudaMalloc(&out->buf, bytes);
    if (e != cudaSuccess) return e;
    unsigned char* b = (unsigned char*)out->buf;
    if ((e = cudaMemcpy(b, probs.data(), probs.size(), cudaMemcpyHostToDevice)) != cudaSuccess) return e;
    if ((e = cudaMemcpy(b + out->off_start, start.data(), sizeof(int64_t) * (out->n + 1),
                        cudaMemcpyHostToDevice)) != cudaSuccess)
        return e;
    return cudaMemcpy(b + out->off_gx, gx.data(), sizeof(int64_t) * out->n, cudaMemcpyHostToDevice);
}

template <int S>
static cudaError_t multi_launch_s(const TcMulti& m, DevStatus* st, cudaStream_t s) {
    const unsigned char* b = (const unsigned char*)m.buf;
    const int64_t* start = (const int64_t*)(b + m.off_start);
    const int64_t* gx = (const int64_t*)(b + m.off_gx);
    if (m.kind == TC_MULTI_GRAM)
        return tc::launch_many<S>((const tc::GramBulk*)b, start, gx, m.n, m.items, st, 1, s);
    if (m.kind == TC_MULTI_RECON1)
        return tc::launch_many<S>((const tc::ReconB1*)b, start, gx, m.n, m.items, st, 2, s);
    return tc::launch_many<S>((const tc::ReconB2*)b, start, gx, m.n, m.items, st, 8, s);
}

cudaError_t tc_multi_launch(const TcMulti& m, int slices, DevStatus* st, cudaStream_t s) {
    if (m.n == 0 || m.items == 0) return cudaSuccess;
    return slices == 3 ? multi_launch_s<3>(m, st, s) : multi_launch_s<2>(m, st, s);
}

void tc_multi_free(TcMulti* m) {
    if (m->buf) cudaFree(m->buf);
    *m = TcMulti{};
}

namespace tc {
// SMs of the current device (persistent grids hold one CTA per SM)
int sm_count() {
    static int cached_dev = -1, cached = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (dev != cached_dev) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
        cached = n;
        cached_dev = dev;
    }
    return cached;
}
}  // namespace tc

bool tc_available() {
    int dev = 0, major = 0, minor = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) return false;
    return major == 10 && minor == 3;
}

namespace tc {
// ------------------------------------------------------------------ Recon x data on the tensor cores
// X[f][n] = sum_j Recon[n][j] D[f][j] for frames f < F <= BN. The sample range is
// split over tile columns: column tile bx covers frames 0..BN-1 of split bx
// (samples [bx * chunk, ...)), whose FP32 partials go to part[bx][f][n].
struct ApplyTC {
    static constexpr bool kPrefetch = true;  // Recon streams from HBM
    const float2* R;   // Recon [N][M], c64
    const float2* D;   // data [F][M], c64
    float2* part;      // [splits][F][N]
    int64_t N, M, F, chunk;
    __device__ bool tile(int64_t bx, int64_t by, int64_t& i0, int64_t& j0, int64_t& kb, int64_t& ke) const {
        i0 = by * BM;
        j0 = bx * BN;
        kb = bx * chunk;
        ke = kb + chunk < M ? kb + chunk : M;
        return true;
    }
    __device__ RowPtr row_a(int64_t i) const { return RowPtr{R + (i < N ? i : 0) * M, i < N}; }
    __device__ RowPtr row_b(int64_t j) const {
        const int64_t f = j % BN;
        return RowPtr{D + (f < F ? f : 0) * M, f < F};
    }
    __device__ void a8(const RowPtr& r, int64_t k, int64_t ke, float2 (&v)[8]) const {
        load8f(r.p + k, r.ok ? (int)(ke - k) : 0, v);
    }
    __device__ void b8(const RowPtr& r, int64_t k, int64_t ke, float2 (&v)[8]) const {
        load8f(r.p + k, r.ok ? (int)(ke - k) : 0, v);
    }
    __device__ bool row_ok(int64_t i) const { return i < N; }
    __device__ bool col_ok(int64_t j) const { return j % BN < F; }
    __device__ void store(int64_t i, int64_t j, float2 v) const {
        part[((j / BN) * F + j % BN) * N + i] = v;
    }
};
}  // namespace tc

// ------------------------------------------------------------------ FP32 SIMT apply
// X[f][n] = sum_j R[n][j] D[f][j] for c64 Recon and data (frames along the tile's columns).
template <int BMv, int BNv, int TM, int TN, int BKv>
__global__ void __launch_bounds__(256) k_apply32(const float2* __restrict__ R, int64_t N, int64_t M,
                                                 const float2* __restrict__ D, int64_t F, float2* __restrict__ X) {
    constexpr int TX = BNv / TN, TY = BMv / TM;
    static_assert(TX * TY == 256, "256 threads");
    __shared__ float2 As[BKv][BMv + 1];
    __shared__ float2 Bs[BKv][BNv + 1];
    const int64_t i0 = (int64_t)blockIdx.y * BMv, j0 = (int64_t)blockIdx.x * BNv;
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    float2 acc[TM][TN];
#pragma unroll
    for (int r = 0; r < TM; ++r)
#pragma unroll
        for (int c = 0; c < TN; ++c) acc[r][c] = make_float2(0.f, 0.f);
    for (int64_t k0 = 0; k0 < M; k0 += BKv) {
        for (int e = tid; e < BKv * BMv; e += 256) {
            const int kk = e % BKv, ii = e / BKv;
            const int64_t gi = i0 + ii, gk = k0 + kk;
            As[kk][ii] = (gi < N && gk < M) ? R[gi * M + gk] : make_float2(0.f, 0.f);
        }
        for (int e = tid; e < BKv * BNv; e += 256) {
            const int kk = e % BKv, jj = e / BKv;
            const int64_t gj = j0 + jj, gk = k0 + kk;
            Bs[kk][jj] = (gj < F && gk < M) ? D[gj * M + gk] : make_float2(0.f, 0.f);
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < BKv; ++kk) {
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
            if (gi < N && gj < F) X[gj * N + gi] = acc[r][c];
        }
}

template <int BMv, int BNv, int TM, int TN, int BKv>
static cudaError_t apply32_shape(const float2* R, int64_t N, int64_t M, const float2* D, int64_t F, float2* X,
                                 cudaStream_t s) {
    dim3 grid(cdiv(F, BNv), cdiv(N, BMv));
    k_apply32<BMv, BNv, TM, TN, BKv><<<grid, 256, 0, s>>>(R, N, M, D, F, X);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_apply_reduce(const float2* __restrict__ part, int splits, int64_t n, float2* __restrict__ X) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float2 a = part[i];
    for (int z = 1; z < splits; ++z) {
        const float2 b = part[(int64_t)z * n + i];
        a.x += b.x;
        a.y += b.y;
    }
    X[i] = a;
}

// splits of the sample range: about two tiles per SM, chunks of at least 1024 samples
// sample-range parts of the tensor-core apply: whole waves of tiles, parts of at
// least 1024 samples
int apply_tc_splits(int64_t N, int64_t M) {
    const int64_t rows = (N + tc::BM - 1) / tc::BM;
    const int hi = (int)std::max<int64_t>(1, std::min<int64_t>(64, M / 1024));
    return tc::wave_splits(rows, M, 1, hi, 256);
}

// the fewest frames for which Recon x data runs on the tensor cores: every count
// (a 64x64, 8-coil Recon applied to 1-12 frames: 8.9-9.2 ms by the SIMT kernel,
// 24.5 ms at 8, and 2.9-3.0 ms here). PINV_APPLY_TC_MIN_FRAMES: another count.
static int64_t apply_tc_min_frames() {
    static const int64_t v = [] {
        const char* e = std::getenv("PINV_APPLY_TC_MIN_FRAMES");
        return e ? std::max<int64_t>(1, std::atoll(e)) : (int64_t)1;
    }();
    return v;
}
bool apply_tc_ok(int64_t F) { return F >= apply_tc_min_frames() && tc_available(); }

size_t apply_tc_work_elems(int64_t N, int64_t M, int64_t F) {
    return (size_t)apply_tc_splits(N, M) * (size_t)N * (size_t)std::min<int64_t>(F, tc::BN);
}

// frames in chunks of BN (one column tile per split)
cudaError_t launch_apply_tc(const float2* R, int64_t N, int64_t M, const float2* D, int64_t F, float2* X,
                            float2* work, int slices, DevStatus* st, cudaStream_t s) {
    const int sp = apply_tc_splits(N, M);
    const int64_t chunk = ((M + sp - 1) / sp + tc::KC - 1) / tc::KC * tc::KC;
    for (int64_t f0 = 0; f0 < F; f0 += tc::BN) {
        const int64_t Fc = std::min<int64_t>(tc::BN, F - f0);
        tc::ApplyTC p{R, D + f0 * M, work, N, M, Fc, chunk};
        cudaError_t e = run(p, dim3((unsigned)sp, cdiv(N, tc::BM)), slices, st, 9, s);
        if (e != cudaSuccess) return e;
        const int64_t n = N * Fc;
        k_apply_reduce<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(work, sp, n, X + f0 * N);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Tile shape per frame-count class, chosen by the autotuner (all candidates
// sum over the rows of Recon in the same order).
cudaError_t launch_apply32(const float2* R, int64_t N, int64_t M, const float2* D, int64_t F, float2* X,
                           cudaStream_t s) {
    if (F == 0) return cudaSuccess;
    if (F >= 48) {
        auto run = [&](int c) -> cudaError_t {
            switch (c) {
                case 1: return apply32_shape<128, 64, 8, 4, 16>(R, N, M, D, F, X, s);
                case 2: return apply32_shape<32, 64, 2, 4, 32>(R, N, M, D, F, X, s);
                case 3: return apply32_shape<64, 32, 4, 2, 32>(R, N, M, D, F, X, s);
                default: return apply32_shape<64, 64, 4, 4, 32>(R, N, M, D, F, X, s);
            }
        };
        return run(tune_pick("apply32", N, F, 4, run, s));
    }
    if (F >= 8) {
        auto run = [&](int c) -> cudaError_t {
            switch (c) {
                case 1: return apply32_shape<128, 16, 8, 1, 16>(R, N, M, D, F, X, s);
                case 2: return apply32_shape<32, 16, 2, 1, 32>(R, N, M, D, F, X, s);
                default: return apply32_shape<64, 16, 4, 1, 32>(R, N, M, D, F, X, s);
            }
        };
        return run(tune_pick("apply32", N, F, 3, run, s));
    }
    auto run = [&](int c) -> cudaError_t {
        switch (c) {
            case 1: return apply32_shape<128, 2, 1, 1, 16>(R, N, M, D, F, X, s);
            default: return apply32_shape<256, 1, 1, 1, 16>(R, N, M, D, F, X, s);
        }
    };
    return run(tune_pick("apply32", N, F, 2, run, s));
}

}  // namespace pinv

extern "C" int pinv_tc_available(void) { return pinv::tc_available() ? 1 : 0; }
