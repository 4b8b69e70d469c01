// E^H d formed exactly on the tensor cores (fixed-point digit splitting).
//
// b[f][n] = sum_j conj(E[j][n]) d[f][j] must be accurate to about 1e-10
// relative for the refinement (its fixed point solves G x = b; errors in b
// grow by kappa(G)). The double-float SIMT kernel reaches that at 48 FP32
// instructions per complex MAC; this kernel reaches it with bf16 MMAs whose
// every product and partial sum is an exact integer:
//
//  * The coil factor is taken out: the sample range is split at coil
//    boundaries, each CTA forms sum_m conj(A[m][n]) d_c[f][m] with the
//    coil-free |A| = 1, and multiplies its double-float partial by
//    conj(s_c(n)) before the ordered reduction over all splits.
//  * Each real operand value x, scaled by a power of two so |x| <= 1 (A needs
//    none; data by the largest component of its frame), is written as
//    x = sum_i x_i 2^(-6-7i), i = 0..5, with integer digits |x_i| <= 64
//    (exact in bf16); the remainder is below 2^-42.
//  * Digit products x_i y_j are integers of at most 12 bits, exact in the FP32
//    accumulator, and so is every partial sum below 2^24. Pairs with the same
//    weight class w = i + j accumulate in one TMEM region (six regions of 64
//    columns); the 21 pairs with w <= 5 are kept (dropped pairs weigh below
//    2^-42 relative).
//  * Every DRAIN stages (each class sum then stays below 2^24) the producer
//    warps read the six regions, scale class w by 2^(-12-7w) (exact) and add
//    it into double-float accumulators held in registers.
//
// Tiles are 128 voxels x 32 frames (64 output columns, real and imaginary side
// by side, as in the split-BF16 engine), or 128 x 8 for calls of at most eight
// frames (the condition estimate's two vectors, small requests: the MMAs of a
// 32-frame tile would be mostly padding); the sample range is split over CTAs
// and the double-float partials reduced in a fixed order. One MMA takes an A
// digit against up to four B digits stacked along N (N <= 256, or 64 for the
// narrow tile), so a stage's 21 digit pairs cost 8 MMAs per 16-deep k half. Every
// entry's digit products, class sums and drains are the same whatever the tile. The producers form conj(A) from the
// separable phase tables of plans without B0; plans with B0 copy the digits of
// conj(A) (with its B0 factor) from a per-build table.
//
// The forward product E x (XFWD) runs the same way with the roles of samples and
// voxels exchanged: the A operand is a per-build table of the digits of A itself
// (rows of 128 samples, k = voxels), the B operand the digits of s_c(n) x[f][n]
// per coil, and each coil's samples get their own partial sums, reduced into
// u = d - E x. With both, the refinement residual r = E^H (d - E x) - lambda x of
// plans with B0 runs on the tensor cores too.
//
// The digits of the B operand (data, or x) are written once per call by
// k_b_digits. The digits of the A operand either come from the producer warps
// (XGEN) or are copied with one bulk copy per stage from a table in the stage layout:
// the exact Gram's digit tiles for the refinement residual (XGRAM), or the
// digits of conj(A) written once per build (XADJT; the same digits XGEN
// forms, which it would otherwise form again for every coil and frame tile).
#include <algorithm>
#include <cstdlib>

#include "df.cuh"
#include "tc_engine.cuh"

namespace pinv {
namespace tcx {

using namespace tc;

constexpr int XM = 128;        // voxels per tile
constexpr int XN = 32;         // frames per tile (MMA N = 64 per B digit)
constexpr int XNN = 8;         // frames per tile of the narrow variant (MMA N = 16 per B digit)
constexpr int XKC = 16;        // complex samples per stage
constexpr int NDIG = 6;        // digits per real value
constexpr int NCLS = 6;        // weight classes kept (i + j <= 5)
constexpr int XDRAIN = 16;     // stages per exact accumulation group
constexpr int XSTAGES = 3;
constexpr int XA_SL = XM * 64;         // one digit slice of A: 128 rows x 32 bf16 = 8 KiB
// per frame-tile width XNT: one digit slice of B (2 XNT stacked rows x 32 bf16: 4 KiB
// for 32 frames), a stage (72 KiB for 32 frames) and the dynamic shared memory
template <int XNT>
struct XS {
    static constexpr int B_SL = 2 * XNT * 64;
    static constexpr int STAGE = NDIG * (XA_SL + B_SL);
    static constexpr int SMEM = XSTAGES * STAGE + 1024;
};
// bf16 x bf16 -> f32, K-major operands, M = XM, N = n
__host__ __device__ constexpr uint32_t xidesc(int n) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(XM >> 4) << 24);
}
// The B digit slices lie one after another (B_SL apart, 8-row groups 512 B apart
// throughout), so slices j0 .. j0 + nd - 1 form one operand of 2 XNT nd rows, and
// the classes i + j of A digit i are adjacent TMEM regions of 2 XNT columns: one
// MMA covers several digit pairs. Per A digit i: (first B slice, B slices) of its
// MMAs, at most four slices.
struct XPairRun {
    int i, j0, nd;
};
__device__ __forceinline__ XPairRun xrun(int r) {
    constexpr XPairRun t[8] = {{0, 0, 4}, {0, 4, 2}, {1, 0, 4}, {1, 4, 1},
                               {2, 0, 4}, {3, 0, 3}, {4, 0, 2}, {5, 0, 1}};
    return t[r];
}
// Per class and group: at most 6 pairs x 32 products x XDRAIN stages, each below 2^12.
static_assert(NCLS * 32 * XDRAIN * 4096 < (1 << 24), "exact class sums");

__device__ inline float rint_f(float x) { return rintf(x); }

// Digits of 8 double-float values (h, l) times `scale` (a power of two),
// written slice by slice: w[t] packs values 2t, 2t+1 of digit `dig` as bf16.
struct Digits8 {
    float rh[8], rl[8];
    __device__ void init(const float (&h)[8], const float (&l)[8], float scale) {
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            rh[t] = h[t] * (scale * 64.f);
            rl[t] = l[t] * (scale * 64.f);
        }
    }
    // next digit of every value, packed in 4 words; the remainder moves up by 2^7.
    // (rh, rl) stays a normalised pair, so r = rh - d is either 0 or at least
    // ulp(rh) > |rl| and the fast two-sum is exact.
    __device__ void next(uint32_t (&w)[4], uint32_t flip) {
        float d[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
            d[t] = rint_f(rh[t]);
            float s, e;
            fast_two_sum(rh[t] - d[t], rl[t], s, e);  // rh - d is exact
            rh[t] = s * 128.f;
            rl[t] = e * 128.f;
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            __nv_bfloat162 v = __floats2bfloat162_rn(d[2 * t], d[2 * t + 1]);  // exact: |d| <= 64
            w[t] = *reinterpret_cast<uint32_t*>(&v) ^ flip;
        }
    }
};

struct XArgs {
    EncodeDev e;
    const double2* D;   // adjoint: data [F][M]; Gram residual: x [F][N] (FP64)
    const int* fexp;    // per-frame exponent: |D_f| <= 2^fexp
    int64_t F, M;
    int64_t chunk;      // k per split (multiple of XKC); adjoint splits never cross a coil
    int sub;            // splits per coil (Gram residual: splits)
    float4* part;       // [splits][F][N] double-float partials, or null (one split, no coil maps)
    double2* B;         // output [F][N] when part is null
    const uint8_t* Gd;  // Gram residual: digit tiles of G ([row block][k block][digit] x 8 KiB)
    const int* eG;      // Gram residual: |G| <= 2^eG
    int64_t KB;         // k blocks of 16 per row block (per coil for the adjoint)
    const uint8_t* Bd;  // digit tiles of the B operand (k_b_digits)
    int C;              // coils (Gram residual: 1)
};

// conj(A[m][n]) for 8 consecutive samples m (< mend) of voxel n, double-float,
// from the sample-contiguous tables (rows of Mkp, m a multiple of 8)
__device__ inline void gen_ah8(const EncodeDev& e, int64_t n, int64_t m, int64_t mend, float (&reh)[8],
                               float (&rel)[8], float (&imh)[8], float (&iml)[8]) {
    float4 v[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) v[t] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (e.b0df) {  // A with its B0 factor, element by element from the double-float tables
#pragma unroll
        for (int t = 0; t < 8; ++t)
            if (n < e.N && m + t < mend) v[t] = gen_a_df(e, m + t, n);
    } else if (n < e.N && m < mend) {  // m is a multiple of 8 below M_k, so m + 7 < Mkp
        const int* g = e.vox_ijk + 3 * n;
        const float4* px = e.extdf + (int64_t)g[0] * e.Mkp + m;
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = px[t];
        if (e.ny > 1) {
            const float4* py = e.eytdf + (int64_t)g[1] * e.Mkp + m;
#pragma unroll
            for (int t = 0; t < 8; ++t) v[t] = cdf_mul(v[t], py[t]);
        }
        if (e.nz > 1) {
            const float4* pz = e.eztdf + (int64_t)g[2] * e.Mkp + m;
#pragma unroll
            for (int t = 0; t < 8; ++t) v[t] = cdf_mul(v[t], pz[t]);
        }
    }
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const bool in = n < e.N && m + t < mend;
        reh[t] = in ? v[t].x : 0.f;
        rel[t] = in ? v[t].y : 0.f;
        imh[t] = in ? -v[t].z : 0.f;  // conjugate
        iml[t] = in ? -v[t].w : 0.f;
    }
}

// A operand of the exact kernel
enum XMode { XGEN = 0, XGRAM = 1, XADJT = 2, XFWD = 3 };

// Digits of conj(A) for one (voxel tile, 16-sample chunk): NDIG slices of 8 KiB in
// the stage layout, exactly as the XGEN producers write them to shared memory.
__global__ void __launch_bounds__(256) k_adj_digits(EncodeDev e, int64_t KB, uint8_t* Ad) {
    const int64_t kb = blockIdx.x, rb = blockIdx.y;
    const int ra = threadIdx.x & (XM - 1), ga = threadIdx.x >> 7;
    float reh[8], rel[8], imh[8], iml[8];
    gen_ah8(e, rb * XM + ra, kb * XKC + 8 * ga, e.Mk, reh, rel, imh, iml);
    Digits8 dr, di;
    dr.init(reh, rel, 1.f);
    di.init(imh, iml, 1.f);
    uint8_t* blk = Ad + (rb * KB + kb) * (int64_t)(NDIG * XA_SL);
#pragma unroll
    for (int dg = 0; dg < NDIG; ++dg) {
        uint32_t w[4];
        dr.next(w, 0u);
        *reinterpret_cast<uint4*>(blk + dg * XA_SL + koff(ra, ga)) = make_uint4(w[0], w[1], w[2], w[3]);
        di.next(w, 0u);
        *reinterpret_cast<uint4*>(blk + dg * XA_SL + koff(ra, ga + 2)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Digits of A itself for one (128-sample tile, 16-voxel chunk), the A operand of
// the forward product: row r = sample rb * 128 + r, k = voxels kb * 16 .. + 15.
__global__ void __launch_bounds__(256) k_fwd_digits(EncodeDev e, int64_t KB, uint8_t* Af) {
    const int64_t kb = blockIdx.x, rb = blockIdx.y;
    const int ra = threadIdx.x & (XM - 1), ga = threadIdx.x >> 7;
    const int64_t m = rb * XM + ra, n0 = kb * XKC + 8 * ga;
    float reh[8], rel[8], imh[8], iml[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (m < e.Mk && n0 + t < e.N) v = gen_a_df(e, m, n0 + t);
        reh[t] = v.x;
        rel[t] = v.y;
        imh[t] = v.z;
        iml[t] = v.w;
    }
    Digits8 dr, di;
    dr.init(reh, rel, 1.f);
    di.init(imh, iml, 1.f);
    uint8_t* blk = Af + (rb * KB + kb) * (int64_t)(NDIG * XA_SL);
#pragma unroll
    for (int dg = 0; dg < NDIG; ++dg) {
        uint32_t w[4];
        dr.next(w, 0u);
        *reinterpret_cast<uint4*>(blk + dg * XA_SL + koff(ra, ga)) = make_uint4(w[0], w[1], w[2], w[3]);
        di.next(w, 0u);
        *reinterpret_cast<uint4*>(blk + dg * XA_SL + koff(ra, ga + 2)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// Y[f][c][n] = s_c(n) x[f][n] in double-float (FP64 in and out), the forward
// product's B operand before its digits
__global__ void k_coil_times(EncodeDev e, const double2* X, int64_t F, double2* Y) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= F * e.C * e.N) return;
    const int64_t n = idx % e.N, fc = idx / e.N;
    const int c = (int)(fc % e.C);
    const int64_t f = fc / e.C;
    float4 v = to_df_i(X[f * e.N + n]);
    if (e.coilsdf) v = cdf_mul(v, e.coilsdf[(int64_t)c * e.N + n]);
    Y[idx] = from_df(v);
}

// Digits of the B operand (data d, or x for the Gram residual) for one (XNT-frame
// tile, coil, 16-sample chunk): NDIG slices of B_SL bytes in the stage layout.
// Frame f of the tile owns row f, [Br | -Bi], and row XNT + f, [Bi | Br], each value
// scaled by 2^-fexp[f]; samples at or past Kc (the coil's end) and frames at or past
// F are zero. Value (f, c, m) is D[f * ld + c * Kc + m]. 256 / (2 XNT) chunks per
// 256-thread block, one (frame, 8 samples) unit per thread.
template <int XNT>
__global__ void __launch_bounds__(256) k_b_digits(const double2* D, int64_t ld, int64_t F, int C, int64_t Kc,
                                                  int64_t KB, const int* fexp, uint8_t* Bd) {
    constexpr int TPT = 2 * XNT;  // threads per chunk
    const int64_t FT = (F + XNT - 1) / XNT;
    const int64_t tile = (int64_t)blockIdx.x * (256 / TPT) + threadIdx.x / TPT;
    if (tile >= FT * C * KB) return;
    const int64_t kb = tile % KB, fc = tile / KB;
    const int c = (int)(fc % C);
    const int cb = (int)(threadIdx.x % XNT), gb = (int)((threadIdx.x / XNT) & 1);
    const int64_t f = (fc / C) * XNT + cb;
    const int64_t mk0 = kb * XKC + 8 * gb;
    float reh[8], rel[8], imh[8], iml[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        const int64_t m = mk0 + t;
        const float4 v = to_df_i((f < F && m < Kc) ? D[f * ld + (int64_t)c * Kc + m] : make_double2(0.0, 0.0));
        reh[t] = v.x;
        rel[t] = v.y;
        imh[t] = v.z;
        iml[t] = v.w;
    }
    const float scale = f < F ? __int_as_float((127 - fexp[f]) << 23) : 1.f;
    Digits8 dr, di;
    dr.init(reh, rel, scale);
    di.init(imh, iml, scale);
    uint8_t* bb = Bd + tile * (int64_t)(NDIG * XS<XNT>::B_SL);
#pragma unroll
    for (int dg = 0; dg < NDIG; ++dg) {
        uint32_t wr[4], wi[4];
        dr.next(wr, 0u);
        di.next(wi, 0u);
        uint8_t* sl = bb + dg * XS<XNT>::B_SL;
        *reinterpret_cast<uint4*>(sl + koff(cb, gb)) = make_uint4(wr[0], wr[1], wr[2], wr[3]);  // [Br|-Bi]
        *reinterpret_cast<uint4*>(sl + koff(cb, gb + 2)) =
            make_uint4(wi[0] ^ 0x80008000u, wi[1] ^ 0x80008000u, wi[2] ^ 0x80008000u, wi[3] ^ 0x80008000u);
        *reinterpret_cast<uint4*>(sl + koff(XNT + cb, gb)) = make_uint4(wi[0], wi[1], wi[2], wi[3]);  // [Bi|Br]
        *reinterpret_cast<uint4*>(sl + koff(XNT + cb, gb + 2)) = make_uint4(wr[0], wr[1], wr[2], wr[3]);
    }
}

// XGEN / XADJT: b = E^H d; XGRAM: G x with the digits of G in tile layout and x as
// the B operand. The B operand's digit tiles (k_b_digits) are copied per stage.
//
// One-dimensional grid, frame tile fastest, then coil, row block and split: the
// CTAs that read one A tile (all frame tiles and coils of a row block and split)
// run side by side and share it in L2.
template <int MODE, int XNT>
__global__ void __launch_bounds__(NTHREADS, 1) k_exact(XArgs a, DevStatus* st) {
    constexpr bool GRAM = MODE == XGRAM;
    constexpr bool FWD = MODE == XFWD;
    constexpr int B_SL = XS<XNT>::B_SL, XSTAGE = XS<XNT>::STAGE;
    constexpr int FPT = XNT / 2;  // frames per drain thread (two halves of the tile)
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t full_bar[XSTAGES], empty_bar[XSTAGES];
    __shared__ uint64_t abar[XSTAGES];  // the stage's bulk copies (their bytes)
    __shared__ uint64_t tfull, tempty, done_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_flag;
    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long wlim = st->wait_limit > 0 ? st->wait_limit : WAIT_LIMIT;  // pipeline waits
    // output rows (voxels; samples of one coil for the forward product)
    const int64_t N = FWD ? a.e.Mk : a.e.N;
    const int64_t FT = (a.F + XNT - 1) / XNT, RB = (N + XM - 1) / XM;
    int64_t lin = blockIdx.x;
    const int64_t ft = lin % FT;
    lin /= FT;
    const int coil = (int)(lin % a.C);
    lin /= a.C;
    const int64_t rb = lin % RB;
    const int split = (int)(lin / RB);
    const int64_t zpart = (int64_t)coil * a.sub + split;  // partial slot
    const int64_t n0 = rb * XM, f0 = ft * XNT;
    // k range [mb, me): adjoint samples inside coil `coil`, Gram columns, or the
    // voxels of the forward product
    const int64_t Mk = GRAM ? N : (FWD ? a.e.N : a.e.Mk);
    const int64_t mb = (int64_t)split * a.chunk;
    const int64_t me = mb + a.chunk < Mk ? mb + a.chunk : Mk;
    const int nk = me > mb ? (int)((me - mb + XKC - 1) / XKC) : 0;
    const int ngroups = (nk + XDRAIN - 1) / XDRAIN;

    if (threadIdx.x == 0) {
        for (int s = 0; s < XSTAGES; ++s) {
            mbar_init(&full_bar[s], NPW * 32);
            mbar_init(&empty_bar[s], 1);
            mbar_init(&abar[s], 1);
        }
        mbar_init(&tfull, 1);
        mbar_init(&tempty, NPW * 32);
        mbar_init(&done_bar, 1);
        abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == NPW) tmem_alloc(&tmem_base_sh, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;

    if (warp < NPW) {
        // ---------------- producers, drains, epilogue
        const int q = warp & 3, h = warp >> 2;  // TMEM lane quarter, half of the tile's frames
        const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16);
        float acc[4][FPT];  // re.hi, re.lo, im.hi, im.lo for this thread's FPT frames
#pragma unroll
        for (int u = 0; u < FPT; ++u) acc[0][u] = acc[1][u] = acc[2][u] = acc[3][u] = 0.f;
        bool ok = true;
        int drained = 0;
        auto drain = [&](int g) -> bool {
            if (!mbar_wait(&tfull, (uint32_t)g & 1u, &abort_flag, wlim)) return false;
            tc_fence_after();
#pragma unroll 1
            for (int w = 0; w < NCLS; ++w) {
                // region w: columns 2 XNT w .. (real parts of the tile's frames, then imaginary)
                uint32_t vr[FPT], vi[FPT];
                if constexpr (XNT == 32) {
                    tmem_ld16(trow + (uint32_t)(64 * w + 16 * h), vr);
                    tmem_ld16(trow + (uint32_t)(64 * w + XNT + 16 * h), vi);
                    tmem_wait_ld();
                } else {
                    static_assert(XNT == 8, "tile widths 32 and 8");
                    uint32_t v[16];
                    tmem_ld16(trow + (uint32_t)(16 * w), v);
                    tmem_wait_ld();
#pragma unroll
                    for (int u = 0; u < FPT; ++u) {  // constant indices: v stays in registers
                        vr[u] = h ? v[FPT + u] : v[u];
                        vi[u] = h ? v[XNT + FPT + u] : v[XNT + u];
                    }
                }
                const float sc = __int_as_float((127 - 12 - 7 * w) << 23);  // 2^(-12-7w)
#pragma unroll
                for (int u = 0; u < FPT; ++u) {
                    float s, e;
                    two_sum(acc[0][u], __uint_as_float(vr[u]) * sc, s, e);
                    acc[0][u] = s;
                    acc[1][u] += e;
                    two_sum(acc[2][u], __uint_as_float(vi[u]) * sc, s, e);
                    acc[2][u] = s;
                    acc[3][u] += e;
                }
            }
            tc_fence_before();
            mbar_arrive(&tempty);
            return true;
        };
        // A unit (XGEN): voxel row ua & 127, 8 samples of k-group ua >> 7
        const int ua = threadIdx.x, ra = ua & (XM - 1), ga = ua >> 7;
        const int64_t nrow = n0 + ra;
        int a_issued = 0;  // stages whose tiles this thread (thread 0) has started copying
        constexpr uint32_t kTx = (MODE != XGEN ? NDIG * XA_SL : 0) + NDIG * B_SL;
        const uint8_t* bsrc = a.Bd + ((ft * a.C + coil) * a.KB) * (int64_t)(NDIG * B_SL);
        for (int kt = 0; kt < nk && ok; ++kt) {
            const int s = kt % XSTAGES;
            const uint32_t ph = (uint32_t)(kt / XSTAGES) & 1u;
            if (kt >= XSTAGES && !(ok = mbar_wait(&empty_bar[s], ph ^ 1u, &abort_flag, wlim))) break;
            uint8_t* base = smem + s * XSTAGE;
            const int64_t m0 = mb + (int64_t)kt * XKC;  // k index (sample inside the coil, or Gram column)
            const int64_t kb = m0 / XKC;
            if (threadIdx.x == 0) {
                // the stage's digit tiles: A (NDIG x 8 KiB, unless formed below) and
                // B (NDIG x 4 KiB), counted in bytes on abar
                mbar_arrive_expect_tx(&abar[s], kTx);
                if (MODE != XGEN)
                    bulk_g2s(base, a.Gd + (rb * a.KB + kb) * (int64_t)(NDIG * XA_SL), (uint32_t)(NDIG * XA_SL),
                             &abar[s]);
                bulk_g2s(base + NDIG * XA_SL, bsrc + kb * (int64_t)(NDIG * B_SL), (uint32_t)(NDIG * B_SL),
                         &abar[s]);
                a_issued = kt + 1;
            }
            if constexpr (MODE == XGEN) {
                float reh[8], rel[8], imh[8], iml[8];
                gen_ah8(a.e, nrow, m0 + 8 * ga, me, reh, rel, imh, iml);
                Digits8 dr, di;
                dr.init(reh, rel, 1.f);
                di.init(imh, iml, 1.f);
#pragma unroll
                for (int dg = 0; dg < NDIG; ++dg) {
                    uint32_t w[4];
                    dr.next(w, 0u);
                    *reinterpret_cast<uint4*>(base + dg * XA_SL + koff(ra, ga)) = make_uint4(w[0], w[1], w[2], w[3]);
                    di.next(w, 0u);
                    *reinterpret_cast<uint4*>(base + dg * XA_SL + koff(ra, ga + 2)) =
                        make_uint4(w[0], w[1], w[2], w[3]);
                }
                fence_proxy_async();
                mbar_arrive(&full_bar[s]);
            }
            // a group is drained once the stages after it are in flight: its last
            // stage's slot came back at this stage's empty wait
            while (drained < ngroups && (drained + 1) * XDRAIN + XSTAGES - 1 <= kt) {
                if (!(ok = drain(drained))) break;
                ++drained;
            }
        }
        while (ok && drained < ngroups) {
            ok = drain(drained);
            ++drained;
        }
        if (ok && !abort_flag) {
            // this thread: voxel n0 + q*32 + lane, frames f0 + FPT h .. + FPT - 1
            const int64_t n = n0 + q * 32 + lane;
            if (n < N) {
                float4 cs = make_float4(1.f, 0.f, 0.f, 0.f);
                if (!GRAM && !FWD && a.e.coilsdf) cs = cdf_conj(a.e.coilsdf[(int64_t)coil * N + n]);
                const int eA = GRAM ? *a.eG : 0;
#pragma unroll
                for (int u = 0; u < FPT; ++u) {
                    const int64_t f = f0 + FPT * h + u;
                    if (f >= a.F) continue;
                    const float sc = __int_as_float((127 + eA + a.fexp[f]) << 23);
                    float4 v = make_float4(acc[0][u] * sc, acc[1][u] * sc, acc[2][u] * sc, acc[3][u] * sc);
                    if (!GRAM && !FWD && a.e.coilsdf) v = cdf_mul(v, cs);
                    if (a.part)
                        a.part[(zpart * a.F + f) * N + n] = v;
                    else
                        a.B[f * N + n] = from_df(v);
                }
            }
        }
        if (threadIdx.x == 0) {
            // copies still in flight (only after an abort): wait, bounded, for their bytes
            for (int kg = a_issued > XSTAGES ? a_issued - XSTAGES : 0; kg < a_issued; ++kg)
                mbar_wait(&abar[kg % XSTAGES], (uint32_t)(kg / XSTAGES) & 1u, nullptr);
        }
    } else if (lane == 0) {
        // ---------------- MMA issuer: 21 digit pairs per stage in 8 MMAs per k half,
        // class w = i + j into region w
        for (int kt = 0; kt < nk; ++kt) {
            const int g = kt / XDRAIN;
            const bool first = (kt % XDRAIN) == 0;
            if (first && g >= 1 && !mbar_wait(&tempty, (uint32_t)(g - 1) & 1u, &abort_flag, wlim)) break;
            const int s = kt % XSTAGES;
            const uint32_t ph = (uint32_t)(kt / XSTAGES) & 1u;
            if (MODE == XGEN && !mbar_wait(&full_bar[s], ph, &abort_flag, wlim)) break;
            if (!mbar_wait(&abar[s], ph, &abort_flag, wlim)) break;
            tc_fence_after();
            const uint32_t abase = smem_u32(smem + s * XSTAGE);
            const uint32_t bbase = abase + NDIG * XA_SL;
#pragma unroll
            for (int kk = 0; kk < 2; ++kk) {
#pragma unroll
                for (int r = 0; r < 8; ++r) {
                    // the runs of A digit 0 cover all six regions: they start each group
                    const XPairRun u = xrun(r);
                    const uint64_t da = sdesc(abase + u.i * XA_SL + kk * 256, 128, 512);
                    const uint64_t db = sdesc(bbase + u.j0 * B_SL + kk * 256, 128, 512);
                    mma_bf16(tmem + (uint32_t)(2 * XNT * (u.i + u.j0)), da, db, xidesc(2 * XNT * u.nd),
                             (first && u.i == 0 && kk == 0) ? 0u : 1u);
                }
            }
            mma_commit(&empty_bar[s]);
            if ((kt % XDRAIN) == XDRAIN - 1 || kt == nk - 1) mma_commit(&tfull);
        }
        mma_commit(&done_bar);
    }

    tc_fence_before();
    __syncthreads();
    if (warp == NPW) {
        mbar_wait(&done_bar, 0, nullptr);
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
    if (threadIdx.x == 0 && abort_flag) atomicMax(&st->timeout_site, 20);
}

// store functor for the ordered reduction of the partials
struct BStore {
    double2* B;
    int64_t N;
    __device__ void store(int64_t i, int64_t j, double2 v) const { B[j * N + i] = v; }
};

__global__ void k_exact_reduce(BStore o, const float4* part, int splits, int64_t rows, int64_t F) {
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
    o.store(i, j, from_df(a));
}

// r[f][n] = b[f][n] - sum_z part[z][f][n], partials added in order
__global__ void k_resid_reduce(const double2* b, const float4* part, int splits, int64_t N, int64_t F,
                               double2* r) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * F) return;
    float4 a = part[idx];
    for (int z = 1; z < splits; ++z) {
        const float4 c = part[(int64_t)z * N * F + idx];
        float rh, rl, ih, il;
        df_add(a.x, a.y, c.x, c.y, rh, rl);
        df_add(a.z, a.w, c.z, c.w, ih, il);
        a = make_float4(rh, rl, ih, il);
    }
    const double2 g = from_df(a), bb = b[idx];
    r[idx] = make_double2(bb.x - g.x, bb.y - g.y);
}

// u[f][c Mk + m] = d[f][c Mk + m] - sum_s part[c sub + s][f][m] (d may be null:
// u = -E x), the splits of each coil added in order
__global__ void k_fwd_reduce(const double2* d, const float4* part, int sub, int C, int64_t Mk, int64_t F,
                             double2* u) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t M = Mk * C;
    if (idx >= M * F) return;
    const int64_t f = idx / M, cm = idx % M;
    const int c = (int)(cm / Mk);
    const int64_t m = cm % Mk;
    float4 a = part[(((int64_t)c * sub) * F + f) * Mk + m];
    for (int z = 1; z < sub; ++z) {
        const float4 b = part[(((int64_t)c * sub + z) * F + f) * Mk + m];
        float rh, rl, ih, il;
        df_add(a.x, a.y, b.x, b.y, rh, rl);
        df_add(a.z, a.w, b.z, b.w, ih, il);
        a = make_float4(rh, rl, ih, il);
    }
    const double2 g = from_df(a);
    const double2 dd = d ? d[idx] : make_double2(0.0, 0.0);
    u[idx] = make_double2(dd.x - g.x, dd.y - g.y);
}

// r[i] -= lam * x[i] (FP64)
__global__ void k_minus_lam(double2* r, const double2* x, double lam, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) r[i] = make_double2(r[i].x - lam * x[i].x, r[i].y - lam * x[i].y);
}

// |G| <= 2^eG from the largest diagonal entry (G Hermitian positive definite)
__global__ void k_gram_exp(const float4* G, int64_t N, int* eG) {
    __shared__ double red[256];
    double m = 0.0;
    for (int64_t n = threadIdx.x; n < N; n += blockDim.x) {
        const float4 g = G[n * N + n];
        m = fmax(m, fabs((double)g.x + (double)g.y));
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        int ex = 0;
        const double mant = red[0] > 0.0 ? frexp(red[0], &ex) : 0.0;
        if (mant == 0.5) --ex;
        *eG = red[0] > 0.0 ? ex : 0;
    }
}

// Digit tiles of G: one thread per (row n, 8 columns); every position of the
// padded [RB * 128][KB * 16] array is written (zeros outside N x N).
__global__ void k_gram_digits(const float4* G, int64_t N, int64_t KB, const int* eG, uint8_t* Gd) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t RB = (N + XM - 1) / XM;
    if (idx >= RB * XM * KB * 2) return;
    const int64_t n = idx / (KB * 2), rem = idx % (KB * 2);
    const int64_t kb = rem / 2;
    const int g = (int)(rem % 2);
    const int64_t c0 = kb * XKC + 8 * g;
    float reh[8], rel[8], imh[8], iml[8];
#pragma unroll
    for (int t = 0; t < 8; ++t) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (n < N && c0 + t < N) v = G[n * N + c0 + t];
        reh[t] = v.x;
        rel[t] = v.y;
        imh[t] = v.z;
        iml[t] = v.w;
    }
    const float scale = __int_as_float((127 - *eG) << 23);
    Digits8 dr, di;
    dr.init(reh, rel, scale);
    di.init(imh, iml, scale);
    uint8_t* tile = Gd + ((n / XM) * KB + kb) * (int64_t)(NDIG * XA_SL);
    const int r = (int)(n % XM);
#pragma unroll
    for (int dg = 0; dg < NDIG; ++dg) {
        uint32_t w[4];
        dr.next(w, 0u);
        *reinterpret_cast<uint4*>(tile + dg * XA_SL + koff(r, g)) = make_uint4(w[0], w[1], w[2], w[3]);
        di.next(w, 0u);
        *reinterpret_cast<uint4*>(tile + dg * XA_SL + koff(r, g + 2)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
}

// per-frame exponent: |re|, |im| of frame f all <= 2^fexp[f]
// fexp[f] = the least e with max_j |D[f][j]| <= 2^e (0 for a zero frame). The
// maximum is taken over the bit patterns with the sign cleared, whose order is the
// order of the magnitudes (NaN and infinity left out), on the integer pipe.
__device__ inline unsigned long long mag_bits(double x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
    return (b >> 52) == 0x7ffull ? 0ull : b;
}
__global__ void __launch_bounds__(256) k_frame_exp(const double2* D, int64_t M, int* fexp) {
    __shared__ unsigned long long red[256];
    const int64_t f = blockIdx.x;
    unsigned long long m = 0ull;
    const double2* row = D + f * M;
    int64_t j = threadIdx.x;
    for (; j + 768 < M; j += 1024) {  // four loads in flight
        const double2 a = row[j], b = row[j + 256], c = row[j + 512], d = row[j + 768];
        m = max(m, max(max(mag_bits(a.x), mag_bits(a.y)), max(mag_bits(b.x), mag_bits(b.y))));
        m = max(m, max(max(mag_bits(c.x), mag_bits(c.y)), max(mag_bits(d.x), mag_bits(d.y))));
    }
    for (; j < M; j += 256) m = max(m, max(mag_bits(row[j].x), mag_bits(row[j].y)));
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] = max(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const unsigned long long B = red[0];
        const int eb = (int)(B >> 52);
        const unsigned long long mf = B & ((1ull << 52) - 1ull);
        int e = 0;
        if (B == 0ull)
            e = 0;
        else if (eb == 0)  // subnormal: B = mf 2^-1074
            e = (64 - __clzll((long long)mf)) - 1074 - ((mf & (mf - 1ull)) == 0ull ? 1 : 0);
        else  // (1 + mf 2^-52) 2^(eb - 1023): one more bit unless a power of two
            e = eb - 1023 + (mf != 0ull ? 1 : 0);
        fexp[f] = e;
    }
}

}  // namespace tcx

// frame-tile width of a call of F frames (the narrow tile for at most eight), and
// the number of frame tiles
static int exact_xn(int64_t F) { return F <= tcx::XNN ? tcx::XNN : tcx::XN; }
static int64_t exact_ft(int64_t F) { return (F + exact_xn(F) - 1) / exact_xn(F); }

template <int MODE, int XNT>
static cudaError_t exact_attr() {
    static bool attr = false;
    if (attr) return cudaSuccess;
    cudaError_t err = cudaFuncSetAttribute(tcx::k_exact<MODE, XNT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           tcx::XS<XNT>::SMEM);
    if (err == cudaSuccess) attr = true;
    return err;
}
// the exact kernel for a call of F frames, `grid` CTAs
template <int MODE>
static cudaError_t launch_exact(const tcx::XArgs& a, int64_t F, unsigned grid, DevStatus* st, cudaStream_t s) {
    cudaError_t err;
    if (exact_xn(F) == tcx::XNN) {
        if ((err = exact_attr<MODE, tcx::XNN>()) != cudaSuccess) return err;
        tcx::k_exact<MODE, tcx::XNN><<<grid, tc::NTHREADS, tcx::XS<tcx::XNN>::SMEM, s>>>(a, st);
    } else {
        if ((err = exact_attr<MODE, tcx::XN>()) != cudaSuccess) return err;
        tcx::k_exact<MODE, tcx::XN><<<grid, tc::NTHREADS, tcx::XS<tcx::XN>::SMEM, s>>>(a, st);
    }
    note_launch();
    return cudaGetLastError();
}

// splits per coil: whole waves of CTAs over all coils, chunks of at least two
// accumulation groups
static int exact_sub(const EncodeDev& e, int64_t F) {
    const int64_t tiles = ((e.N + tcx::XM - 1) / tcx::XM) * exact_ft(F) * e.C;
    const int hi = (int)std::max<int64_t>(1, std::min<int64_t>(32, e.Mk / (tcx::XKC * tcx::XDRAIN * 2)));
    return tc::wave_splits(tiles, e.Mk, 1, hi, 256);
}

size_t exact_work_elems(const EncodeDev& e, int64_t F) {
    const int64_t splits = (int64_t)exact_sub(e, F) * e.C;
    return splits > 1 || e.coilsdf ? (size_t)splits * (size_t)e.N * (size_t)F : 0;
}

// digit tiles of the B operand: frame tiles x coils x 16-sample chunks per coil
static size_t b_digit_bytes(int64_t F, int64_t C, int64_t Kc) {
    return (size_t)exact_ft(F) * (size_t)C * (size_t)((Kc + tcx::XKC - 1) / tcx::XKC) *
           (size_t)(tcx::NDIG * 2 * exact_xn(F) * 64);
}

static cudaError_t launch_b_digits(const double2* D, int64_t ld, int64_t F, int C, int64_t Kc, const int* fexp,
                                   uint8_t* Bd, cudaStream_t s) {
    const int64_t KB = (Kc + tcx::XKC - 1) / tcx::XKC;
    const int64_t tiles = exact_ft(F) * C * KB;
    const int64_t per = 256 / (2 * exact_xn(F));  // chunks per block
    if (exact_xn(F) == tcx::XNN)
        tcx::k_b_digits<tcx::XNN><<<(unsigned)((tiles + per - 1) / per), 256, 0, s>>>(D, ld, F, C, Kc, KB, fexp, Bd);
    else
        tcx::k_b_digits<tcx::XN><<<(unsigned)((tiles + per - 1) / per), 256, 0, s>>>(D, ld, F, C, Kc, KB, fexp, Bd);
    note_launch();
    return cudaGetLastError();
}

size_t exact_bdigit_bytes(const EncodeDev& e, int64_t F) { return b_digit_bytes(F, e.C, e.Mk); }

// the fewest frames for which the exact products replace the double-float ones:
// every count since calls of up to eight frames take the 8-frame tile (a 64x64
// apply of 1-12 frames: 11.5-14 ms with the double-float products, 1.8-2.1 ms with
// these and the tensor-core correction). PINV_EXACT_MIN_FRAMES: another count.
static int64_t exact_min_frames() {
    static const int64_t v = [] {
        const char* s = std::getenv("PINV_EXACT_MIN_FRAMES");
        return s ? std::max<int64_t>(1, std::atoll(s)) : (int64_t)1;
    }();
    return v;
}

bool exact_adjoint_ok(const EncodeDev& e, int64_t F, bool table) {
    // plans with B0 only from the per-build table of conj(A) (the producers form
    // A from the separable tables of plans without B0)
    const bool gen = e.extdf && !e.b0df && !e.b0tab;
    const bool tab = table && e.b0df && e.exdf;
    return (gen || tab) && F >= exact_min_frames() && tc_available();
}

size_t adj_digit_bytes(const EncodeDev& e) {
    const int64_t RB = (e.N + tcx::XM - 1) / tcx::XM, KB = (e.Mk + tcx::XKC - 1) / tcx::XKC;
    return (size_t)RB * (size_t)KB * (size_t)(tcx::NDIG * tcx::XA_SL);
}

cudaError_t launch_adj_digits(const EncodeDev& e, uint8_t* Ad, cudaStream_t s) {
    const int64_t RB = (e.N + tcx::XM - 1) / tcx::XM, KB = (e.Mk + tcx::XKC - 1) / tcx::XKC;
    tcx::k_adj_digits<<<dim3((unsigned)KB, (unsigned)RB), 256, 0, s>>>(e, KB, Ad);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_adjoint_exact(const EncodeDev& e, const double2* D, int64_t F, int* fexp, uint8_t* Bd,
                                 double2* B, float4* work, DevStatus* st, cudaStream_t s, const uint8_t* Ad) {
    if (F == 0) return cudaSuccess;
    if (!Bd) return cudaErrorInvalidValue;
    const int64_t M = e.Mk * e.C;
    tcx::k_frame_exp<<<(unsigned)F, 256, 0, s>>>(D, M, fexp);
    note_launch();
    cudaError_t berr = launch_b_digits(D, M, F, (int)e.C, e.Mk, fexp, Bd, s);
    if (berr != cudaSuccess) return berr;
    const int sub = exact_sub(e, F);
    const int64_t splits = (int64_t)sub * e.C;
    const bool partials = splits > 1 || e.coilsdf;
    if (partials && !work) return cudaErrorInvalidValue;
    const int64_t chunk = ((e.Mk + sub - 1) / sub + tcx::XKC - 1) / tcx::XKC * tcx::XKC;
    const int64_t KB = (e.Mk + tcx::XKC - 1) / tcx::XKC;
    tcx::XArgs a{e, D, fexp, F, M, chunk, sub, partials ? work : nullptr, B, Ad, nullptr, KB, Bd, (int)e.C};
    const unsigned grid = (unsigned)(exact_ft(F) * ((e.N + tcx::XM - 1) / tcx::XM) * splits);
    cudaError_t err = Ad ? launch_exact<tcx::XADJT>(a, F, grid, st, s) : launch_exact<tcx::XGEN>(a, F, grid, st, s);
    if (err != cudaSuccess || !partials) return err;
    const int64_t n = e.N * F;
    tcx::k_exact_reduce<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(tcx::BStore{B, e.N}, work, (int)splits, e.N, F);
    note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------ exact forward product
// splits of the voxel range per coil: whole waves of CTAs over all coils
static int fwd_sub(const EncodeDev& e, int64_t F) {
    const int64_t tiles = ((e.Mk + tcx::XM - 1) / tcx::XM) * exact_ft(F) * e.C;
    const int hi = (int)std::max<int64_t>(1, std::min<int64_t>(32, e.N / (tcx::XKC * tcx::XDRAIN * 2)));
    return tc::wave_splits(tiles, e.N, 1, hi, 256);
}

size_t fwd_digit_bytes(const EncodeDev& e) {
    const int64_t RB = (e.Mk + tcx::XM - 1) / tcx::XM, KB = (e.N + tcx::XKC - 1) / tcx::XKC;
    return (size_t)RB * (size_t)KB * (size_t)(tcx::NDIG * tcx::XA_SL);
}

cudaError_t launch_fwd_digits(const EncodeDev& e, uint8_t* Af, cudaStream_t s) {
    const int64_t RB = (e.Mk + tcx::XM - 1) / tcx::XM, KB = (e.N + tcx::XKC - 1) / tcx::XKC;
    tcx::k_fwd_digits<<<dim3((unsigned)KB, (unsigned)RB), 256, 0, s>>>(e, KB, Af);
    note_launch();
    return cudaGetLastError();
}

size_t exact_fwd_work_elems(const EncodeDev& e, int64_t F) {
    return (size_t)fwd_sub(e, F) * (size_t)e.C * (size_t)F * (size_t)e.Mk;
}
size_t exact_fwd_bdigit_bytes(const EncodeDev& e, int64_t F) { return b_digit_bytes(F, e.C, e.N); }
size_t exact_fwd_y_elems(const EncodeDev& e, int64_t F) { return (size_t)F * (size_t)e.C * (size_t)e.N; }

cudaError_t launch_forward_exact(const EncodeDev& e, const double2* X, int64_t F, const double2* D, double2* U,
                                 const uint8_t* Af, double2* Y, int* fexp, uint8_t* Bd, float4* work,
                                 DevStatus* st, cudaStream_t s) {
    if (F == 0) return cudaSuccess;
    if (!Af || !Y || !Bd || !work) return cudaErrorInvalidValue;
    cudaError_t err;
    const int64_t ny = F * e.C * e.N;
    tcx::k_coil_times<<<(unsigned)((ny + 255) / 256), 256, 0, s>>>(e, X, F, Y);  // Y[f][c] = s_c o x_f
    tcx::k_frame_exp<<<(unsigned)F, 256, 0, s>>>(Y, e.C * e.N, fexp);
    note_launch(2);
    if ((err = launch_b_digits(Y, e.C * e.N, F, (int)e.C, e.N, fexp, Bd, s)) != cudaSuccess) return err;
    const int sub = fwd_sub(e, F);
    const int64_t chunk = ((e.N + sub - 1) / sub + tcx::XKC - 1) / tcx::XKC * tcx::XKC;
    const int64_t KB = (e.N + tcx::XKC - 1) / tcx::XKC;
    tcx::XArgs a{e, Y, fexp, F, e.C * e.N, chunk, sub, work, nullptr, Af, nullptr, KB, Bd, (int)e.C};
    const unsigned grid = (unsigned)(exact_ft(F) * ((e.Mk + tcx::XM - 1) / tcx::XM) * e.C * sub);
    if ((err = launch_exact<tcx::XFWD>(a, F, grid, st, s)) != cudaSuccess) return err;
    const int64_t n = e.Mk * e.C * F;
    tcx::k_fwd_reduce<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(D, work, sub, (int)e.C, e.Mk, F, U);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_minus_lambda(double2* R, const double2* X, double lam, int64_t n, cudaStream_t s) {
    tcx::k_minus_lam<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(R, X, lam, n);
    note_launch();
    return cudaGetLastError();
}

// ------------------------------------------------------------------ exact Gram residual
size_t gram_digit_bytes(int64_t N) {
    const int64_t RB = (N + tcx::XM - 1) / tcx::XM, KB = (N + tcx::XKC - 1) / tcx::XKC;
    return (size_t)RB * (size_t)KB * (size_t)(tcx::NDIG * tcx::XA_SL);
}

cudaError_t launch_gram_digits(const float4* G, int64_t N, int* eG, uint8_t* Gd, cudaStream_t s) {
    tcx::k_gram_exp<<<1, 256, 0, s>>>(G, N, eG);
    note_launch();
    const int64_t KB = (N + tcx::XKC - 1) / tcx::XKC, RB = (N + tcx::XM - 1) / tcx::XM;
    const int64_t n = RB * tcx::XM * KB * 2;
    tcx::k_gram_digits<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(G, N, KB, eG, Gd);
    note_launch();
    return cudaGetLastError();
}

static int resid_splits(int64_t N, int64_t F) {
    const int64_t tiles = ((N + tcx::XM - 1) / tcx::XM) * exact_ft(F);
    const int hi = (int)std::max<int64_t>(1, std::min<int64_t>(32, N / (tcx::XKC * tcx::XDRAIN * 2)));
    return tc::wave_splits(tiles, N, 1, hi, 256);
}

size_t resid_exact_work_elems(int64_t N, int64_t F) { return (size_t)resid_splits(N, F) * (size_t)N * (size_t)F; }

size_t resid_bdigit_bytes(int64_t N, int64_t F) { return b_digit_bytes(F, 1, N); }

cudaError_t launch_gram_resid_exact(const uint8_t* Gd, const int* eG, int64_t N, const double2* Bv,
                                    const double2* X, int64_t F, int* fexp, uint8_t* Bd, double2* R,
                                    float4* work, DevStatus* st, cudaStream_t s) {
    if (F == 0) return cudaSuccess;
    if (!Bd) return cudaErrorInvalidValue;
    cudaError_t err;
    tcx::k_frame_exp<<<(unsigned)F, 256, 0, s>>>(X, N, fexp);
    note_launch();
    if ((err = launch_b_digits(X, N, F, 1, N, fexp, Bd, s)) != cudaSuccess) return err;
    const int sp = resid_splits(N, F);
    const int64_t chunk = ((N + sp - 1) / sp + tcx::XKC - 1) / tcx::XKC * tcx::XKC;
    EncodeDev e{};
    e.N = N;
    const int64_t KB = (N + tcx::XKC - 1) / tcx::XKC;
    tcx::XArgs a{e, X, fexp, F, N, chunk, sp, work, nullptr, Gd, eG, KB, Bd, 1};
    const unsigned grid = (unsigned)(exact_ft(F) * ((N + tcx::XM - 1) / tcx::XM) * sp);
    if ((err = launch_exact<tcx::XGRAM>(a, F, grid, st, s)) != cudaSuccess) return err;
    const int64_t n = N * F;
    tcx::k_resid_reduce<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(Bv, work, sp, N, F, R);
    note_launch();
    return cudaGetLastError();
}

}  // namespace pinv
