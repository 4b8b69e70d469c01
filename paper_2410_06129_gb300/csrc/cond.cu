// Condition estimate of the Gram matrix (Section 2.1: the condition number
// measures how the inversion amplifies errors; Section 2.2: the Tikhonov load
// lambda makes G = E^H E + lambda I positive definite, every eigenvalue at
// least lambda).
//
// kappa_1(G) = ||G||_1 ||G^-1||_1.
//   ||G||_1 (= ||G||_inf for Hermitian G) is the largest column sum of |G|. It is
//   read from G before the Cholesky overwrites it, or from the exact Gram where
//   the plan forms one.
//   ||G^-1||_1 is estimated by Hager's method in Higham's complex form. Start
//   from x = (1/N, ..., 1/N); then y = G^-1 x, xi = y / |y| elementwise,
//   z = G^-1 xi (G^-1 is Hermitian), x = e_j at the largest |z_j|; repeat while
//   the estimate grows and the index changes (at most five rounds), and try one
//   more vector of alternating signs with growing magnitude. Each value
//   ||G^-1 v||_1 / ||v||_1 is a lower bound of ||G^-1||_1.
//
// The solves use the plan's factor: the FP64 G^-1 of FP64 plans, or W^H W with
// the FP32 W = L^-1 of mixed plans. A mixed factor is off by up to kappa(G)
// times the split rounding, so for mixed plans the two final candidates y are
// refined once (y += W^H W (v - G y)) and then certified against G itself:
// ||y||_1 / ||G y||_1 <= ||G^-1||_1 holds for every y, and G y is formed by the
// plan's refinement residual operator (the exact tensor-core Gram, or
// E^H E y + lambda y generated in double-float or FP64). The estimate therefore
// stays below kappa_1(G) up to the rounding of the sums.
//
// Everything runs on the device with no host synchronisation: single-block
// kernels keep the iteration's state in device memory, and once it has
// converged the remaining kernels of the fixed launch sequence return at once.
#include <algorithm>
#include <cmath>
#include <string>
#include <type_traits>
#include <vector>

#include "df.cuh"
#include "plan_impl.h"

namespace pinv {
namespace {

constexpr int CB = 1024;       // threads of the single-block kernels
constexpr int HAGER_ROUNDS = 5;

pinv_status cuda_err(cudaError_t e, const char* where) {
    return set_error(e == cudaErrorMemoryAllocation ? PINV_ERR_OOM : PINV_ERR_CUDA,
                     std::string(where) + ": " + cudaGetErrorString(e));
}
#define CKC(call)                                              \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_err(e_, #call);     \
    } while (0)

struct HagerState {
    double est;       // best ||G^-1 v||_1 / ||v||_1 so far (v = the start vector or some e_j)
    double est_alt;   // the same for the alternating-sign vector
    int j, jlast;     // current and previous unit-vector index
    int done;         // the iteration has finished
    int rounds;       // unit-vector rounds taken
    int best_j;       // start vector of the best estimate: -1 = uniform, else e_best_j
};

// |a + ib| in FP32 from FP64 parts, without the FP64 pipe
__device__ inline float abs_f(double2 g) {
    const float x = f64_to_f32_rn(g.x), y = f64_to_f32_rn(g.y);
    return sqrtf(fmaf(x, x, y * y));
}

// double-float sum of a warp's (hi, lo) pairs, result in every lane
__device__ inline float2 warp_sum_df(float h, float l) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oh = __shfl_xor_sync(0xffffffffu, h, o), ol = __shfl_xor_sync(0xffffffffu, l, o);
        df_add(h, l, oh, ol, h, l);
    }
    return make_float2(h, l);
}
__device__ inline void acc_df(float& h, float& l, float v) { df_add(h, l, v, 0.f, h, l); }

// -------------------------------------------------------------------- ||G||_1
// rs[i] = sum_{j <= i} |G[i][j]| over the stored lower triangle (full = false),
// or sum_j |G[i][j]| over the whole row (full = true); one warp per row
template <class T, bool FULL>
__global__ void k_abs_rows(const T* G, int64_t N, int64_t ld, float2* rs) {
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= N) return;
    const T* row = G + i * ld;
    const int64_t end = FULL ? N : i + 1;
    float h = 0.f, l = 0.f;
    for (int64_t j = lane; j < end; j += 32) {
        float a;
        if constexpr (std::is_same<T, float4>::value) {
            const float4 g = reinterpret_cast<const float4*>(row)[j];  // double-float: |hi| suffices
            a = sqrtf(fmaf(g.x, g.x, g.z * g.z));
        } else {
            a = abs_f(row[j]);
        }
        acc_df(h, l, a);
    }
    const float2 s = warp_sum_df(h, l);
    if (lane == 0) rs[i] = s;
}

// part[s][j] = sum over rows i of chunk s with i > j of |G[i][j]| (the strictly
// lower part of column j); consecutive threads read consecutive columns. G in
// FP64 (double2) or double-float (float4, |hi| suffices) storage.
template <class T>
__global__ void k_abs_cols_lower(const T* G, int64_t N, int64_t ld, int64_t rows_per_chunk, float2* part) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.y * rows_per_chunk;
    const int64_t i1 = N < i0 + rows_per_chunk ? N : i0 + rows_per_chunk;
    if (j >= N) return;
    float h = 0.f, l = 0.f;
    for (int64_t i = i0 > j + 1 ? i0 : j + 1; i < i1; ++i) {
        if constexpr (std::is_same<T, float4>::value) {
            const float4 g = G[i * ld + j];
            acc_df(h, l, sqrtf(fmaf(g.x, g.x, g.z * g.z)));
        } else {
            acc_df(h, l, abs_f(G[i * ld + j]));
        }
    }
    part[(int64_t)blockIdx.y * N + j] = make_float2(h, l);
}

// out = max_j (rs[j] + sum_s part[s][j])
__global__ void __launch_bounds__(CB) k_norm1_finish(const float2* rs, const float2* part, int chunks, int64_t N,
                                                     double* out) {
    __shared__ double red[CB];
    double m = 0.0;
    for (int64_t j = threadIdx.x; j < N; j += CB) {
        float h = rs[j].x, l = rs[j].y;
        for (int s = 0; s < chunks; ++s) {
            const float2 p = part[(int64_t)s * N + j];
            df_add(h, l, p.x, p.y, h, l);
        }
        m = fmax(m, (double)h + (double)l);
    }
    red[threadIdx.x] = m;
    __syncthreads();
    for (int w = CB / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// -------------------------------------------------------------------- solves
// Products with the FP32 W = L^-1 for F <= 2 vectors at once, FP32 arithmetic
// (the search only needs the estimate's order; the final candidates are refined
// and certified against G).
constexpr int FMAX = 2;

// u[f] = W x[f], W lower FP32 [N][N] row-major; one warp per row
__global__ void k_w_mv(const float2* W, int64_t N, int F, const float2* x, float2* u, const int* skip) {
    if (skip && *skip) return;
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= N) return;
    const float2* row = W + i * N;
    float re[FMAX] = {0.f, 0.f}, im[FMAX] = {0.f, 0.f};
    auto mac = [&](float2 w, int64_t j) {
#pragma unroll
        for (int f = 0; f < FMAX; ++f) {
            if (f < F) {
                const float2 v = x[(int64_t)f * N + j];
                re[f] = fmaf(w.x, v.x, fmaf(-w.y, v.y, re[f]));
                im[f] = fmaf(w.x, v.y, fmaf(w.y, v.x, im[f]));
            }
        }
    };
    if ((N & 1) == 0) {  // rows start on 16-byte boundaries: two entries per load
        const float4* row4 = reinterpret_cast<const float4*>(row);
#pragma unroll 4
        for (int64_t q = lane; 2 * q <= i; q += 32) {
            const float4 w = row4[q];
            mac(make_float2(w.x, w.y), 2 * q);
            if (2 * q + 1 <= i) mac(make_float2(w.z, w.w), 2 * q + 1);
        }
    } else {
#pragma unroll 4
        for (int64_t j = lane; j <= i; j += 32) mac(row[j], j);
    }
#pragma unroll
    for (int f = 0; f < FMAX; ++f) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            re[f] += __shfl_xor_sync(0xffffffffu, re[f], o);
            im[f] += __shfl_xor_sync(0xffffffffu, im[f], o);
        }
        if (lane == 0 && f < F) u[(int64_t)f * N + i] = make_float2(re[f], im[f]);
    }
}

// part[s][f][j] = sum over rows i of chunk s with i >= j of conj(W[i][j]) u[f][i]
__global__ void k_wh_part(const float2* W, int64_t N, int F, const float2* u, int64_t rows_per_chunk, float2* part,
                          const int* skip) {
    if (skip && *skip) return;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t i0 = (int64_t)blockIdx.y * rows_per_chunk;
    const int64_t i1 = N < i0 + rows_per_chunk ? N : i0 + rows_per_chunk;
    if (j >= N) return;
    float re[FMAX] = {0.f, 0.f}, im[FMAX] = {0.f, 0.f};
#pragma unroll 4
    for (int64_t i = i0 > j ? i0 : j; i < i1; ++i) {
        const float2 w = W[i * N + j];
#pragma unroll
        for (int f = 0; f < FMAX; ++f) {
            if (f < F) {
                const float2 v = u[(int64_t)f * N + i];
                re[f] = fmaf(w.x, v.x, fmaf(w.y, v.y, re[f]));
                im[f] = fmaf(w.x, v.y, fmaf(-w.y, v.x, im[f]));
            }
        }
    }
    for (int f = 0; f < F; ++f) part[((int64_t)blockIdx.y * F + f) * N + j] = make_float2(re[f], im[f]);
}

// y[f][j] (+)= sum_s part[s][f][j]
__global__ void k_part_sum(const float2* part, int chunks, int64_t N, int F, double2* y, int accumulate,
                           const int* skip) {
    if (skip && *skip) return;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * F) return;
    float re = 0.f, im = 0.f;
    for (int s = 0; s < chunks; ++s) {
        const float2 p = part[(int64_t)s * N * F + idx];
        re += p.x;
        im += p.y;
    }
    double2 v = make_double2((double)re, (double)im);
    if (accumulate) v = zadd(y[idx], v);
    y[idx] = v;
}

// y = H x with the full Hermitian FP64 H (G^-1 of FP64 plans); one warp per row
__global__ void k_hemv_full(const double2* H, int64_t N, const float2* xf, double2* y, const int* skip) {
    if (skip && *skip) return;
    const int lane = threadIdx.x & 31;
    const int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (i >= N) return;
    const double2* row = H + i * N;
    double2 acc = make_double2(0.0, 0.0);
    for (int64_t j = lane; j < N; j += 32) zfma(acc, row[j], make_double2(xf[j].x, xf[j].y));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) y[i] = acc;
}

// FP64 -> FP32 vector copy on the integer pipe
__global__ void k_vec_f32(const double2* a, float2* b, int64_t n) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = make_float2(f64_to_f32_rn(a[i].x), f64_to_f32_rn(a[i].y));
}

// -------------------------------------------------------------------- Hager's iteration
// |v| in FP32 from FP64 parts, without the FP64 pipe
__device__ inline float mag(double2 v) { return abs_f(v); }

// block sum of |v[i]| (FP32 magnitudes, double-float sums), result in every thread
__device__ double block_abs_sum(const double2* v, int64_t N, float2* red) {
    float h = 0.f, l = 0.f;
    for (int64_t i = threadIdx.x; i < N; i += CB) acc_df(h, l, mag(v[i]));
    const float2 w = warp_sum_df(h, l);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = w;
    __syncthreads();
    float2 t = threadIdx.x < CB / 32 ? red[threadIdx.x] : make_float2(0.f, 0.f);
    if (threadIdx.x < 32) t = warp_sum_df(t.x, t.y);
    if (threadIdx.x == 0) red[0] = t;
    __syncthreads();
    const double r = (double)red[0].x + (double)red[0].y;
    __syncthreads();
    return r;
}

__global__ void k_hg_init(float2* x, int64_t N, HagerState* h) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < N) x[i] = make_float2((float)(1.0 / (double)N), 0.f);
    if (i == 0) *h = HagerState{0.0, 0.0, -1, -1, 0, 0, -1};
}

// After y = G^-1 v with v the start vector (first = 1) or e_j: record the
// estimate ||y||_1 (||v||_1 = 1), stop when it no longer grows, keep the best y
// in ybest, and write xi = y / |y| (1 where y vanishes) for the next solve.
__global__ void __launch_bounds__(CB) k_hg_sign(const double2* y, float2* xi, double2* ybest, int64_t N,
                                                HagerState* h, int first) {
    __shared__ float2 red[CB / 32];
    __shared__ int stop;
    if (h->done) return;
    const double s = block_abs_sum(y, N, red);
    if (threadIdx.x == 0) {
        stop = 0;
        if (!first && s <= h->est) {
            h->done = 1;  // no growth: the iteration has converged
            stop = 1;
        } else {
            h->est = s;
            h->best_j = first ? -1 : h->j;
        }
    }
    __syncthreads();
    if (stop) return;
    for (int64_t i = threadIdx.x; i < N; i += CB) {
        const double2 v = y[i];
        ybest[i] = v;
        const float re = f64_to_f32_rn(v.x), im = f64_to_f32_rn(v.y);
        const float a = sqrtf(fmaf(re, re, im * im));
        xi[i] = a > 0.f ? make_float2(re / a, im / a) : make_float2(1.f, 0.f);
    }
}

// After z = G^-1 xi: j = the first index of the largest |z_j|. Stop when the
// previous index attains the same maximum or after HAGER_ROUNDS rounds;
// otherwise x = e_j.
__global__ void __launch_bounds__(CB) k_hg_pick(const double2* z, float2* x, int64_t N, HagerState* h) {
    __shared__ float rv[CB];
    __shared__ int ri[CB];
    __shared__ int stop, jn;
    if (h->done) return;
    float best = -1.f;
    int bi = 0;
    for (int64_t i = threadIdx.x; i < N; i += CB) {
        const float a = mag(z[i]);
        if (a > best) {
            best = a;
            bi = (int)i;
        }
    }
    rv[threadIdx.x] = best;
    ri[threadIdx.x] = bi;
    __syncthreads();
    for (int w = CB / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            const float o = rv[threadIdx.x + w];
            const int oi = ri[threadIdx.x + w];
            if (o > rv[threadIdx.x] || (o == rv[threadIdx.x] && oi < ri[threadIdx.x])) {
                rv[threadIdx.x] = o;
                ri[threadIdx.x] = oi;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const int j = ri[0];
        stop = 0;
        if (h->j >= 0 && (mag(z[h->j]) >= rv[0] || h->rounds >= HAGER_ROUNDS)) stop = 1;
        if (stop) h->done = 1;
        h->jlast = h->j;
        h->j = j;
        h->rounds += 1;
        jn = j;
    }
    __syncthreads();
    if (stop) return;
    for (int64_t i = threadIdx.x; i < N; i += CB) x[i] = make_float2(i == jn ? 1.f : 0.f, 0.f);
}

// x_i = (-1)^i (1 + i / (N - 1)), scaled to ||x||_1 = 1
__global__ void k_hg_alt(float2* x, int64_t N) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double v = N > 1 ? (1.0 + (double)i / (double)(N - 1)) / (1.5 * (double)N) : 1.0;
    x[i] = make_float2((float)((i & 1) ? -v : v), 0.f);
}

// est_alt = ||y||_1 / ||x||_1 for the rounded alternating vector; y kept in yalt
__global__ void __launch_bounds__(CB) k_hg_alt_finish(const double2* y, const float2* x, double2* yalt, int64_t N,
                                                      HagerState* h) {
    __shared__ float2 red[CB / 32];
    const double s = block_abs_sum(y, N, red);
    float th = 0.f, tl = 0.f;
    for (int64_t i = threadIdx.x; i < N; i += CB) {
        acc_df(th, tl, fabsf(x[i].x));
        yalt[i] = y[i];
    }
    const float2 w = warp_sum_df(th, tl);
    __syncthreads();
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = w;
    __syncthreads();
    if (threadIdx.x < 32) {
        float2 t = threadIdx.x < CB / 32 ? red[threadIdx.x] : make_float2(0.f, 0.f);
        t = warp_sum_df(t.x, t.y);
        if (threadIdx.x == 0) h->est_alt = s / ((double)t.x + (double)t.y);
    }
}

// the two final candidate vectors v in FP64: V[0] = the best iterate's start
// vector (uniform or e_j), V[1] = the alternating-sign vector (x)
__global__ void k_hg_vecs(const HagerState* h, const float2* x, double2* V, int64_t N) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const int bj = h->best_j;
    V[i] = make_double2(bj < 0 ? 1.0 / (double)N : (i == bj ? 1.0 : 0.0), 0.0);
    V[N + i] = make_double2(x[i].x, x[i].y);
}

// FP64 plans: kappa = ||G||_1 max(est, est_alt) (their G^-1 is accurate)
__global__ void k_hg_final(const HagerState* h, DevStatus* st) {
    st->kappa_est = st->norm1_g * fmax(h->est, h->est_alt);
}

// Mixed plans: kappa = ||G||_1 max_f ||Y[f]||_1 / ||R[f]||_1 with R = -G Y
__global__ void __launch_bounds__(CB) k_hg_certify(const double2* Y, const double2* R, int64_t N, DevStatus* st) {
    __shared__ float2 red[CB / 32];
    double best = 0.0;
    for (int f = 0; f < 2; ++f) {
        const double ny = block_abs_sum(Y + (int64_t)f * N, N, red);
        const double nr = block_abs_sum(R + (int64_t)f * N, N, red);
        if (nr > 0.0) best = fmax(best, ny / nr);
    }
    if (threadIdx.x == 0) st->kappa_est = st->norm1_g * best;
}

// row chunks of the column-sum kernels: at least 128 rows, at most 64 chunks
int64_t rows_per_chunk(int64_t N) { return std::max<int64_t>(128, (N + 63) / 64); }
int chunks_for(int64_t N) { return (int)((N + rows_per_chunk(N) - 1) / rows_per_chunk(N)); }

}  // namespace

// ||G||_1 into st->norm1_g: from the stored lower triangle of G (FP64 G, or
// double-float Gdf) or from the full double-float exact Gram Gx; one of the three
cudaError_t launch_gram_norm1(const double2* G, const float4* Gdf, const float4* Gx, int64_t N, int64_t ld,
                              DevStatus* st, cudaStream_t s) {
    const int chunks = Gx ? 0 : chunks_for(N);
    const int64_t rpc = rows_per_chunk(N);
    float2 *rs = nullptr, *part = nullptr;
    cudaError_t e = work_alloc((void**)&rs, sizeof(float2) * N, s);
    if (e != cudaSuccess) return e;
    if (chunks && (e = work_alloc((void**)&part, sizeof(float2) * N * chunks, s)) != cudaSuccess) return e;
    const unsigned rows_blocks = (unsigned)((N + 7) / 8);
    const dim3 cg((unsigned)((N + 255) / 256), (unsigned)chunks);
    if (Gx) {
        k_abs_rows<float4, true><<<rows_blocks, 256, 0, s>>>(Gx, N, N, rs);
    } else if (Gdf) {
        k_abs_rows<float4, false><<<rows_blocks, 256, 0, s>>>(Gdf, N, ld, rs);
        k_abs_cols_lower<float4><<<cg, 256, 0, s>>>(Gdf, N, ld, rpc, part);
        note_launch();
    } else {
        k_abs_rows<double2, false><<<rows_blocks, 256, 0, s>>>(G, N, ld, rs);
        k_abs_cols_lower<double2><<<cg, 256, 0, s>>>(G, N, ld, rpc, part);
        note_launch();
    }
    k_norm1_finish<<<1, CB, 0, s>>>(rs, part, chunks, N, &st->norm1_g);
    note_launch(2);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if (part) cudaFreeAsync(part, s);
    return cudaFreeAsync(rs, s);
}

// Hager's estimate of ||G^-1||_1 and kappa_1(G) = ||G||_1 ||G^-1||_1 into
// st->kappa_est (st->norm1_g must be set); runs after the factorisation.
pinv_status build_condition(pinv_plan* p, cudaStream_t s) {
    const int64_t N = p->N, M = p->M;
    const bool mixed = p->precision != PINV_FP64;
    const int chunks = chunks_for(N);
    const int64_t rpc = rows_per_chunk(N);
    // every buffer goes back to the pool in stream order when this returns, on
    // every path (the kernels enqueued before it still see it)
    struct Release {
        std::vector<void*> q;
        cudaStream_t s;
        ~Release() {
            for (void* b : q) cudaFreeAsync(b, s);
        }
    } bufs_{{}, s};
    auto take = [&](void** q, size_t bytes) -> cudaError_t {
        cudaError_t e = work_alloc(q, bytes, s);
        if (e == cudaSuccess) bufs_.q.push_back(*q);
        return e;
    };
    HagerState* h = nullptr;
    float2 *x = nullptr, *u = nullptr, *part = nullptr;
    double2 *y = nullptr, *z = nullptr, *Y2 = nullptr, *V2 = nullptr, *R2 = nullptr, *zero = nullptr, *U2 = nullptr;
    CKC(take((void**)&h, sizeof(HagerState)));
    CKC(take((void**)&x, sizeof(float2) * FMAX * N));
    CKC(take((void**)&y, sizeof(double2) * N));
    CKC(take((void**)&z, sizeof(double2) * N));
    CKC(take((void**)&Y2, sizeof(double2) * 2 * N));
    if (mixed) {
        CKC(take((void**)&u, sizeof(float2) * FMAX * N));
        CKC(take((void**)&part, sizeof(float2) * FMAX * N * chunks));
    }
    const unsigned vb = (unsigned)((N + 255) / 256), wb = (unsigned)((N + 7) / 8);
    const int* skip = &h->done;
    // out (+)= G^-1 x for F vectors in x (float2 [F][N]); skip_on: return at once
    // once the iteration is done
    auto solve = [&](double2* out, int F, bool skip_on, int accumulate) -> cudaError_t {
        const int* sk = skip_on ? skip : nullptr;
        if (mixed) {
            k_w_mv<<<wb, 256, 0, s>>>(p->W32, N, F, x, u, sk);
            k_wh_part<<<dim3(vb, (unsigned)chunks), 256, 0, s>>>(p->W32, N, F, u, rpc, part, sk);
            k_part_sum<<<(unsigned)((N * F + 255) / 256), 256, 0, s>>>(part, chunks, N, F, out, accumulate, sk);
            note_launch(3);
        } else {
            k_hemv_full<<<wb, 256, 0, s>>>(p->Ginv, N, x, out, sk);
            note_launch();
        }
        return cudaGetLastError();
    };
    k_hg_init<<<vb, 256, 0, s>>>(x, N, h);
    note_launch();
    CKC(solve(y, 1, false, 0));
    k_hg_sign<<<1, CB, 0, s>>>(y, x, Y2, N, h, 1);
    note_launch();
    CKC(solve(z, 1, true, 0));
    k_hg_pick<<<1, CB, 0, s>>>(z, x, N, h);
    note_launch();
    for (int r = 1; r < HAGER_ROUNDS; ++r) {
        CKC(solve(y, 1, true, 0));
        k_hg_sign<<<1, CB, 0, s>>>(y, x, Y2, N, h, 0);
        note_launch();
        CKC(solve(z, 1, true, 0));
        k_hg_pick<<<1, CB, 0, s>>>(z, x, N, h);
        note_launch();
    }
    k_hg_alt<<<vb, 256, 0, s>>>(x, N);
    note_launch();
    CKC(solve(y, 1, false, 0));
    k_hg_alt_finish<<<1, CB, 0, s>>>(y, x, Y2 + N, N, h);
    note_launch();
    CKC(cudaGetLastError());
    if (!mixed) {
        k_hg_final<<<1, 1, 0, s>>>(h, p->st);
        note_launch();
        return PINV_OK;
    }
    // Mixed plans: the two candidates v (V2) and their solves y (Y2), refined
    // (r = v - G y, y += W^H W r), then certified with R2 = -G Y2
    CKC(take((void**)&V2, sizeof(double2) * 2 * N));
    CKC(take((void**)&R2, sizeof(double2) * 2 * N));
    k_hg_vecs<<<vb, 256, 0, s>>>(h, x, V2, N);
    note_launch();
    const bool toep = p->refine_residual == PINV_RESIDUAL_TOEPLITZ;
    // plans with B0 and the digit tables of A and conj(A): E y and E^H u exactly on
    // the tensor cores (two frames in one 32-frame tile), far cheaper here than the
    // double-float products at two right-hand sides
    const bool xb0 = !toep && p->Af && p->Ad;
    float4* work = nullptr;
    uint8_t* bd = nullptr;
    int* fexp = nullptr;
    double2* Yb = nullptr;
    CKC(take((void**)&zero, sizeof(double2) * 2 * (toep ? N : M)));
    CKC(cudaMemsetAsync(zero, 0, sizeof(double2) * 2 * (toep ? N : M), s));
    if (toep && p->Gd) {
        const size_t wel = resid_exact_work_elems(N, 2);
        CKC(take((void**)&fexp, sizeof(int) * 2));
        CKC(take((void**)&bd, resid_bdigit_bytes(N, 2)));
        if (wel) CKC(take((void**)&work, sizeof(float4) * wel));
    } else if (toep) {
        const size_t wel = df_work_elems(N, 2, N);
        if (wel) CKC(take((void**)&work, sizeof(float4) * wel));
    } else if (xb0) {
        const size_t wel = std::max(exact_work_elems(p->enc, 2), exact_fwd_work_elems(p->enc, 2));
        CKC(take((void**)&U2, sizeof(double2) * 2 * M));
        CKC(take((void**)&fexp, sizeof(int) * 2));
        CKC(take((void**)&bd, std::max(exact_bdigit_bytes(p->enc, 2), exact_fwd_bdigit_bytes(p->enc, 2))));
        CKC(take((void**)&Yb, sizeof(double2) * exact_fwd_y_elems(p->enc, 2)));
        if (wel) CKC(take((void**)&work, sizeof(float4) * wel));
    } else {
        const size_t wel = std::max(df_work_elems(M, 2, N), df_work_elems(N, 2, M));
        CKC(take((void**)&U2, sizeof(double2) * 2 * M));
        if (wel && p->refine_residual == PINV_RESIDUAL_DOUBLE_FLOAT) CKC(take((void**)&work, sizeof(float4) * wel));
    }
    // R = B - G X by the refinement's residual operator (B = nullptr: R = -G X)
    auto resid = [&](const double2* B, const double2* X, double2* R) -> cudaError_t {
        cudaError_t e;
        if (toep && p->Gd) return launch_gram_resid_exact(p->Gd, p->eG, N, B ? B : zero, X, 2, fexp, bd, R, work,
                                                          p->st, s);
        if (toep) return launch_gram_resid_df(p->Gx, N, B ? B : zero, X, 2, R, s, work);
        if (xb0) {
            if ((e = launch_forward_exact(p->enc, X, 2, nullptr, U2, p->Af, Yb, fexp, bd, work, p->st, s)) !=
                cudaSuccess)  // U = -E X
                return e;
            if ((e = launch_adjoint_exact(p->enc, U2, 2, fexp, bd, R, work, p->st, s, p->Ad)) != cudaSuccess)
                return e;  // R = E^H U
            if ((e = launch_minus_lambda(R, X, p->lambda_abs, 2 * N, s)) != cudaSuccess) return e;
        } else if (p->refine_residual == PINV_RESIDUAL_DOUBLE_FLOAT) {
            if ((e = launch_forward_df(p->enc, X, 2, zero, U2, s, work)) != cudaSuccess) return e;  // U = -E X
            if ((e = launch_adjoint_df(p->enc, U2, 2, p->lambda_abs, X, R, s, work)) != cudaSuccess) return e;
        } else {
            if ((e = launch_forward64(p->enc, X, 2, nullptr, U2, s)) != cudaSuccess) return e;
            if ((e = launch_adjoint64(p->enc, U2, 2, p->lambda_abs, X, R, s)) != cudaSuccess) return e;
        }
        return B ? launch_zaxpy(R, B, 2 * N, s) : cudaSuccess;  // R = B - G X
    };
    // one refinement step: the split factor's error shrinks about kappa(G) u_split
    // times (tens of times), far more than a factor-3 estimate needs
    for (int it = 0; it < 1; ++it) {
        CKC(resid(V2, Y2, R2));
        k_vec_f32<<<(unsigned)((2 * N + 255) / 256), 256, 0, s>>>(R2, x, 2 * N);
        note_launch();
        CKC(solve(Y2, 2, false, 1));
    }
    CKC(resid(nullptr, Y2, R2));
    k_hg_certify<<<1, CB, 0, s>>>(Y2, R2, N, p->st);
    note_launch();
    CKC(cudaGetLastError());
    return PINV_OK;
}

}  // namespace pinv
