// Eigenvalue decomposition of the Gram matrix and the truncated reconstruction
// (Section 2.1: the SVD spectrum of Encode, truncated SVD, and the eigenvalue
// decomposition E^H E + lambda I = P Lambda P^H of the normal equations).
//
// Parallel cyclic Jacobi, two-sided, in FP64 on a copy of the plan's kept Gram.
// A sweep is np - 1 rounds (np = n rounded up to even; an odd n leaves one index
// idle per round). Round r pairs every index once by the circle method: index
// np - 1 with r, and (r + k) mod (np - 1) with (r - k) mod (np - 1). Pair (p, q)
// gets the rotation J = diag(1, e^{-i phi}) R(theta) that zeroes G[p][q] (phi the
// phase of G[p][q], theta the real Jacobi angle of the phase-corrected 2 x 2
// block). The rotations of a round touch disjoint rows and columns, so they apply
// together and in place: G <- G J (each row mixes its entries p and q; a CTA
// rotates a row staged in shared memory), G <- J^H G (a CTA mixes rows p and q),
// and V <- V J. The rounds of a sweep are captured once into a CUDA graph and
// replayed. Sweeps stop when the off-diagonal Frobenius norm is below 4 n eps of
// the whole (the rounding floor of the rotations grows with n), or when a sweep
// no longer halves it once it is below 1e-10 of the whole, or after 30.
#include <algorithm>
#include <cmath>
#include <climits>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "plan_impl.h"

namespace pinv {
namespace {

pinv_status eig_err(cudaError_t e, const char* where) {
    return set_error(e == cudaErrorMemoryAllocation ? PINV_ERR_OOM : PINV_ERR_CUDA,
                     std::string(where) + ": " + cudaGetErrorString(e));
}

constexpr int EIG_MAX_N = 8192;   // Jacobi path: the sort stages all eigenvalues in one CTA
constexpr int EIG_MAX_SWEEPS = 30;

__device__ inline double2 cmul(double2 a, double2 b) { return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x); }
__device__ inline double2 cconj(double2 a) { return make_double2(a.x, -a.y); }
__device__ inline double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }

// pair k of round r (circle method over np indices), p < q
__device__ inline void round_pair(int np, int r, int k, int& p, int& q) {
    if (k == 0) {
        p = r;
        q = np - 1;
    } else {
        p = (r + k) % (np - 1);
        q = (r - k + np - 1) % (np - 1);
    }
    if (p > q) {
        const int t = p;
        p = q;
        q = t;
    }
}

// One rotation per pair: new column j = column j * ca[j] + column part[j] * cb[j].
__global__ void k_jac_rot(const double2* __restrict__ A, int n, int np, int r, double2* ca, double2* cb, int* part) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= np / 2) return;
    int p, q;
    round_pair(np, r, k, p, q);
    if (q >= n) {  // p is paired with the idle index
        ca[p] = make_double2(1.0, 0.0);
        cb[p] = make_double2(0.0, 0.0);
        part[p] = p;
        return;
    }
    const double a = A[(int64_t)p * n + p].x, d = A[(int64_t)q * n + q].x;
    const double2 b = A[(int64_t)p * n + q];
    const double babs = hypot(b.x, b.y);
    double2 jpp = make_double2(1.0, 0.0), jpq = make_double2(0.0, 0.0), jqp = make_double2(0.0, 0.0),
            jqq = make_double2(1.0, 0.0);
    if (babs > 0.0) {
        const double2 ph = make_double2(b.x / babs, b.y / babs);  // G[p][q] = |G[p][q]| e^{i phi}
        const double zeta = (d - a) / (2.0 * babs);
        const double t = fabs(zeta) > 1e150 ? 0.5 / zeta
                                            : (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
        // J = diag(1, e^{-i phi}) [[c, s], [-s, c]]
        jpp = make_double2(c, 0.0);
        jpq = make_double2(s, 0.0);
        jqp = make_double2(-s * ph.x, s * ph.y);  // -s conj(ph)
        jqq = make_double2(c * ph.x, -c * ph.y);  // c conj(ph)
    }
    ca[p] = jpp;
    cb[p] = jqp;
    part[p] = q;
    ca[q] = jqq;
    cb[q] = jpq;
    part[q] = p;
}

// M <- M J for G and V (blockIdx.y: row, blockIdx.z: 0 = G, 1 = V), in place through shared memory
__global__ void __launch_bounds__(256) k_jac_cols(double2* G, double2* V, int n, const double2* __restrict__ ca,
                                                 const double2* __restrict__ cb, const int* __restrict__ part) {
    extern __shared__ double2 row[];
    double2* M = blockIdx.z ? V : G;
    double2* m = M + (int64_t)blockIdx.y * n;
    for (int j = threadIdx.x; j < n; j += blockDim.x) row[j] = m[j];
    __syncthreads();
    for (int j = threadIdx.x; j < n; j += blockDim.x) m[j] = cadd(cmul(row[j], ca[j]), cmul(row[part[j]], cb[j]));
}

// G <- J^H G: row j becomes conj(ca[j]) row j + conj(cb[j]) row part[j] (one CTA per pair)
__global__ void __launch_bounds__(256) k_jac_rows(double2* G, int n, int np, int r, const double2* __restrict__ ca,
                                                 const double2* __restrict__ cb) {
    int p, q;
    round_pair(np, r, blockIdx.x, p, q);
    if (q >= n) return;
    double2* gp = G + (int64_t)p * n;
    double2* gq = G + (int64_t)q * n;
    const double2 app = cconj(ca[p]), apq = cconj(cb[p]), aqq = cconj(ca[q]), aqp = cconj(cb[q]);
    for (int c = threadIdx.x; c < n; c += blockDim.x) {
        const double2 x = gp[c], y = gq[c];
        gp[c] = cadd(cmul(app, x), cmul(apq, y));
        gq[c] = cadd(cmul(aqq, y), cmul(aqp, x));
    }
}

// the upper triangle from the lower (the Gram kernels write only the lower part)
__global__ void k_hermitian_fill(double2* A, int n) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * n) return;
    const int i = (int)(idx / n), j = (int)(idx % n);
    if (j > i) A[idx] = cconj(A[(int64_t)j * n + i]);
    if (j == i) A[idx].y = 0.0;
}

__global__ void k_identity(double2* V, int n) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx < (int64_t)n * n) V[idx] = make_double2(idx / n == idx % n ? 1.0 : 0.0, 0.0);
}

// per-row sums of |A_ij|^2: off-diagonal in part[i], the diagonal in part[n + i]
__global__ void __launch_bounds__(256) k_row_norms(const double2* __restrict__ A, int n, double* part) {
    __shared__ double s_off[256], s_dia[256];
    const int i = blockIdx.x;
    double off = 0.0, dia = 0.0;
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const double2 v = A[(int64_t)i * n + j];
        const double m = v.x * v.x + v.y * v.y;
        if (j == i) dia += m;
        else off += m;
    }
    s_off[threadIdx.x] = off;
    s_dia[threadIdx.x] = dia;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            s_off[threadIdx.x] += s_off[threadIdx.x + w];
            s_dia[threadIdx.x] += s_dia[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[i] = s_off[0];
        part[n + i] = s_dia[0];
    }
}
// out[0] = off-diagonal, out[1] = whole squared Frobenius norm (fixed summation order)
__global__ void __launch_bounds__(256) k_sum_norms(const double* part, int n, double* out) {
    __shared__ double s_off[256], s_all[256];
    double off = 0.0, all = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        off += part[i];
        all += part[i] + part[n + i];
    }
    s_off[threadIdx.x] = off;
    s_all[threadIdx.x] = all;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) {
            s_off[threadIdx.x] += s_off[threadIdx.x + w];
            s_all[threadIdx.x] += s_all[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = s_off[0];
        out[1] = s_all[0];
    }
}

// Eigenvalues (diag(A) - lam) in decreasing order, ties by index: bitonic sort of
// (value, index) in one CTA over a power-of-two padding; order[i] = index of mu[i].
__global__ void __launch_bounds__(1024) k_eig_sort(const double2* __restrict__ A, int n, int npow, double lam,
                                                  double* mu, int* order) {
    extern __shared__ double sv[];
    int* si = reinterpret_cast<int*>(sv + npow);
    for (int i = threadIdx.x; i < npow; i += blockDim.x) {
        sv[i] = i < n ? A[(int64_t)i * n + i].x - lam : -INFINITY;
        si[i] = i;
    }
    __syncthreads();
    for (int size = 2; size <= npow; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int i = threadIdx.x; i < npow; i += blockDim.x) {
                const int j = i ^ stride;
                if (j > i) {
                    // descending by value, ascending by index: "before" means larger value or same value, smaller index
                    const bool i_before = sv[i] > sv[j] || (sv[i] == sv[j] && si[i] < si[j]);
                    const bool want_i_before = (i & size) == 0;
                    if (i_before != want_i_before) {
                        const double tv = sv[i];
                        sv[i] = sv[j];
                        sv[j] = tv;
                        const int ti = si[i];
                        si[i] = si[j];
                        si[j] = ti;
                    }
                }
            }
            __syncthreads();
        }
    }
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        mu[i] = sv[i];
        order[i] = si[i];
    }
}

// P[row][i] = V[row][order[i]] (conj = 0), or Ph[i][row] = conj(V[row][order[i]]) (conj = 1)
__global__ void k_eig_gather(const double2* __restrict__ V, int n, const int* __restrict__ order, int conj_t,
                             double2* out) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * n) return;
    const int row = (int)(idx / n), i = (int)(idx % n);
    const double2 v = V[(int64_t)row * n + order[i]];
    if (conj_t) out[(int64_t)i * n + row] = cconj(v);
    else out[idx] = v;
}

// rank r: the fewest leading eigenvalues holding `energy` of their (non-negative)
// sum, summed in order by one thread; weights w_i = 1 / (mu_i + lam) for i < r, else 0
__global__ void k_tsvd_rank(const double* mu, int n, double energy, double lam, int* rank, double* kappa, double* w) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        double total = 0.0;
        for (int i = 0; i < n; ++i) total += fmax(mu[i], 0.0);
        const double target = energy * total;
        double c = 0.0;
        int r = n;
        for (int i = 0; i < n; ++i) {
            c += fmax(mu[i], 0.0);
            if (c >= target) {
                r = i + 1;
                break;
            }
        }
        *rank = r;
        *kappa = mu[r - 1] > 0.0 ? sqrt(mu[0] / mu[r - 1]) : INFINITY;
    }
    __syncthreads();
    const int r = *rank;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        w[i] = i < r ? 1.0 / (mu[i] + lam) : 0.0;
}

// Ph[i][row] = conj(P[row][i])
__global__ void k_conj_transpose(const double2* __restrict__ P, int n, double2* __restrict__ Ph) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * n) return;
    const int row = (int)(idx / n), i = (int)(idx % n);
    Ph[(int64_t)i * n + row] = cconj(P[idx]);
}

// C[f][i] *= w[i]
__global__ void k_scale_rows(double2* C, int64_t F, int n, const double* __restrict__ w) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= F * n) return;
    const double s = w[idx % n];
    C[idx].x *= s;
    C[idx].y *= s;
}

// ------------------------------------------------------------------ eigenvalues only
// Householder reduction of the Hermitian A to a real symmetric tridiagonal, one
// column k at a time (the reflector's scalar tau is chosen so that the subdiagonal
// entry beta is real), then bisection with Sturm counts, one eigenvalue per thread.
// Column k below the diagonal is read as the conjugate of row k to the right of it.
// With H = I - tau v v^H: p = tau A v, c = -Re(conj(tau) v^H p) / 2,
// w = p + c v, A <- H^H A H = A - w v^H - v w^H on the trailing block.
struct HhScalars {
    double2 tau;
    double beta;
    double c;
};

// reflector of x = A[k + 1 ..][k]: v (v[0] = 1), tau, beta; d[k] and e[k] recorded
__global__ void __launch_bounds__(256) k_hh_reflector(const double2* __restrict__ A, int n, int k, double2* v,
                                                     HhScalars* hs, double* d, double* e) {
    __shared__ double red[256];
    const int m = n - k - 1;
    const double2* row = A + (int64_t)k * n + k + 1;  // conj(x_j) = row[j]
    double s = 0.0;
    for (int j = 1 + threadIdx.x; j < m; j += blockDim.x) s += row[j].x * row[j].x + row[j].y * row[j].y;
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const double xnorm2 = red[0];
    const double2 alpha = cconj(row[0]);
    double2 tau = make_double2(0.0, 0.0), scale = make_double2(0.0, 0.0);
    double beta = alpha.x;
    if (xnorm2 > 0.0 || alpha.y != 0.0) {
        const double nrm = sqrt(alpha.x * alpha.x + alpha.y * alpha.y + xnorm2);
        beta = alpha.x >= 0.0 ? -nrm : nrm;
        tau = make_double2((beta - alpha.x) / beta, -alpha.y / beta);
        // scale = 1 / (alpha - beta)
        const double2 den = make_double2(alpha.x - beta, alpha.y);
        const double dd = den.x * den.x + den.y * den.y;
        scale = make_double2(den.x / dd, -den.y / dd);
    }
    for (int j = threadIdx.x; j < m; j += blockDim.x)
        v[j] = j == 0 ? make_double2(1.0, 0.0) : cmul(cconj(row[j]), scale);
    if (threadIdx.x == 0) {
        hs->tau = tau;
        hs->beta = beta;
        d[k] = A[(int64_t)k * n + k].x;
        e[k] = beta;
    }
}

// p = tau A22 v (A22 = A[k + 1 ..][k + 1 ..]), one warp per row
__global__ void __launch_bounds__(256) k_hh_matvec(const double2* __restrict__ A, int n, int k,
                                                  const double2* __restrict__ v, const HhScalars* hs, double2* p) {
    const int m = n - k - 1;
    const int i = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (i >= m) return;
    const double2* row = A + (int64_t)(k + 1 + i) * n + k + 1;
    double2 acc = make_double2(0.0, 0.0);
    for (int j = lane; j < m; j += 32) acc = cadd(acc, cmul(row[j], v[j]));
    for (int o = 16; o > 0; o >>= 1) {
        acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
        acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) p[i] = cmul(hs->tau, acc);
}

// c = -Re(conj(tau) v^H p) / 2
__global__ void __launch_bounds__(256) k_hh_coef(int n, int k, const double2* __restrict__ v,
                                                const double2* __restrict__ p, HhScalars* hs) {
    __shared__ double red[256];
    const int m = n - k - 1;
    double2 acc = make_double2(0.0, 0.0);
    for (int j = threadIdx.x; j < m; j += blockDim.x) acc = cadd(acc, cmul(cconj(v[j]), p[j]));
    // real part of conj(tau) * acc
    const double2 t = cconj(hs->tau);
    red[threadIdx.x] = t.x * acc.x - t.y * acc.y;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) hs->c = -0.5 * red[0];
}

// A22 -= w v^H + v w^H with w = p + c v; row k's part beyond the diagonal becomes (beta, 0, ..)
__global__ void __launch_bounds__(256) k_hh_update(double2* A, int n, int k, const double2* __restrict__ v,
                                                  const double2* __restrict__ p, const HhScalars* hs) {
    const int m = n - k - 1;
    const int i = blockIdx.y;
    const double c = hs->c;
    const double2 vi = v[i], wi = cadd(p[i], make_double2(c * vi.x, c * vi.y));
    double2* row = A + (int64_t)(k + 1 + i) * n + k + 1;
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < m; j += gridDim.x * blockDim.x) {
        const double2 vj = v[j], wj = cadd(p[j], make_double2(c * vj.x, c * vj.y));
        const double2 t = cadd(cmul(wi, cconj(vj)), cmul(vi, cconj(wj)));
        row[j] = make_double2(row[j].x - t.x, row[j].y - t.y);
    }
}

// last 2 x 2 block: d[n-2], d[n-1], e[n-2] = |A[n-1][n-2]|
__global__ void k_hh_tail(const double2* __restrict__ A, int n, double* d, double* e) {
    if (n >= 2) {
        d[n - 2] = A[(int64_t)(n - 2) * n + n - 2].x;
        const double2 b = A[(int64_t)(n - 1) * n + n - 2];
        e[n - 2] = hypot(b.x, b.y);
    }
    d[n - 1] = A[(int64_t)(n - 1) * n + n - 1].x;
}

// eigenvalue number i (ascending) of the symmetric tridiagonal (d, e) by bisection;
// mu[n - 1 - i] = it minus lam (decreasing order)
__global__ void k_tridiag_bisect(const double* __restrict__ d, const double* __restrict__ e, int n, double lam,
                                 double* mu) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double lo = INFINITY, hi = -INFINITY;
    for (int k = 0; k < n; ++k) {
        const double r = (k > 0 ? fabs(e[k - 1]) : 0.0) + (k < n - 1 ? fabs(e[k]) : 0.0);
        lo = fmin(lo, d[k] - r);
        hi = fmax(hi, d[k] + r);
    }
    const double span = fmax(fabs(lo), fabs(hi));
    const double pivmin = 1e-300 + span * 1e-300;
    for (int it = 0; it < 200 && hi - lo > 2.220446049250313e-16 * fmax(fabs(lo), fabs(hi)); ++it) {
        const double x = 0.5 * (lo + hi);
        int cnt = 0;
        double q = d[0] - x;
        if (fabs(q) < pivmin) q = -pivmin;
        cnt += q < 0.0;
        for (int k = 1; k < n; ++k) {
            q = d[k] - x - e[k - 1] * e[k - 1] / q;
            if (fabs(q) < pivmin) q = -pivmin;
            cnt += q < 0.0;
        }
        if (cnt > i) hi = x;  // at least i + 1 eigenvalues below x
        else lo = x;
    }
    mu[n - 1 - i] = 0.5 * (lo + hi) - lam;
}

inline unsigned blocks(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

}  // namespace
}  // namespace pinv

using namespace pinv;

extern "C" pinv_status pinv_plan_eig(pinv_plan* p, double* d_mu, void* d_P, int* sweeps_out, void* stream) {
    if (!p || !d_mu) return set_error(PINV_ERR_INVALID_ARG, "null plan or eigenvalue output");
    if (!p->built) return set_error(PINV_ERR_NOT_BUILT, "plan not built");
    if (!p->Gkeep) return set_error(PINV_ERR_UNSUPPORTED, "the eigendecomposition needs the kept Gram (keep_gram)");
    if (d_P && p->N > EIG_MAX_N)
        return set_error(PINV_ERR_UNSUPPORTED, "eigenvectors limited to N <= 8192 (eigenvalues alone are not)");
    if (p->N > INT_MAX / 2) return set_error(PINV_ERR_UNSUPPORTED, "N too large");
    const int n = (int)p->N, np = n + (n & 1);
    cudaStream_t us = (cudaStream_t)stream;
    const size_t nn = (size_t)n * n;
    double2 *A = nullptr, *V = nullptr, *ca = nullptr, *cb = nullptr;
    int *part = nullptr, *order = nullptr;
    double *norms = nullptr, *hn = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t ev = nullptr;
    cudaGraphExec_t sweep = nullptr;
    pinv_status result = PINV_OK;
    auto done = [&](pinv_status st) {
        if (sweep) cudaGraphExecDestroy(sweep);
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
        if (ev) cudaEventDestroy(ev);
        for (void* ptr : {(void*)A, (void*)V, (void*)ca, (void*)cb, (void*)part, (void*)order, (void*)norms})
            if (ptr) cudaFree(ptr);
        if (hn) cudaFreeHost(hn);
        return st;
    };
#define CKE(call)                                                \
    do {                                                         \
        cudaError_t e_ = (call);                                 \
        if (e_ != cudaSuccess) return done(eig_err(e_, #call));  \
    } while (0)
    CKE(cudaMalloc(&A, sizeof(double2) * nn));
    CKE(cudaMalloc(&V, sizeof(double2) * nn));
    CKE(cudaMalloc(&ca, sizeof(double2) * np));
    CKE(cudaMalloc(&cb, sizeof(double2) * np));
    CKE(cudaMalloc(&part, sizeof(int) * np));
    CKE(cudaMalloc(&order, sizeof(int) * np));
    CKE(cudaMalloc(&norms, sizeof(double) * (2 * (size_t)n + 2)));
    CKE(cudaMallocHost(&hn, sizeof(double) * 2));
    // a private stream (graph capture needs one), ordered after the caller's work
    CKE(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
    CKE(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    CKE(cudaEventRecord(ev, us));
    CKE(cudaStreamWaitEvent(s, ev, 0));

    CKE(cudaMemcpyAsync(A, p->Gkeep, sizeof(double2) * nn, cudaMemcpyDeviceToDevice, s));
    k_hermitian_fill<<<blocks((int64_t)nn), 256, 0, s>>>(A, n);
    note_launch();
    CKE(cudaGetLastError());
    if (!d_P) {
        // eigenvalues only: Householder tridiagonalisation, then bisection; the
        // 4 (n - 2) launches of the reduction run from one graph
        double2 *v = V, *pv = V + n;  // V is not needed on this path: its first 2n entries hold v and p
        double *dd = norms, *ee = norms + n;
        HhScalars* hs = reinterpret_cast<HhScalars*>(ca);
        cudaGraph_t g = nullptr;
        CKE(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        for (int k = 0; k + 2 < n; ++k) {
            const int m = n - k - 1;
            k_hh_reflector<<<1, 256, 0, s>>>(A, n, k, v, hs, dd, ee);
            k_hh_matvec<<<blocks(m, 8), 256, 0, s>>>(A, n, k, v, hs, pv);
            k_hh_coef<<<1, 256, 0, s>>>(n, k, v, pv, hs);
            k_hh_update<<<dim3(blocks(m), m), 256, 0, s>>>(A, n, k, v, pv, hs);
        }
        k_hh_tail<<<1, 1, 0, s>>>(A, n, dd, ee);
        k_tridiag_bisect<<<blocks(n, 128), 128, 0, s>>>(dd, ee, n, p->lambda_abs, d_mu);
        const cudaError_t ec = cudaStreamEndCapture(s, &g);
        if (ec != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return done(eig_err(ec, "cudaStreamEndCapture"));
        }
        const cudaError_t ei = cudaGraphInstantiate(&sweep, g, 0);
        cudaGraphDestroy(g);
        CKE(ei);
        CKE(cudaGraphLaunch(sweep, s));
        note_launch((unsigned long long)4 * (n > 2 ? n - 2 : 0) + 2);
        CKE(cudaEventRecord(ev, s));
        CKE(cudaStreamWaitEvent(us, ev, 0));
        if (sweeps_out) *sweeps_out = 0;
        return done(PINV_OK);
    }
    k_identity<<<blocks((int64_t)nn), 256, 0, s>>>(V, n);
    note_launch();
    CKE(cudaGetLastError());
    const size_t row_smem = sizeof(double2) * n;
    CKE(cudaFuncSetAttribute(k_jac_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)row_smem));

    // one sweep as a graph: np - 1 rounds of (rotations, G J and V J, J^H G)
    {
        cudaGraph_t g = nullptr;
        CKE(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        for (int r = 0; r < np - 1; ++r) {
            k_jac_rot<<<blocks(np / 2), 256, 0, s>>>(A, n, np, r, ca, cb, part);
            k_jac_cols<<<dim3(1, n, 2), 256, row_smem, s>>>(A, V, n, ca, cb, part);
            k_jac_rows<<<np / 2, 256, 0, s>>>(A, n, np, r, ca, cb);
        }
        const cudaError_t ec = cudaStreamEndCapture(s, &g);
        if (ec != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return done(eig_err(ec, "cudaStreamEndCapture"));
        }
        const cudaError_t ei = cudaGraphInstantiate(&sweep, g, 0);
        cudaGraphDestroy(g);
        CKE(ei);
    }
    const double tol = 4.0 * n * 2.220446049250313e-16;  // relative off-diagonal norm
    int sweeps = 0;
    double prev = INFINITY;
    bool converged = false;
    for (;; ++sweeps) {
        k_row_norms<<<n, 256, 0, s>>>(A, n, norms);
        k_sum_norms<<<1, 256, 0, s>>>(norms, n, norms + 2 * n);
        note_launch(2);
        CKE(cudaMemcpyAsync(hn, norms + 2 * n, sizeof(double) * 2, cudaMemcpyDeviceToHost, s));
        CKE(cudaStreamSynchronize(s));
        const double off = hn[1] > 0.0 ? sqrt(hn[0] / hn[1]) : 0.0;
        if (off <= tol || (off <= 1e-10 && off > 0.5 * prev)) {
            converged = true;
            break;
        }
        if (sweeps == EIG_MAX_SWEEPS) break;
        prev = off;
        CKE(cudaGraphLaunch(sweep, s));
        note_launch((unsigned long long)3 * (np - 1));
    }
    if (!converged) result = set_error(PINV_ERR_INTERNAL, "Jacobi sweeps did not converge");
    int npow = 1;
    while (npow < n) npow <<= 1;
    const size_t sort_smem = (sizeof(double) + sizeof(int)) * npow;
    CKE(cudaFuncSetAttribute(k_eig_sort, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sort_smem));
    k_eig_sort<<<1, 1024, sort_smem, s>>>(A, n, npow, p->lambda_abs, d_mu, order);
    note_launch();
    if (d_P) {
        k_eig_gather<<<blocks((int64_t)nn), 256, 0, s>>>(V, n, order, 0, (double2*)d_P);
        note_launch();
    }
    CKE(cudaGetLastError());
    // the caller's stream sees the results
    CKE(cudaEventRecord(ev, s));
    CKE(cudaStreamWaitEvent(us, ev, 0));
    if (sweeps_out) *sweeps_out = sweeps;
#undef CKE
    return done(result);
}

extern "C" pinv_status pinv_tsvd_apply(pinv_plan* p, const double* d_mu, const void* d_P, double energy,
                                       double lam, const void* d_data, void* d_image, int64_t F, int dtype,
                                       int* rank_out, double* kappa_out, void* stream) {
    pinv_status st = apply_check(p, d_data, d_image, F, dtype);
    if (st != PINV_OK) return st;
    if (!d_mu || !d_P) return set_error(PINV_ERR_INVALID_ARG, "null eigenvalues or eigenvectors");
    if (!(energy > 0.0 && energy <= 1.0)) return set_error(PINV_ERR_INVALID_ARG, "energy must be in (0, 1]");
    if (!(lam >= 0.0)) return set_error(PINV_ERR_INVALID_ARG, "lam must be >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = p->N, M = p->M;
    double2 *D = nullptr, *b = nullptr, *c = nullptr, *Ph = nullptr, *X = nullptr;
    double* w = nullptr;
    int* dev_rank = nullptr;
    double* dev_kappa = nullptr;
    auto release = [&]() {
        for (void* ptr : {(void*)D, (void*)b, (void*)c, (void*)Ph, (void*)X, (void*)w, (void*)dev_rank, (void*)dev_kappa})
            if (ptr) cudaFreeAsync(ptr, s);
    };
#define CKT(call)                                        \
    do {                                                 \
        cudaError_t e_ = (call);                         \
        if (e_ != cudaSuccess) {                         \
            release();                                   \
            return eig_err(e_, #call);                   \
        }                                                \
    } while (0)
    CKT(work_alloc((void**)&w, sizeof(double) * N, s));
    CKT(work_alloc((void**)&dev_rank, sizeof(int), s));
    CKT(work_alloc((void**)&dev_kappa, sizeof(double), s));
    k_tsvd_rank<<<1, 256, 0, s>>>(d_mu, (int)N, energy, lam, dev_rank, dev_kappa, w);
    note_launch();
    CKT(cudaGetLastError());
    if (F > 0) {
        const double2* Dd = (const double2*)d_data;
        if (dtype == PINV_C64) {
            CKT(work_alloc((void**)&D, sizeof(double2) * F * M, s));
            CKT(launch_c64_to_c128((const float2*)d_data, D, F * M, s));
            Dd = D;
        }
        double2* Xd = (double2*)d_image;
        if (dtype == PINV_C64) {
            CKT(work_alloc((void**)&X, sizeof(double2) * F * N, s));
            Xd = X;
        }
        CKT(work_alloc((void**)&b, sizeof(double2) * F * N, s));
        CKT(work_alloc((void**)&c, sizeof(double2) * F * N, s));
        CKT(work_alloc((void**)&Ph, sizeof(double2) * N * N, s));
        CKT(launch_adjoint64(p->enc, Dd, F, 0.0, nullptr, b, s));  // b = E^H d
        k_conj_transpose<<<blocks(N * N), 256, 0, s>>>((const double2*)d_P, (int)N, Ph);  // Ph = P^H
        note_launch();
        CKT(cudaGetLastError());
        CKT(launch_apply64(Ph, N, N, b, F, c, s));  // c = P^H b
        k_scale_rows<<<blocks(F * N), 256, 0, s>>>(c, F, (int)N, w);
        note_launch();
        CKT(cudaGetLastError());
        CKT(launch_apply64((const double2*)d_P, N, N, c, F, Xd, s));  // x = P c
        if (dtype == PINV_C64) CKT(launch_c128_to_c64(Xd, (float2*)d_image, F * N, s));
    }
    if (rank_out || kappa_out) {
        int hr = 0;
        double hk = 0.0;
        CKT(cudaMemcpyAsync(&hr, dev_rank, sizeof(int), cudaMemcpyDeviceToHost, s));
        CKT(cudaMemcpyAsync(&hk, dev_kappa, sizeof(double), cudaMemcpyDeviceToHost, s));
        CKT(cudaStreamSynchronize(s));
        if (rank_out) *rank_out = hr;
        if (kappa_out) *kappa_out = hk;
    }
    release();
#undef CKT
    return PINV_OK;
}
