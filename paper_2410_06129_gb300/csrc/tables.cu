// Phase tables and small elementwise kernels.
//
// The Fourier factor of Eq. 2 separates over grid dimensions for voxels on a
// Cartesian grid: exp(-i2pi k.r) = prod_d exp(-i2pi k_d r_d). The tables hold
// each 1-D factor per sample, so an element of the encoding matrix costs one
// or two complex multiplies instead of a full sincos. The B0 factor of
// Section 3.3, exp(-i2pi df_n t_m), depends on the sample only through its
// time; samples sharing a time (same position within a readout) share a row.
// Arguments are reduced modulo one cycle in FP64 before sincospi.
#include <climits>

#include "df.cuh"

namespace pinv {

__device__ inline double2 phasor_neg2pi(double cycles) {
    double red = cycles - rint(cycles);
    double s, c;
    sincospi(2.0 * red, &s, &c);
    return make_double2(c, -s);
}

__global__ void k_tables(const double* __restrict__ traj, int ndim, int64_t Mk, int d, int width,
                         double fov, double2* __restrict__ out, float2* __restrict__ out32) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= Mk * width) return;
    int64_t m = idx / width;
    int i = (int)(idx % width);
    double x = ((double)i - width / 2.0) / width * fov;
    double k = traj[m * ndim + d];
    double2 v = phasor_neg2pi(k * x);
    out[idx] = v;
    out32[idx] = make_float2((float)v.x, (float)v.y);
}

__global__ void k_ones(int64_t n, double2* out, float2* out32) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        out[i] = make_double2(1.0, 0.0);
        out32[i] = make_float2(1.f, 0.f);
    }
}

static inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

cudaError_t launch_tables(const double* traj, int ndim, int64_t Mk, const int* dims,
                          const double* fov, double2* ex, double2* ey, double2* ez,
                          float2* ex32, float2* ey32, float2* ez32, cudaStream_t s) {
    double2* outs[3] = {ex, ey, ez};
    float2* outs32[3] = {ex32, ey32, ez32};
    for (int d = 0; d < 3; ++d) {
        if (d < ndim) {
            int64_t n = Mk * dims[d];
            k_tables<<<nblk(n, 256), 256, 0, s>>>(traj, ndim, Mk, d, dims[d], fov[d], outs[d],
                                                  outs32[d]);
            note_launch();
        } else {
            k_ones<<<nblk(Mk, 256), 256, 0, s>>>(Mk, outs[d], outs32[d]);
            note_launch();
        }
    }
    return cudaGetLastError();
}

__global__ void k_b0(const double* __restrict__ b0, const double* __restrict__ tu, int T, int64_t N,
                     double2* __restrict__ tab, float2* __restrict__ tab32) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)T * N) return;
    int64_t u = idx / N, n = idx % N;
    double2 v = phasor_neg2pi(b0[n] * tu[u]);
    tab[idx] = v;
    tab32[idx] = make_float2((float)v.x, (float)v.y);
}

cudaError_t launch_b0_table(const double* b0, const double* tuniq, int T, int64_t N, double2* tab,
                            float2* tab32, cudaStream_t s) {
    k_b0<<<nblk((int64_t)T * N, 256), 256, 0, s>>>(b0, tuniq, T, N, tab, tab32);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_to_f32(const double2* a, float2* b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = make_float2((float)a[i].x, (float)a[i].y);
}
cudaError_t launch_to_f32(const double2* src, float2* dst, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_to_f32<<<nblk(n, 256), 256, 0, s>>>(src, dst, n);
    note_launch();
    return cudaGetLastError();
}
cudaError_t launch_c128_to_c64(const double2* a, float2* b, int64_t n, cudaStream_t s) {
    return launch_to_f32(a, b, n, s);
}

__global__ void k_to_f64(const float2* a, double2* b, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = make_double2((double)a[i].x, (double)a[i].y);
}
cudaError_t launch_c64_to_c128(const float2* a, double2* b, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_to_f64<<<nblk(n, 256), 256, 0, s>>>(a, b, n);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_identity(double2* W, int64_t N, int64_t ld) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * N) return;
    int64_t i = idx / N, j = idx % N;
    W[i * ld + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
}
cudaError_t launch_fill_identity(double2* W, int64_t N, int64_t ld, cudaStream_t s) {
    k_identity<<<nblk(N * N, 256), 256, 0, s>>>(W, N, ld);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_identity_df(float4* W, int64_t N, int64_t ld) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * N) return;
    int64_t i = idx / N, j = idx % N;
    W[i * ld + j] = make_float4(i == j ? 1.f : 0.f, 0.f, 0.f, 0.f);
}
cudaError_t launch_fill_identity_df(float4* W, int64_t N, int64_t ld, cudaStream_t s) {
    k_identity_df<<<nblk(N * N, 256), 256, 0, s>>>(W, N, ld);
    note_launch();
    return cudaGetLastError();
}

// each entry in place: the 16 bytes of a double-float complex become the FP64
// value (join_f64, integer pipe). Above the diagonal W32 is written as zero, and so
// is W inside the diagonal blocks of width `blk`; the rest of W's upper triangle
// holds zero bits already (written once, the same in both forms).
__global__ void k_df_finish(float4* W, int64_t N, int64_t ld, int64_t blk, float2* W32) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * N) return;
    int64_t i = idx / N, j = idx % N;
    if (j <= i) {
        const float4 a = W[i * ld + j];
        W32[i * N + j] = df_to_f32(a);
        reinterpret_cast<double2*>(W)[i * ld + j] = df_to_f64(a);
    } else {
        W32[i * N + j] = make_float2(0.f, 0.f);
        if (j < (i / blk + 1) * blk) reinterpret_cast<double2*>(W)[i * ld + j] = make_double2(0.0, 0.0);
    }
}
cudaError_t launch_df_finish(float4* W, int64_t N, int64_t ld, int64_t blk, float2* W32, cudaStream_t s) {
    if (N == 0) return cudaSuccess;
    k_df_finish<<<nblk(N * N, 256), 256, 0, s>>>(W, N, ld, blk, W32);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_copy_lower(const double2* G, int64_t N, int64_t ld, double2* L) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * N) return;
    int64_t i = idx / N, j = idx % N;
    L[i * ld + j] = (j <= i) ? G[i * ld + j] : make_double2(0.0, 0.0);
}
cudaError_t launch_copy_lower(const double2* G, int64_t N, int64_t ld, double2* L, cudaStream_t s) {
    k_copy_lower<<<nblk(N * N, 256), 256, 0, s>>>(G, N, ld, L);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_copy_lower_df(const float4* G, int64_t N, int64_t ld, double2* L) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= N * N) return;
    int64_t i = idx / N, j = idx % N;
    L[i * ld + j] = (j <= i) ? df_to_f64(G[i * ld + j]) : make_double2(0.0, 0.0);
}
cudaError_t launch_copy_lower_df(const float4* G, int64_t N, int64_t ld, double2* L, cudaStream_t s) {
    k_copy_lower_df<<<nblk(N * N, 256), 256, 0, s>>>(G, N, ld, L);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_df_to_f64(const float4* a, int64_t n, double2* b) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) b[i] = df_to_f64(a[i]);
}
cudaError_t launch_df_to_f64(const float4* a, int64_t n, double2* b, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_df_to_f64<<<nblk(n, 256), 256, 0, s>>>(a, n, b);
    note_launch();
    return cudaGetLastError();
}

// min / max of the real diagonal of L (positive values: integer ordering of
// the IEEE bits matches numeric ordering, so atomicMin/Max on the bits works).
__global__ void k_pivot_stats(const double2* L, int64_t N, int64_t ld, DevStatus* st) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    double v = L[i * ld + i].x;
    if (!(v > 0.0)) return;
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    atomicMin((unsigned long long*)&st->min_pivot, b);
    atomicMax((unsigned long long*)&st->max_pivot, b);
}
cudaError_t launch_pivot_stats(const double2* L, int64_t N, int64_t ld, DevStatus* st,
                               cudaStream_t s) {
    k_pivot_stats<<<nblk(N, 256), 256, 0, s>>>(L, N, ld, st);
    note_launch();
    return cudaGetLastError();
}
__global__ void k_pivot_stats_df(const float4* L, int64_t N, int64_t ld, DevStatus* st) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const float4 d = L[i * ld + i];
    double v = join_f64(d.x, d.y);
    if (!(v > 0.0)) return;
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    atomicMin((unsigned long long*)&st->min_pivot, b);
    atomicMax((unsigned long long*)&st->max_pivot, b);
}
cudaError_t launch_pivot_stats_df(const float4* L, int64_t N, int64_t ld, DevStatus* st, cudaStream_t s) {
    k_pivot_stats_df<<<nblk(N, 256), 256, 0, s>>>(L, N, ld, st);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_frame_norms(const double2* X, int64_t n, double* out) {
    // one block per frame
    const double2* x = X + (int64_t)blockIdx.x * n;
    double acc = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += x[i].x * x[i].x + x[i].y * x[i].y;
    __shared__ double red[256];
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}
cudaError_t launch_frame_norms(const double2* X, int64_t F, int64_t n, double* out, cudaStream_t s) {
    if (F == 0) return cudaSuccess;
    k_frame_norms<<<(unsigned)F, 256, 0, s>>>(X, n, out);
    note_launch();
    return cudaGetLastError();
}

__global__ void k_zaxpy(double2* X, const double2* Y, int64_t n) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) X[i] = zadd(X[i], Y[i]);
}
cudaError_t launch_zaxpy(double2* X, const double2* Y, int64_t n, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_zaxpy<<<nblk(n, 256), 256, 0, s>>>(X, Y, n);
    note_launch();
    return cudaGetLastError();
}

}  // namespace pinv

namespace pinv {

// Tiled transpose through shared memory: dst[c][r] = src[r][c], zero padding for r in [rows, ldd).
__global__ void k_transpose32(const float2* __restrict__ src, int64_t rows, int64_t cols,
                              float2* __restrict__ dst, int64_t ldd) {
    __shared__ float2 t[32][33];
    const int64_t r0 = (int64_t)blockIdx.y * 32, c0 = (int64_t)blockIdx.x * 32;
    for (int dy = threadIdx.y; dy < 32; dy += 8) {
        const int64_t r = r0 + dy, c = c0 + threadIdx.x;
        t[dy][threadIdx.x] = (r < rows && c < cols) ? src[r * cols + c] : make_float2(0.f, 0.f);
    }
    __syncthreads();
    for (int dy = threadIdx.y; dy < 32; dy += 8) {
        const int64_t c = c0 + dy, r = r0 + threadIdx.x;
        if (c < cols && r < ldd) dst[c * ldd + r] = t[threadIdx.x][dy];
    }
}

cudaError_t launch_transpose32(const float2* src, int64_t rows, int64_t cols, float2* dst, int64_t ldd,
                               cudaStream_t s) {
    if (rows == 0 || cols == 0) return cudaSuccess;
    dim3 grid((unsigned)((cols + 31) / 32), (unsigned)((ldd + 31) / 32));
    k_transpose32<<<grid, dim3(32, 8), 0, s>>>(src, rows, cols, dst, ldd);
    note_launch();
    return cudaGetLastError();
}

// status word back to "no error" (a kernel, so that builds can be captured in graphs)
__global__ void k_reset_status(DevStatus* st, long long wait_limit) {
    st->not_pd_pivot = INT_MAX;
    st->timeout_site = 0;
    st->error_code = 0;
    st->pad = 0;
    st->min_pivot = INFINITY;
    st->max_pivot = 0.0;
    st->sched_next = 0;
    st->sched_done = 0;
    st->norm1_g = 0.0;
    st->kappa_est = 0.0;
    st->wait_limit = wait_limit;
}

cudaError_t launch_reset_status(DevStatus* st, cudaStream_t s) {
    k_reset_status<<<1, 1, 0, s>>>(st, wait_limit_setting());
    note_launch();
    return cudaGetLastError();
}

// a bounded wait that gave up on another stream's status block counts for the plan
__global__ void k_merge_timeout(DevStatus* dst, const DevStatus* src) {
    if (src->timeout_site) atomicMax(&dst->timeout_site, src->timeout_site);
}
cudaError_t launch_merge_timeout(DevStatus* dst, const DevStatus* src, cudaStream_t s) {
    k_merge_timeout<<<1, 1, 0, s>>>(dst, src);
    note_launch();
    return cudaGetLastError();
}

// dst[c][r] = src[r][c] for double-float tables, rows padded with zeros to ldd
__global__ void k_transpose_df(const float4* __restrict__ src, int64_t rows, int64_t cols, float4* __restrict__ dst,
                               int64_t ldd) {
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= cols * ldd) return;
    const int64_t c = idx / ldd, r = idx % ldd;
    dst[idx] = r < rows ? src[r * cols + c] : make_float4(0.f, 0.f, 0.f, 0.f);
}

cudaError_t launch_transpose_df(const float4* src, int64_t rows, int64_t cols, float4* dst, int64_t ldd,
                                cudaStream_t s) {
    const int64_t n = cols * ldd;
    if (n == 0) return cudaSuccess;
    k_transpose_df<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(src, rows, cols, dst, ldd);
    note_launch();
    return cudaGetLastError();
}

}  // namespace pinv
