// Split-BF16 complex contraction engine on the 5th-generation tensor cores.
//
// A CTA computes a 128 x 128 tile of a complex product C[i][j] = sum_k a(i,k) b(k,j).
//
// Real embedding. Each complex operand value is split into S bf16 slices
// (v = v0 + v1 [+ v2], each slice the bf16 rounding of what the previous ones
// left). Per 16-wide complex k chunk the A tile holds rows [Ar | Ai] and the B
// tile holds, for every output column j, the rows [Br | -Bi] (real output) and
// [Bi | Br] (imaginary output). One M = 128, N = 256, K = 16 MMA pair therefore
// produces Cr and Ci side by side:
//     Cr = Ar Br - Ai Bi,   Ci = Ar Bi + Ai Br,
// with 4 real MACs per complex MAC and no wasted products. Slice pairs kept:
// (0,0) (0,1) (1,0) for two slices; plus (0,2) (2,0) (1,1) for three.
//
// Accumulation. The tensor core's FP32 accumulation truncates (measured: a
// bias that grows linearly with the number of accumulation steps). The MMAs
// therefore accumulate at most DRAIN stages into a 256-column TMEM buffer; the
// producer warps then add the buffer into a running total held in the other
// 256 TMEM columns (tcgen05.ld, round-to-nearest FP32 add, tcgen05.st) while
// the MMA issuer waits. The relative bias stays near 3 * DRAIN * 2^-24
// regardless of K.
//
// Roles. 8 producer warps generate or load operand values (problem functors:
// row_a / row_b build a per-thread context once per tile, a8 / b8 then return
// 8 consecutive k for that row or column), split them and write
// the canonical K-major no-swizzle layout into a ring of shared-memory stages.
// One thread issues tcgen05.mma and commits stages back to the producers and
// full buffers to the drains. The producer warps also run the epilogue from
// the TMEM total. Every mbarrier wait is bounded by a clock64
// limit: on expiry the CTA raises an abort flag, stops, waits (bounded) for its
// issued MMAs, frees TMEM and records the failure in the plan's status word.
//
// Bulk-fed problems (kBulk = true) keep their operands in global memory already
// split and laid out as stage tiles (bulk_a: one 8 KiB A slice tile, bulk_b: one
// 16 KiB B slice tile). A tenth warp then loads each stage with asynchronous
// bulk copies (cp.async.bulk, completion counted in bytes on the stage's full
// barrier), and nothing passes through registers. The MMA accumulator is
// double-buffered (two 256-column halves of TMEM, group g in half g & 1), and
// the running total lives in the eight drain warps' registers, so the MMAs do
// not wait while a group is drained; the sums are the same (group sums added in
// order with round-to-nearest FP32 adds).
#pragma once

#include <cuda_bf16.h>

#include <type_traits>

#include "df.cuh"

namespace pinv {
namespace tc {

constexpr int BM = 128;          // complex rows per tile (MMA M)
constexpr int BN = 128;          // complex columns per tile (MMA N = 2 * BN)
constexpr int KC = 16;           // complex k per stage
constexpr int NPW = 8;           // producer / drain / epilogue warps
constexpr int NTHREADS = (NPW + 1) * 32;
constexpr int DRAIN = 8;         // stages per TMEM accumulation group
constexpr long long WAIT_LIMIT = 4000000000LL;  // clock64 cycles, about 2 s

constexpr int ROWB = 2 * KC * 2;                 // bytes per embedded row: K' = 32 bf16
constexpr int A_SL = BM * ROWB;                  // 8 KiB
constexpr int B_SL = 2 * BN * ROWB;              // 16 KiB
constexpr int SLICE = A_SL + B_SL;               // 24 KiB per slice per stage

template <int S>
struct Cfg {
    static constexpr int STAGES = S == 3 ? 3 : 4;
    static constexpr int STAGE_BYTES = S * SLICE;
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024;
    static constexpr int NPAIRS = S == 3 ? 6 : 3;
};
static_assert(DRAIN >= 4, "drain group must outlast the stage ring");

// instruction descriptor, kind::f16: D f32, A/B bf16, K-major, N = 256, M = 128
constexpr uint32_t IDESC =
    (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)((2 * BN) >> 3) << 17) | ((uint32_t)(BM >> 4) << 24);

// problems that declare `static constexpr bool kBulk = true` are bulk-fed
template <class P, class = void>
struct IsBulk : std::false_type {};
template <class P>
struct IsBulk<P, std::void_t<decltype(P::kBulk)>> : std::integral_constant<bool, P::kBulk> {};

// ... a bulk problem may write its results 16 columns at a time (store16) and
// ask for its B tiles to be kept in L2 (kHintB)
template <class P, class = void>
struct HasStore16 : std::false_type {};
template <class P>
struct HasStore16<P, std::void_t<decltype(&P::store16)>> : std::true_type {};
// ... or through a row-major copy of the tile in shared memory (store4: a warp
// then writes whole rows, lane l columns j0 + l + 32 u, u = 0..3, so that each
// access of the warp covers 32 consecutive entries)
template <class P, class = void>
struct HasStore4 : std::false_type {};
template <class P>
struct HasStore4<P, std::void_t<decltype(&P::store4)>> : std::true_type {};
// ... or subtract the tile from a double-float matrix (rmw_ptr(i, j): the entry
// to update, or null): each warp then has several rows' entries in flight at
// once, copied into the idle stage ring (cp.async), and the updates are FP32
// arithmetic (df_sub_f32)
template <class P, class = void>
struct HasRmw : std::false_type {};
template <class P>
struct HasRmw<P, std::void_t<decltype(&P::rmw_ptr)>> : std::true_type {};
// ... and name the entries it will read (prefetch: brought into L2 while the
// tile's MMAs run)
template <class P, class = void>
struct HasPrefetch : std::false_type {};
template <class P>
struct HasPrefetch<P, std::void_t<decltype(&P::prefetch)>> : std::true_type {};
template <class P, class = void>
struct HintB : std::false_type {};
template <class P>
struct HintB<P, std::void_t<decltype(P::kHintB)>> : std::integral_constant<bool, P::kHintB> {};

// ... a generating problem whose operands stream from HBM (kPrefetch) has its
// producers load the next two stages into registers while splitting this one
template <class P, class = void>
struct Prefetch : std::false_type {};
template <class P>
struct Prefetch<P, std::void_t<decltype(P::kPrefetch)>> : std::integral_constant<bool, P::kPrefetch> {};

constexpr int NTHREADS_BULK = NTHREADS + 32;  // + one loader warp

// slice pairs in decreasing weight: (0,0) (0,1) (1,0) (0,2) (2,0) (1,1)
__host__ __device__ constexpr int pair_a(int q) { return q == 2 ? 1 : q == 4 ? 2 : q == 5 ? 1 : 0; }
__host__ __device__ constexpr int pair_b(int q) { return q == 1 ? 1 : q == 3 ? 2 : q == 5 ? 1 : 0; }

// ------------------------------------------------------------------ PTX helpers
__device__ inline uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ inline void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ inline void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ inline bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: false if the limit expired or another role raised abort. Pipeline
// waits pass the kernel's runtime limit (DevStatus::wait_limit); the waits of the
// clean-up (every issued MMA finished before TMEM is freed, copies in flight
// landed) pass no abort flag and keep WAIT_LIMIT whatever the setting.
__device__ inline bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag,
                                 long long limit = WAIT_LIMIT) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (abort_flag && *abort_flag) return false;
        if (clock64() - t0 > limit) {
            if (abort_flag) *abort_flag = 1;
            return false;
        }
    }
}
__device__ inline void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// barrier among the first `threads` threads of the CTA (id 1; id 0 is __syncthreads)
__device__ inline void named_barrier(uint32_t threads) {
    asm volatile("bar.sync 1, %0;" ::"r"(threads) : "memory");
}
// ... that also returns the OR of v over those threads (the same value in all of them)
__device__ inline bool named_barrier_or(uint32_t threads, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.or.pred q, 1, %2, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(threads)
        : "memory");
    return r != 0;
}
__device__ inline void fence_barrier_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
__device__ inline void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ inline void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// expect `bytes` of asynchronous copies on this phase, with this thread's arrival
__device__ inline void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}
// expect `bytes` of asynchronous copies on the current phase, without arriving
__device__ inline void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.expect_tx.relaxed.cta.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
// global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16),
// completing `bytes` on the mbarrier
__device__ inline void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}
// ... with an L2 eviction-priority policy (createpolicy)
__device__ inline void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes, uint64_t* bar, uint64_t pol) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], "
        "%4;" ::"r"(smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
        : "memory");
}
// 16-byte global -> shared copy through L2 (cp.async), and the wait for all of this thread's
__device__ inline void cp_async16(void* dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ inline void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }
// global -> L2 bulk prefetch (16-byte aligned address, size a multiple of 16); a hint, no completion
__device__ inline void bulk_prefetch_l2(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ inline uint64_t policy_evict_last() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

__device__ inline void tmem_alloc(uint32_t* dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ inline void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// shared-memory matrix descriptor: canonical K-major layout without swizzle
__device__ inline uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version for tcgen05
    return d;                // base offset 0, layout type 0 (no swizzle)
}

__device__ inline void mma_bf16(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ inline void mma_commit(uint64_t* bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

__device__ inline void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
}
__device__ inline void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// byte offset of (row r, 8-wide k' group g in 0..3) in a [R][32] K-major no-swizzle tile
__device__ inline uint32_t koff(int r, int g) { return (uint32_t)((r >> 3) * 512 + g * 128 + (r & 7) * 16); }

// split 8 floats into S bf16 slices, packed 2 per word: w[s][0..3]
template <int S>
__device__ inline void split8(float (&x)[8], uint32_t (&w)[S][4]) {
#pragma unroll
    for (int s = 0; s < S; ++s) {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * t], x[2 * t + 1]);
            if (s + 1 < S) {
                const float2 back = __bfloat1622float2(h);
                x[2 * t] -= back.x;
                x[2 * t + 1] -= back.y;
            }
            w[s][t] = *reinterpret_cast<uint32_t*>(&h);
        }
    }
}

template <int S>
__device__ inline void store_slices(uint8_t* p, const uint32_t (&w)[S][4], uint32_t flip) {
#pragma unroll
    for (int s = 0; s < S; ++s)
        *reinterpret_cast<uint4*>(p + s * SLICE) =
            make_uint4(w[s][0] ^ flip, w[s][1] ^ flip, w[s][2] ^ flip, w[s][3] ^ flip);
}

__device__ inline void tmem_st16(uint32_t taddr, const uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(taddr),
        "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8]),
        "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
        : "memory");
}
__device__ inline void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

constexpr uint32_t TOTAL_COL = 2 * BN;  // running total after the MMA buffer

// Add this warp's part of the MMA buffer (32 rows x 64 complex columns: real
// parts at col0, imaginary at col0 + BN) into the running total.
__device__ inline void drain_to_total(uint32_t taddr_row, bool first) {
#pragma unroll
    for (int part = 0; part < 8; ++part) {
        const uint32_t col = (uint32_t)((part & 4) ? BN : 0) + 16u * (part & 3);
        uint32_t b[16], t[16];
        tmem_ld16(taddr_row + col, b);
        if (!first) tmem_ld16(taddr_row + TOTAL_COL + col, t);
        tmem_wait_ld();
        if (!first) {
#pragma unroll
            for (int i = 0; i < 16; ++i) b[i] = __float_as_uint(__uint_as_float(b[i]) + __uint_as_float(t[i]));
        }
        tmem_st16(taddr_row + TOTAL_COL + col, b);
    }
    tmem_wait_st();
}

// Bulk mode: add (or, for a tile's first group, copy) this warp's part of an
// MMA buffer into the running total in registers: tot[0..63] real parts of the
// warp's 64 columns, tot[64..127] imaginary parts.
__device__ inline void drain_to_regs(uint32_t taddr_buf, float (&tot)[128], bool first) {
#pragma unroll
    for (int part = 0; part < 8; ++part) {
        uint32_t b[16];
        tmem_ld16(taddr_buf + (uint32_t)((part & 4) ? BN : 0) + 16u * (part & 3), b);
        tmem_wait_ld();
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            float& t = tot[16 * part + i];
            t = first ? __uint_as_float(b[i]) : t + __uint_as_float(b[i]);
        }
    }
}

// ... and write the totals back to TMEM (the same columns of a free buffer) for the epilogue
__device__ inline void regs_to_tmem(uint32_t taddr_buf, const float (&tot)[128]) {
#pragma unroll
    for (int part = 0; part < 8; ++part) {
        uint32_t b[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) b[i] = __float_as_uint(tot[16 * part + i]);
        tmem_st16(taddr_buf + (uint32_t)((part & 4) ? BN : 0) + 16u * (part & 3), b);
    }
    tmem_wait_st();
}

// Tile schedulers of the persistent kernel: item t -> (problem, bx, by).
// OneProblem covers a gx x gy grid of tiles of one problem; ManyProblems
// concatenates the tile grids of several problems (e.g. one per plan of a
// batch) held in device memory.
// rev: hand out items last to first (the longest tiles of a triangular
// operand first, so they do not form the tail).
template <class P>
struct OneProblem {
    using Prob = P;
    P p;
    int64_t gx, n;
    bool rev;
    __device__ int64_t count() const { return n; }
    __device__ const P& get(int64_t t, int64_t& bx, int64_t& by) const {
        if (rev) t = n - 1 - t;
        bx = t % gx;
        by = t / gx;
        return p;
    }
};

template <class P>
struct ManyProblems {
    using Prob = P;
    const P* probs;         // [n]
    const int64_t* start;   // [n + 1], first item of each problem
    const int64_t* gx;      // [n], tile-grid width of each problem
    int n;
    bool rev;
    __device__ int64_t count() const { return start[n]; }
    __device__ const P& get(int64_t t, int64_t& bx, int64_t& by) const {
        if (rev) {  // last tile of each problem first, problems in order
            int i = 0;
            while (i + 1 < n && start[i + 1] <= t) ++i;
            t = start[i] + (start[i + 1] - 1 - t);
        }
        int i = 0;
        while (i + 1 < n && start[i + 1] <= t) ++i;
        const int64_t l = t - start[i];
        bx = l % gx[i];
        by = l / gx[i];
        return probs[i];
    }
};

// Persistent kernel: each CTA takes the next item from a global counter (in
// the plan's status block) until none is left, so uneven tiles balance across
// SMs. The stage ring and the TMEM accumulation groups run on counters that
// continue across tiles, so barriers are initialised and TMEM allocated once
// per CTA. The last CTA to finish zeroes the item counter for the next launch
// on the same stream.
template <int S, class Sched>
__global__ void __launch_bounds__(NTHREADS, 1) k_tc(Sched sch, DevStatus* st, int site) {
    using CF = Cfg<S>;
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t full_bar[CF::STAGES], empty_bar[CF::STAGES];
    __shared__ uint64_t tfull, tempty, done_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_flag;
    __shared__ long long next_item;

    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    griddep_wait();  // launched behind the previous kernel of the stream: its writes and tile counter
    const long long wlim = st->wait_limit > 0 ? st->wait_limit : WAIT_LIMIT;  // pipeline waits

    if (threadIdx.x == 0) {
        for (int s = 0; s < CF::STAGES; ++s) {
            mbar_init(&full_bar[s], NPW * 32);
            mbar_init(&empty_bar[s], 1);
        }
        mbar_init(&tfull, 1);
        mbar_init(&tempty, NPW * 32);
        mbar_init(&done_bar, 1);
        abort_flag = 0;
        next_item = (long long)atomicAdd(&st->sched_next, 1ull);
        fence_barrier_init();
    }
    if (warp == NPW) tmem_alloc(&tmem_base_sh, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;
    const int q = warp & 3, h = warp >> 2;
    const uint32_t taddr_row = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(64 * h);

    const int64_t items = sch.count();
    uint32_t kq = 0, gq = 0;  // stages and accumulation groups used by earlier tiles
    for (int64_t t = next_item;; ) {
        if (t >= items) break;
        int64_t bx, by;
        const auto& p = sch.get(t, bx, by);
        int64_t i0, j0, kb, ke;
        if (!p.tile(bx, by, i0, j0, kb, ke)) {  // empty tile (uniform per CTA)
            __syncthreads();
            if (threadIdx.x == 0) next_item = (long long)atomicAdd(&st->sched_next, 1ull);
            __syncthreads();
            t = next_item;
            continue;
        }
        const int nk = ke > kb ? (int)((ke - kb + KC - 1) / KC) : 0;
        const int ngroups = (nk + DRAIN - 1) / DRAIN;

        if (warp < NPW) {
            // ---------------- producers, drains, epilogue
            int drained = 0;
            bool ok = true;
            auto drain = [&](int g) -> bool {
                if (!mbar_wait(&tfull, (gq + (uint32_t)g) & 1u, &abort_flag, wlim)) return false;
                tc_fence_after();
                drain_to_total(taddr_row, g == 0);
                tc_fence_before();
                mbar_arrive(&tempty);
                return true;
            };
            const int ua = threadIdx.x;  // A unit: row ua & 127, k group ua >> 7
            const int ubr = threadIdx.x & (BN - 1), ubg = threadIdx.x >> 7;
            // per-thread operand contexts (row pointers, table rows) fixed for the tile
            const auto ra = p.row_a(i0 + (ua & (BM - 1)));
            const auto rb = p.row_b(j0 + ubr);
            constexpr bool PF = Prefetch<typename Sched::Prob>::value;
            float2 pa1[8], pb1[8], pa2[8], pb2[8];  // stages kt + 1, kt + 2 (kPrefetch)
            if constexpr (PF) {
                p.a8(ra, kb + 8 * (ua >> 7), ke, pa1);
                p.b8(rb, kb + 8 * ubg, ke, pb1);
                p.a8(ra, kb + KC + 8 * (ua >> 7), ke, pa2);
                p.b8(rb, kb + KC + 8 * ubg, ke, pb2);
            }
            for (int kt = 0; kt < nk && ok; ++kt) {
                // the MMA cannot start group g + 1 until group g is drained; drain it
                // before the ring can only advance past that point
                while (drained < ngroups && (drained + 1) * DRAIN + CF::STAGES - 1 <= kt) {
                    if (!(ok = drain(drained))) break;
                    ++drained;
                }
                if (!ok) break;
                const uint32_t kg = kq + (uint32_t)kt;
                const int s = (int)(kg % CF::STAGES);
                const uint32_t ph = (kg / CF::STAGES) & 1u;
                if (kg >= CF::STAGES && !(ok = mbar_wait(&empty_bar[s], ph ^ 1u, &abort_flag, wlim))) break;
                uint8_t* base = smem + s * CF::STAGE_BYTES;
                const int64_t k0 = kb + (int64_t)kt * KC;
                float2 va[8], vb[8];
                if constexpr (PF) {
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        va[u] = pa1[u];
                        vb[u] = pb1[u];
                        pa1[u] = pa2[u];
                        pb1[u] = pb2[u];
                    }
                    p.a8(ra, k0 + 2 * KC + 8 * (ua >> 7), ke, pa2);  // zeros past ke
                    p.b8(rb, k0 + 2 * KC + 8 * ubg, ke, pb2);
                } else {
                    p.a8(ra, k0 + 8 * (ua >> 7), ke, va);
                    p.b8(rb, k0 + 8 * ubg, ke, vb);
                }
                {
                    const float2(&v)[8] = va;
                    const int r = ua & (BM - 1), g = ua >> 7;
                    float re[8], im[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) { re[u] = v[u].x; im[u] = v[u].y; }
                    uint32_t wr[S][4], wi[S][4];
                    split8<S>(re, wr);
                    split8<S>(im, wi);
                    store_slices<S>(base + koff(r, g), wr, 0u);
                    store_slices<S>(base + koff(r, g + 2), wi, 0u);
                }
                {
                    const float2(&v)[8] = vb;
                    float re[8], im[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) { re[u] = v[u].x; im[u] = v[u].y; }
                    uint32_t wr[S][4], wi[S][4];
                    split8<S>(re, wr);
                    split8<S>(im, wi);
                    uint8_t* bb = base + A_SL;
                    store_slices<S>(bb + koff(ubr, ubg), wr, 0u);                 // [Br | -Bi]
                    store_slices<S>(bb + koff(ubr, ubg + 2), wi, 0x80008000u);
                    store_slices<S>(bb + koff(BN + ubr, ubg), wi, 0u);            // [Bi |  Br]
                    store_slices<S>(bb + koff(BN + ubr, ubg + 2), wr, 0u);
                }
                fence_proxy_async();
                mbar_arrive(&full_bar[s]);
            }
            while (ok && drained < ngroups) {
                ok = drain(drained);
                ++drained;
            }
            if (ok && !abort_flag) {
                tc_fence_after();
                const int64_t gi = i0 + q * 32 + lane;
#pragma unroll 1
                for (int part = 0; part < 4; ++part) {
                    uint32_t cr[16], ci[16];
                    if (nk > 0) {
                        tmem_ld16(taddr_row + TOTAL_COL + 16 * part, cr);
                        tmem_ld16(taddr_row + TOTAL_COL + BN + 16 * part, ci);
                        tmem_wait_ld();
                    } else {
#pragma unroll
                        for (int u = 0; u < 16; ++u) cr[u] = ci[u] = 0u;
                    }
                    if (p.row_ok(gi)) {
#pragma unroll
                        for (int u = 0; u < 16; ++u) {
                            const int64_t gj = j0 + 64 * h + 16 * part + u;
                            if (p.col_ok(gj))
                                p.store(gi, gj, make_float2(__uint_as_float(cr[u]), __uint_as_float(ci[u])));
                        }
                    }
                }
            }
        } else if (lane == 0) {
            // ---------------- MMA issuer
            for (int kt = 0; kt < nk; ++kt) {
                const uint32_t g = gq + (uint32_t)(kt / DRAIN);
                const bool first = (kt % DRAIN) == 0;
                if (first && g >= 1 && !mbar_wait(&tempty, (g - 1) & 1u, &abort_flag, wlim)) break;
                const uint32_t kg = kq + (uint32_t)kt;
                const int s = (int)(kg % CF::STAGES);
                const uint32_t ph = (kg / CF::STAGES) & 1u;
                if (!mbar_wait(&full_bar[s], ph, &abort_flag, wlim)) break;
                tc_fence_after();
                const uint32_t sbase = smem_u32(smem + s * CF::STAGE_BYTES);
#pragma unroll
                for (int pq = 0; pq < CF::NPAIRS; ++pq) {
                    const uint32_t a = sbase + pair_a(pq) * SLICE;
                    const uint32_t bsl = sbase + pair_b(pq) * SLICE + A_SL;
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        const uint64_t da = sdesc(a + kk * 256, 128, 512);
                        const uint64_t db = sdesc(bsl + kk * 256, 128, 512);
                        mma_bf16(tmem, da, db, IDESC, (first && pq == 0 && kk == 0) ? 0u : 1u);
                    }
                }
                mma_commit(&empty_bar[s]);
                if ((kt % DRAIN) == DRAIN - 1 || kt == nk - 1) mma_commit(&tfull);
            }
        }
        kq += (uint32_t)nk;
        gq += (uint32_t)ngroups;
        // next item: every thread has read next_item for this tile
        __syncthreads();
        if (threadIdx.x == 0) next_item = abort_flag ? (long long)items : (long long)atomicAdd(&st->sched_next, 1ull);
        __syncthreads();
        t = next_item;
    }
    if (warp == NPW && lane == 0) mma_commit(&done_bar);  // completes when every issued MMA has finished

    tc_fence_before();
    __syncthreads();
    if (warp == NPW) {
        mbar_wait(&done_bar, 0, nullptr);  // no MMA may still write TMEM when it is released
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
    if (threadIdx.x == 0) {
        if (abort_flag) atomicMax(&st->timeout_site, site);
        // the last CTA out resets the item counter: all others have stopped taking items
        __threadfence();
        if (atomicAdd(&st->sched_done, 1ull) == (unsigned long long)gridDim.x - 1) {
            st->sched_next = 0;
            st->sched_done = 0;
            __threadfence();
        }
    }
}

// Persistent kernel for bulk-fed problems. Warps 0-7 drain the MMA buffers into
// register totals and run the epilogue, warp 8 issues the MMAs, warp 9 loads
// the stages. Item scheduling, the stage ring and the bounded waits follow k_tc.
template <int S, class Sched>
__global__ void __launch_bounds__(NTHREADS_BULK, 1) k_tc_bulk(Sched sch, DevStatus* st, int site) {
    using CF = Cfg<S>;
    constexpr uint32_t STAGE_TX = (uint32_t)CF::STAGE_BYTES;
    extern __shared__ uint8_t smem_raw[];
    __shared__ uint64_t full_bar[CF::STAGES], empty_bar[CF::STAGES];
    __shared__ uint64_t tfull[2], tempty[2], done_bar;
    __shared__ uint32_t tmem_base_sh;
    __shared__ int abort_flag;
    __shared__ long long next_item;

    uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    griddep_wait();  // launched behind the previous kernel of the stream: its writes and tile counter
    const long long wlim = st->wait_limit > 0 ? st->wait_limit : WAIT_LIMIT;  // pipeline waits

    if (threadIdx.x == 0) {
        for (int s = 0; s < CF::STAGES; ++s) {
            mbar_init(&full_bar[s], 1);  // the loader's arrival plus the stage's bytes
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull[b], 1);
            mbar_init(&tempty[b], NPW * 32);
        }
        mbar_init(&done_bar, 1);
        abort_flag = 0;
        next_item = (long long)atomicAdd(&st->sched_next, 1ull);
        fence_barrier_init();
    }
    if (warp == NPW) tmem_alloc(&tmem_base_sh, 512);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base_sh;
    const int q = warp & 3, h = (warp >> 2) & 1;
    const uint32_t taddr_row = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(64 * h);

    const int64_t items = sch.count();
    uint32_t kq = 0, gq = 0;  // stages and accumulation groups used by earlier tiles
    uint32_t issued = 0;      // stages the loader has started
    for (int64_t t = next_item;;) {
        if (t >= items) break;
        int64_t bx, by;
        const auto& p = sch.get(t, bx, by);
        int64_t i0, j0, kb, ke;
        if (!p.tile(bx, by, i0, j0, kb, ke)) {
            __syncthreads();
            if (threadIdx.x == 0) next_item = (long long)atomicAdd(&st->sched_next, 1ull);
            __syncthreads();
            t = next_item;
            continue;
        }
        const int nk = ke > kb ? (int)((ke - kb + KC - 1) / KC) : 0;
        const int ngroups = (nk + DRAIN - 1) / DRAIN;

        if (warp < NPW) {
            // ---------------- drains and epilogue
            using PE = std::remove_cv_t<std::remove_reference_t<decltype(p)>>;
            if constexpr (HasPrefetch<PE>::value) p.prefetch(i0 + q * 32 + lane, j0 + 64 * h, 64);
            float tot[128];
#pragma unroll
            for (int u = 0; u < 128; ++u) tot[u] = 0.f;
            bool ok = true;
            for (int g = 0; g < ngroups; ++g) {
                const uint32_t G = gq + (uint32_t)g, b = G & 1u;
                if (!(ok = mbar_wait(&tfull[b], (G >> 1) & 1u, &abort_flag, wlim))) break;
                tc_fence_after();
                drain_to_regs(taddr_row + 2u * BN * b, tot, g == 0);
                tc_fence_before();
                mbar_arrive(&tempty[b]);
            }
            if constexpr (HasStore4<PE>::value || HasRmw<PE>::value) {
                // Every stage of the tile has been consumed and the loader waits for the
                // tile barrier, so the stage ring holds a row-major copy of the tile
                // (rows padded by 16 bytes: conflict-free float4 writes); each warp
                // then updates whole rows. Every drain thread reaches the barriers; the
                // OR makes the decision to write the same in all of them.
                if (!named_barrier_or(NPW * 32, !ok || abort_flag)) {
                    constexpr int SP = BN + 2;
                    float2* Rt = reinterpret_cast<float2*>(smem);
                    const int r = q * 32 + lane;
#pragma unroll
                    for (int u = 0; u < 64; u += 2)
                        *reinterpret_cast<float4*>(&Rt[r * SP + 64 * h + u]) =
                            make_float4(tot[u], tot[64 + u], tot[u + 1], tot[64 + u + 1]);
                    named_barrier(NPW * 32);
                    if constexpr (HasRmw<PE>::value) {
                        // RE rows per warp at a time: their entries are copied into the
                        // ring behind the tile (cp.async, no registers held), then each
                        // lane updates the entries it copied (lane l: columns l + 32 u)
                        constexpr int TB = BM * SP * (int)sizeof(float2);
                        constexpr int RE = TB + NPW * 4 * BN * 16 <= CF::STAGES * CF::STAGE_BYTES ? 4 : 2;
                        static_assert(TB + NPW * RE * BN * 16 <= CF::STAGES * CF::STAGE_BYTES, "staging");
                        float4* stg = reinterpret_cast<float4*>(smem + TB) + warp * RE * BN;
                        for (int r0 = warp; r0 < BM; r0 += NPW * RE) {
#pragma unroll
                            for (int r = 0; r < RE; ++r)
#pragma unroll
                                for (int u = 0; u < 4; ++u) {
                                    const float4* g = p.rmw_ptr(i0 + r0 + r * NPW, j0 + lane + 32 * u);
                                    if (g) cp_async16(stg + r * BN + lane + 32 * u, g);
                                }
                            cp_async_wait_all();
#pragma unroll
                            for (int r = 0; r < RE; ++r)
#pragma unroll
                                for (int u = 0; u < 4; ++u) {
                                    float4* g = p.rmw_ptr(i0 + r0 + r * NPW, j0 + lane + 32 * u);
                                    if (g)
                                        *g = df_sub_f32(stg[r * BN + lane + 32 * u],
                                                        Rt[(r0 + r * NPW) * SP + lane + 32 * u]);
                                }
                        }
                    } else {
                        for (int rr = warp; rr < BM; rr += NPW) {
                            const float2 v[4] = {Rt[rr * SP + lane], Rt[rr * SP + lane + 32], Rt[rr * SP + lane + 64],
                                                 Rt[rr * SP + lane + 96]};
                            p.store4(i0 + rr, j0 + lane, v);
                        }
                    }
                    fence_proxy_async();  // generic shared accesses before the next tile's copies
                }
            } else if (ok && !abort_flag) {
                // every group is drained and the MMAs of the next tile wait for the
                // tile barrier, so buffer 0 is free to hold the totals
                regs_to_tmem(taddr_row, tot);
                const int64_t gi = i0 + q * 32 + lane;
#pragma unroll 1
                for (int part = 0; part < 4; ++part) {
                    uint32_t cr[16], ci[16];
                    tmem_ld16(taddr_row + 16 * part, cr);
                    tmem_ld16(taddr_row + BN + 16 * part, ci);
                    tmem_wait_ld();
                    if constexpr (HasStore16<std::remove_cv_t<std::remove_reference_t<decltype(p)>>>::value) {
                        float re[16], im[16];
#pragma unroll
                        for (int u = 0; u < 16; ++u) {
                            re[u] = __uint_as_float(cr[u]);
                            im[u] = __uint_as_float(ci[u]);
                        }
                        p.store16(gi, j0 + 64 * h + 16 * part, re, im);
                    } else if (p.row_ok(gi)) {
#pragma unroll
                        for (int u = 0; u < 16; ++u) {
                            const int64_t gj = j0 + 64 * h + 16 * part + u;
                            if (p.col_ok(gj))
                                p.store(gi, gj, make_float2(__uint_as_float(cr[u]), __uint_as_float(ci[u])));
                        }
                    }
                }
                tc_fence_before();
            }
        } else if (warp == NPW && lane == 0) {
            // ---------------- MMA issuer
            for (int kt = 0; kt < nk; ++kt) {
                const uint32_t G = gq + (uint32_t)(kt / DRAIN), b = G & 1u;
                const bool first = (kt % DRAIN) == 0;
                // buffer b was last used by group G - 2: it must be drained
                if (first && G >= 2 && !mbar_wait(&tempty[b], ((G >> 1) - 1u) & 1u, &abort_flag, wlim)) break;
                const uint32_t kg = kq + (uint32_t)kt;
                const int s = (int)(kg % CF::STAGES);
                const uint32_t ph = (kg / CF::STAGES) & 1u;
                if (!mbar_wait(&full_bar[s], ph, &abort_flag, wlim)) break;
                tc_fence_after();
                const uint32_t sbase = smem_u32(smem + s * CF::STAGE_BYTES);
                const uint32_t dcol = tmem + 2u * BN * b;
#pragma unroll
                for (int pq = 0; pq < CF::NPAIRS; ++pq) {
                    const uint32_t a = sbase + pair_a(pq) * SLICE;
                    const uint32_t bsl = sbase + pair_b(pq) * SLICE + A_SL;
#pragma unroll
                    for (int kk = 0; kk < 2; ++kk) {
                        const uint64_t da = sdesc(a + kk * 256, 128, 512);
                        const uint64_t db = sdesc(bsl + kk * 256, 128, 512);
                        mma_bf16(dcol, da, db, IDESC, (first && pq == 0 && kk == 0) ? 0u : 1u);
                    }
                }
                mma_commit(&empty_bar[s]);
                if ((kt % DRAIN) == DRAIN - 1 || kt == nk - 1) mma_commit(&tfull[b]);
            }
        } else if (warp == NPW + 1 && lane == 0) {
            // ---------------- loader
            using PT = std::remove_cv_t<std::remove_reference_t<decltype(p)>>;
            const uint64_t pol = HintB<PT>::value ? policy_evict_last() : 0ull;
            const int64_t kc0 = kb / KC;
            for (int kt = 0; kt < nk; ++kt) {
                const uint32_t kg = kq + (uint32_t)kt;
                const int s = (int)(kg % CF::STAGES);
                const uint32_t ph = (kg / CF::STAGES) & 1u;
                if (kg >= CF::STAGES && !mbar_wait(&empty_bar[s], ph ^ 1u, &abort_flag, wlim)) break;
                uint8_t* base = smem + s * CF::STAGE_BYTES;
                mbar_arrive_expect_tx(&full_bar[s], STAGE_TX);
#pragma unroll
                for (int sl = 0; sl < S; ++sl) {
                    bulk_g2s(base + sl * SLICE, p.bulk_a(i0, kc0 + kt, sl), A_SL, &full_bar[s]);
                    if constexpr (HintB<PT>::value)
                        bulk_g2s_hint(base + sl * SLICE + A_SL, p.bulk_b(j0, kc0 + kt, sl), B_SL, &full_bar[s], pol);
                    else
                        bulk_g2s(base + sl * SLICE + A_SL, p.bulk_b(j0, kc0 + kt, sl), B_SL, &full_bar[s]);
                }
                issued = kg + 1;
            }
        }
        kq += (uint32_t)nk;
        gq += (uint32_t)ngroups;
        __syncthreads();
        if (threadIdx.x == 0) next_item = abort_flag ? (long long)items : (long long)atomicAdd(&st->sched_next, 1ull);
        __syncthreads();
        t = next_item;
    }
    if (warp == NPW && lane == 0) mma_commit(&done_bar);
    if (warp == NPW + 1 && lane == 0) {
        // copies still in flight (only after an abort): wait, bounded, for their bytes
        for (uint32_t kg = issued > (uint32_t)CF::STAGES ? issued - CF::STAGES : 0u; kg < issued; ++kg)
            mbar_wait(&full_bar[kg % CF::STAGES], (kg / CF::STAGES) & 1u, nullptr);
    }

    tc_fence_before();
    __syncthreads();
    if (warp == NPW) {
        mbar_wait(&done_bar, 0, nullptr);
        tc_fence_after();
        tmem_dealloc(tmem, 512);
    }
    if (threadIdx.x == 0) {
        if (abort_flag) atomicMax(&st->timeout_site, site);
        __threadfence();
        if (atomicAdd(&st->sched_done, 1ull) == (unsigned long long)gridDim.x - 1) {
            st->sched_next = 0;
            st->sched_done = 0;
            __threadfence();
        }
    }
}

int sm_count();

// How many parts to split a k range of `len` into, for launches that run `per_split`
// tiles (one CTA each, one CTA per SM) per part: the count in [lo, hi] that minimises
// waves x (len / parts + overhead), `overhead` standing for each tile's fill,
// drain and epilogue in units of k; the fewest parts on a tie. Whole waves matter:
// 320 tiles on 152 SMs take three waves, the third a tenth full.
inline int wave_splits(int64_t per_split, int64_t len, int lo, int hi, int64_t overhead) {
    const int64_t sms = sm_count();
    int best = lo;
    double bt = 0.0;
    for (int sp = lo; sp <= hi; ++sp) {
        const int64_t waves = (per_split * sp + sms - 1) / sms;
        const double t = (double)waves * ((double)len / sp + (double)overhead);
        if (sp == lo || t < bt * (1.0 - 1e-9)) {
            bt = t;
            best = sp;
        }
    }
    return best;
}

template <class K, class... A>
static cudaError_t launch_persistent(K kern, int threads, int smem, bool& attr, int64_t items, int cap, bool pdl,
                                     cudaStream_t s, const A&... args) {
    if (!attr) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    if (items == 0) return cudaSuccess;
    const int64_t limit = cap > 0 && cap < sm_count() ? cap : sm_count();
    const int64_t ctas = items < limit ? items : limit;
    if (pdl) {
        cudaError_t e = launch_pdl(kern, dim3((unsigned)ctas), dim3(threads), (size_t)smem, s, args...);
        return e != cudaSuccess ? e : cudaGetLastError();
    }
    kern<<<(unsigned)ctas, threads, smem, s>>>(args...);
    note_launch();
    return cudaGetLastError();
}

// cap > 0: at most cap CTAs (SMs), leaving the others to concurrent work; pdl:
// programmatic dependent launch after the previous kernel of the stream
template <int S, class Sched>
static cudaError_t launch_sched(const Sched& sch, int64_t items, DevStatus* st, int site, cudaStream_t s,
                                int cap = 0, bool pdl = false) {
    static bool attr = false;
    if constexpr (IsBulk<typename Sched::Prob>::value)
        return launch_persistent(k_tc_bulk<S, Sched>, NTHREADS_BULK, Cfg<S>::SMEM, attr, items, cap, pdl, s, sch,
                                 st, site);
    else
        return launch_persistent(k_tc<S, Sched>, NTHREADS, Cfg<S>::SMEM, attr, items, cap, pdl, s, sch, st, site);
}

// One problem over a grid.x x grid.y grid of tiles (bx = x, by = y). Launches
// sharing a status block must run one after another (one stream).
template <int S, class P>
static cudaError_t launch(const P& p, dim3 grid, DevStatus* st, int site, cudaStream_t s, bool rev = false,
                          int cap = 0, bool pdl = false) {
    const int64_t n = (int64_t)grid.x * grid.y;
    return launch_sched<S>(OneProblem<P>{p, (int64_t)grid.x, n, rev}, n, st, site, s, cap, pdl);
}

// Several problems of one kind in one persistent launch; the arrays live in
// device memory (filled by the caller), items = start[n].
template <int S, class P>
static cudaError_t launch_many(const P* probs, const int64_t* start, const int64_t* gx, int n, int64_t items,
                               DevStatus* st, int site, cudaStream_t s, bool rev = false) {
    return launch_sched<S>(ManyProblems<P>{probs, start, gx, n, rev}, items, st, site, s);
}

}  // namespace tc
}  // namespace pinv
