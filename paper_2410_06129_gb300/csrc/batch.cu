// Batched build and apply of several plans of uneven size.
//
// A batch groups existing plans (many slices, time series or trajectories).
// Its build runs the dominant tensor-core work of all plans as shared
// persistent launches: one launch forms every plan's Gram, and per chunk of
// samples one launch forms every plan's T = W E^H and one every plan's
// Recon = W^H T (all bulk-fed from per-plan operand tables); the sequential
// Cholesky and triangular inverse of each plan run concurrently on per-plan
// streams between them. Its apply runs every plan's apply (Recon x data plus
// refinement) concurrently on the per-plan streams. With PINV_BATCH_GRAPH the
// whole sequence is captured once into a CUDA graph and replayed, so a step
// of hundreds of launches costs one graph launch on the host.
//
// Results are bit-identical to building and applying the plans one by one:
// the shared launches run the same tile code over the same K order.
#include <algorithm>
#include <cstring>
#include <vector>

#include "plan_impl.h"

using namespace pinv;

struct pinv_batch {
    std::vector<pinv_plan*> plans;
    bool mixed = false, use_graph = false, graph_apply = false;
    int slices = 2;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    // per-plan operand tables (the Gram's, then the Recon's, in the same memory)
    void* work = nullptr;
    std::vector<void*> pwork;
    TcMulti gram;
    std::vector<TcMulti> rec1, rec2;  // per chunk of samples
    DevStatus* st = nullptr;
    DevStatus* st_host = nullptr;
    // graphs: the build is captured on its second call (the first runs
    // eagerly), the apply whenever its buffers or frame counts change
    int build_calls = 0;
    cudaGraphExec_t build_exec = nullptr;
    unsigned long long build_launches = 0;
    cudaGraphExec_t apply_exec = nullptr;
    std::vector<uintptr_t> apply_key;
    unsigned long long apply_launches = 0;
    std::vector<void*> scratch;
    std::vector<size_t> scratch_bytes;
    ~pinv_batch();
};

pinv_batch::~pinv_batch() {
    if (build_exec) cudaGraphExecDestroy(build_exec);
    if (apply_exec) cudaGraphExecDestroy(apply_exec);
    tc_multi_free(&gram);
    for (auto& m : rec1) tc_multi_free(&m);
    for (auto& m : rec2) tc_multi_free(&m);
    if (work) cudaFree(work);
    for (void* p : scratch)
        if (p) cudaFree(p);
    if (st) cudaFree(st);
    if (st_host) cudaFreeHost(st_host);
    for (auto s : side)
        if (s) cudaStreamDestroy(s);
    for (auto e : join)
        if (e) cudaEventDestroy(e);
    if (fork) cudaEventDestroy(fork);
}

namespace {

pinv_status cuda_err(cudaError_t e, const char* where) {
    return set_error(e == cudaErrorMemoryAllocation ? PINV_ERR_OOM : PINV_ERR_CUDA,
                     std::string(where) + ": " + cudaGetErrorString(e));
}
#define CKB(call)                                              \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_err(e_, #call);     \
    } while (0)
#define STB(call)                                              \
    do {                                                       \
        pinv_status s_ = (call);                               \
        if (s_ != PINV_OK) return s_;                          \
    } while (0)

pinv_status fork_all(pinv_batch* b, cudaStream_t s) {
    CKB(cudaEventRecord(b->fork, s));
    for (auto q : b->side) CKB(cudaStreamWaitEvent(q, b->fork, 0));
    return PINV_OK;
}

pinv_status join_all(pinv_batch* b, cudaStream_t s) {
    for (size_t i = 0; i < b->side.size(); ++i) {
        CKB(cudaEventRecord(b->join[i], b->side[i]));
        CKB(cudaStreamWaitEvent(s, b->join[i], 0));
    }
    return PINV_OK;
}

// The build sequence (run eagerly or under stream capture).
pinv_status build_sequence(pinv_batch* b, cudaStream_t s) {
    CKB(launch_reset_status(b->st, s));
    for (auto* p : b->plans) STB(build_begin(p, s));
    if (b->mixed) {
        const size_t n = b->plans.size();
        for (size_t i = 0; i < n; ++i) CKB(gram_bulk_table(b->plans[i]->enc, b->slices, b->pwork[i], s));
        CKB(tc_multi_launch(b->gram, b->slices, b->st, s));  // every plan's Gram
        for (size_t i = 0; i < n; ++i) {
            pinv_plan* p = b->plans[i];
            CKB(gram_bulk_finish(p->enc, p->lambda_abs, b->slices, (float4*)p->G, p->N, b->pwork[i], s));
            STB(build_gram(p, s, false));
        }
        STB(fork_all(b, s));
        for (size_t i = 0; i < n; ++i) {
            pinv_plan* p = b->plans[i];
            STB(build_factor(p, b->side[i], false));
            if (p->recon) CKB(recon_bulk_wtables(p->enc, p->W32, b->slices, b->pwork[i], b->side[i]));
        }
        STB(join_all(b, s));
        for (size_t c = 0; c < b->rec1.size(); ++c) {
            for (size_t i = 0; i < n; ++i)
                if (b->plans[i]->recon) CKB(recon_bulk_et(b->plans[i]->enc, b->slices, b->pwork[i], (int64_t)c, s));
            CKB(tc_multi_launch(b->rec1[c], b->slices, b->st, s));  // every plan's W E^H over chunk c
            CKB(tc_multi_launch(b->rec2[c], b->slices, b->st, s));  // every plan's W^H (W E^H)
        }
    } else {
        STB(fork_all(b, s));
        for (size_t i = 0; i < b->plans.size(); ++i) {
            pinv_plan* p = b->plans[i];
            STB(build_gram(p, b->side[i], true));
            STB(build_factor(p, b->side[i], false));
            STB(build_recon(p, b->side[i]));
        }
        STB(join_all(b, s));
    }
    for (auto* p : b->plans) STB(build_end(p, s));
    CKB(cudaMemcpyAsync(b->st_host, b->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s));
    return PINV_OK;
}

pinv_status apply_sequence(pinv_batch* b, const void* const* data, void* const* image, const int64_t* frames,
                           int dtype, cudaStream_t s) {
    STB(fork_all(b, s));
    for (size_t i = 0; i < b->plans.size(); ++i) {
        pinv_plan* p = b->plans[i];
        ApplyScratch sc;
        apply_scratch_layout(p, frames[i], dtype, b->scratch[i], &sc);
        STB(apply_impl(p, data[i], image[i], frames[i], dtype, b->side[i], sc));
    }
    return join_all(b, s);
}

// Capture fn(s) into a graph, instantiate it and count the kernels it holds.
template <class Fn>
pinv_status capture(cudaStream_t s, cudaGraphExec_t* exec, unsigned long long* launches, Fn fn) {
    if (s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread)
        return set_error(PINV_ERR_INVALID_ARG, "graph capture needs a created (non-default) stream");
    const unsigned long long l0 = g_launches.load();
    CKB(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    pinv_status st = fn();
    cudaGraph_t g = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(s, &g);
    if (st != PINV_OK) {
        if (g) cudaGraphDestroy(g);
        return st;
    }
    if (ec != cudaSuccess) return cuda_err(ec, "cudaStreamEndCapture");
    *launches = g_launches.load() - l0;
    g_launches -= *launches;  // counted again on every replay
    if (*exec) cudaGraphExecDestroy(*exec);
    *exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(exec, g, 0);
    cudaGraphDestroy(g);
    if (ei != cudaSuccess) return cuda_err(ei, "cudaGraphInstantiate");
    return PINV_OK;
}

pinv_status replay(cudaGraphExec_t exec, unsigned long long launches, cudaStream_t s) {
    CKB(cudaGraphLaunch(exec, s));
    g_launches += launches;
    return PINV_OK;
}

}  // namespace

extern "C" {

pinv_status pinv_batch_create(pinv_plan* const* plans, int n, int flags, pinv_batch** out) {
    if (!plans || !out || n < 1 || n > 1024) return set_error(PINV_ERR_INVALID_ARG, "need 1..1024 plans");
    *out = nullptr;
    auto* b = new pinv_batch();
    auto bad = [&](pinv_status st) { delete b; return st; };
    b->plans.assign(plans, plans + n);
    b->use_graph = (flags & PINV_BATCH_GRAPH) != 0;
    b->graph_apply = b->use_graph;
    b->mixed = b->plans[0] && b->plans[0]->precision != PINV_FP64;
    b->slices = b->plans[0] ? b->plans[0]->slices() : 2;
    for (int i = 0; i < n; ++i) {
        pinv_plan* p = b->plans[i];
        if (!p) return bad(set_error(PINV_ERR_INVALID_ARG, "null plan in batch"));
        if (p->lean) return bad(set_error(PINV_ERR_INVALID_ARG, "lean plans move their buffers between builds"));
        for (int j = 0; j < i; ++j)
            if (b->plans[j] == p) return bad(set_error(PINV_ERR_INVALID_ARG, "plan listed twice"));
        if ((p->precision != PINV_FP64) != b->mixed || (b->mixed && p->slices() != b->slices))
            return bad(set_error(PINV_ERR_INVALID_ARG, "a batch holds plans of one precision"));
        if (p->refine_iters > 0 && p->refine_tol > 0.0) b->graph_apply = false;  // host-read stopping rule
    }
    if (cudaMalloc((void**)&b->st, sizeof(DevStatus)) != cudaSuccess ||
        cudaMallocHost((void**)&b->st_host, sizeof(DevStatus)) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess)
        return bad(set_error(PINV_ERR_CUDA, "batch status allocation failed"));
    std::memset(b->st_host, 0, sizeof(DevStatus));
    b->side.assign(n, nullptr);
    b->join.assign(n, nullptr);
    b->scratch.assign(n, nullptr);
    b->scratch_bytes.assign(n, 0);
    for (int i = 0; i < n; ++i)
        if (cudaStreamCreateWithFlags(&b->side[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&b->join[i], cudaEventDisableTiming) != cudaSuccess)
            return bad(set_error(PINV_ERR_CUDA, "batch stream creation failed"));
    if (b->mixed) {
        // operand tables of every plan: the Gram's, then (same memory) the Recon's
        size_t bytes = 0;
        std::vector<size_t> off(n, 0);
        int64_t chunks = 0;
        for (int i = 0; i < n; ++i) {
            const pinv_plan* p = b->plans[i];
            size_t need = gram_bulk_bytes(p->enc, b->slices);
            if (p->recon) {
                need = std::max(need, recon_bulk_bytes(p->enc, b->slices));
                chunks = std::max(chunks, recon_bulk_chunks(p->enc, b->slices));
            }
            off[i] = bytes;
            bytes += (need + 255) & ~(size_t)255;
        }
        cudaError_t e = cudaMalloc(&b->work, bytes);
        if (e != cudaSuccess) return bad(cuda_err(e, "batch workspace"));
        std::vector<TcPlanArgs> all, rec;
        for (int i = 0; i < n; ++i) {
            pinv_plan* p = b->plans[i];
            b->pwork.push_back((unsigned char*)b->work + off[i]);
            const TcPlanArgs a{&p->enc, p->lambda_abs, (float4*)p->G, p->W32, (float2*)p->R, b->pwork[i]};
            all.push_back(a);
            if (p->recon) rec.push_back(a);
        }
        e = tc_multi_create(TC_MULTI_GRAM, all.data(), (int)all.size(), b->slices, 0, &b->gram);
        b->rec1.resize(chunks);
        b->rec2.resize(chunks);
        for (int64_t c = 0; c < chunks && e == cudaSuccess; ++c) {
            e = tc_multi_create(TC_MULTI_RECON1, rec.data(), (int)rec.size(), b->slices, c, &b->rec1[c]);
            if (e == cudaSuccess)
                e = tc_multi_create(TC_MULTI_RECON2, rec.data(), (int)rec.size(), b->slices, c, &b->rec2[c]);
        }
        if (e != cudaSuccess) return bad(cuda_err(e, "batch descriptors"));
    }
    *out = b;
    return PINV_OK;
}

pinv_status pinv_batch_build(pinv_batch* b, void* stream) {
    if (!b) return set_error(PINV_ERR_INVALID_ARG, "null batch");
    cudaStream_t s = (cudaStream_t)stream;
    for (auto* p : b->plans) p->built = false;
    if (b->use_graph && b->build_calls >= 1) {
        if (!b->build_exec)
            STB(capture(s, &b->build_exec, &b->build_launches, [&] { return build_sequence(b, s); }));
        STB(replay(b->build_exec, b->build_launches, s));
    } else {
        STB(build_sequence(b, s));
    }
    ++b->build_calls;
    // per-plan events: the plans report no stage timings in a batch, but their
    // sync and info calls work as after pinv_build
    for (auto* p : b->plans) {
        for (auto& ev : p->ev) CKB(cudaEventRecord(ev, s));
        p->built = true;
    }
    return PINV_OK;
}

pinv_status pinv_batch_apply(pinv_batch* b, const void* const* d_data, void* const* d_image,
                             const int64_t* n_frames, int dtype, void* stream) {
    if (!b || !d_data || !d_image || !n_frames) return set_error(PINV_ERR_INVALID_ARG, "null argument");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t n = b->plans.size();
    std::vector<uintptr_t> key;
    key.push_back((uintptr_t)dtype);
    bool grown = false;
    for (size_t i = 0; i < n; ++i) {
        STB(apply_check(b->plans[i], d_data[i], d_image[i], n_frames[i], dtype));
        const size_t need = apply_scratch_layout(b->plans[i], n_frames[i], dtype, nullptr, nullptr);
        if (need > b->scratch_bytes[i]) {
            // grow outside any capture; a replayed graph would hold the old buffer
            if (b->scratch[i]) CKB(cudaFree(b->scratch[i]));
            b->scratch[i] = nullptr;
            b->scratch_bytes[i] = 0;
            CKB(cudaMalloc(&b->scratch[i], need));
            b->scratch_bytes[i] = need;
            grown = true;
        }
        key.push_back((uintptr_t)d_data[i]);
        key.push_back((uintptr_t)d_image[i]);
        key.push_back((uintptr_t)n_frames[i]);
    }
    if (!b->graph_apply) return apply_sequence(b, d_data, d_image, n_frames, dtype, s);
    if (grown || !b->apply_exec || key != b->apply_key) {
        // one eager run first: it tunes launch shapes, which cannot be timed under capture
        STB(apply_sequence(b, d_data, d_image, n_frames, dtype, s));
        STB(capture(s, &b->apply_exec, &b->apply_launches,
                    [&] { return apply_sequence(b, d_data, d_image, n_frames, dtype, s); }));
        b->apply_key = key;
    }
    return replay(b->apply_exec, b->apply_launches, s);
}

pinv_status pinv_batch_sync(pinv_batch* b, int* failed_plan) {
    if (!b) return set_error(PINV_ERR_INVALID_ARG, "null batch");
    if (failed_plan) *failed_plan = -1;
    for (size_t i = 0; i < b->plans.size(); ++i) {
        const pinv_status st = pinv_plan_sync(b->plans[i]);
        if (st != PINV_OK) {
            if (failed_plan) *failed_plan = (int)i;
            return st;
        }
    }
    if (b->st_host->timeout_site)
        return set_error(PINV_ERR_TIMEOUT, "a bounded device wait gave up in a batched launch (site " +
                                               std::to_string(b->st_host->timeout_site) + ")");
    return PINV_OK;
}

void pinv_batch_destroy(pinv_batch* b) {
    if (!b) return;
    cudaDeviceSynchronize();
    delete b;
}

}  // extern "C"
