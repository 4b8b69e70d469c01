// Continuous-batching serving loop for Pinv-Recon plans.
//
// Reconstruction is split the way the paper motivates it (Section 4.5): Recon
// is built from the trajectory and encoding physics before data arrive, and
// each acquisition then only needs image = Recon x data. A server keeps the
// factored plans of registered trajectories resident in HBM under a byte
// budget and serves reconstruction requests as they arrive:
//
//   * one worker thread issues every CUDA call; callers only queue requests;
//   * requests are admitted in arrival order into up to `max_slots` slots,
//     each with its own stream and scratch, so the work of several requests
//     (and of a plan build) overlaps on the device;
//   * a request whose plan is not resident triggers its build on a separate
//     build stream; the request's slot waits on the build's event, other slots
//     keep running. To make room, idle resident plans are evicted least
//     recently used first; a plan that cannot fit fails its request with
//     PINV_ERR_BUDGET;
//   * completion is detected with events; latency runs from enqueue to the
//     moment the worker sees the request's event complete. Each request also
//     keeps the device times of its work (timing events on its slot's stream),
//     so the overlap of slots can be read back (pinv_serve_times).
//   * with merging on (pinv_server_set_merge), requests of the plan at the head
//     of the queue that wait behind it with the same element type join it in one
//     apply, up to a frame cap: their frames are gathered into the slot's scratch
//     (device-to-device copies on the slot's stream), reconstructed together and
//     scattered back; each still completes, and is counted, on its own;
//   * host fault injection (PINV_FAULT, read when the server is created) makes
//     failures on the host, never on the device: a comma-separated list of
//     one-shot faults, "alloc:P" (the next admission of plan P fails as if its
//     device allocation had, PINV_ERR_OOM), "build:P" (the next build of plan P
//     fails, PINV_ERR_INTERNAL), "drop:T" (request T completes with
//     PINV_ERR_INTERNAL without running) and "delay:T:MS" (request T's
//     completion is reported MS milliseconds after its work finished; its slot
//     is free at once). A plan whose admission or build failed is retried by its
//     next request; every other request runs as it would without the faults.
// Each request's result is computed by the same kernels in the same order as
// a standalone pinv_apply, so it does not depend on what else is in flight.
#include <algorithm>
#include <array>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <string>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "plan_impl.h"

using namespace pinv;

namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// A registered trajectory/encoding: owned copy of its descriptor and its
// resident plan, if any.
struct Registered {
    pinv_plan_desc desc{};
    std::vector<double> traj, coils, b0, times;
    std::vector<int64_t> vox;
    pinv_plan* plan = nullptr;
    cudaEvent_t ready = nullptr;  // recorded on the build stream after the build
    size_t bytes = 0;             // device bytes held while resident
    uint64_t last_use = 0;        // LRU clock
    int inflight = 0;             // requests submitted to slots and not yet completed
    pinv_status failed = PINV_OK; // set once a build of this encoding failed (e.g. NOT_PD)
};

struct Request {
    uint64_t ticket = 0;
    int plan_id = -1;
    const void* data = nullptr;
    void* image = nullptr;
    int64_t frames = 0;
    int dtype = PINV_C64;
    pinv_done_cb cb = nullptr;
    void* user = nullptr;
    double t_enqueue = 0;
    double dev_start_ms = -1, dev_end_ms = -1;  // device times of its work (ms after the server's origin)
};

// one-shot host fault (PINV_FAULT)
enum FaultKind { FAULT_ALLOC = 0, FAULT_BUILD = 1, FAULT_DROP = 2, FAULT_DELAY = 3 };
struct Fault {
    int kind;
    int64_t key;  // plan id (alloc, build) or ticket (drop, delay)
    double ms;    // delay
    bool used;
};
std::vector<Fault> parse_faults(const char* spec) {
    std::vector<Fault> out;
    if (!spec) return out;
    std::string s(spec);
    size_t pos = 0;
    while (pos <= s.size()) {
        size_t end = s.find(',', pos);
        if (end == std::string::npos) end = s.size();
        const std::string item = s.substr(pos, end - pos);
        pos = end + 1;
        const size_t c1 = item.find(':');
        if (c1 == std::string::npos) continue;
        const std::string kind = item.substr(0, c1), rest = item.substr(c1 + 1);
        const size_t c2 = rest.find(':');
        Fault f{-1, 0, 0.0, false};
        f.key = std::strtoll(rest.substr(0, c2).c_str(), nullptr, 10);
        if (kind == "alloc") f.kind = FAULT_ALLOC;
        else if (kind == "build") f.kind = FAULT_BUILD;
        else if (kind == "drop") f.kind = FAULT_DROP;
        else if (kind == "delay" && c2 != std::string::npos) {
            f.kind = FAULT_DELAY;
            f.ms = std::strtod(rest.substr(c2 + 1).c_str(), nullptr);
        }
        if (f.kind >= 0) out.push_back(f);
    }
    return out;
}

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;  // timing: the request's work starts / ends on the stream
    void* scratch = nullptr;
    size_t scratch_bytes = 0;
    bool busy = false;
    Request req;
    std::vector<Request> more;  // requests merged into req's apply
    pinv_status submit_status = PINV_OK;
};

}  // namespace

struct pinv_server {
    size_t budget = 0;
    int device = 0;
    std::vector<Registered> plans;
    std::deque<Request> queue;
    std::vector<Slot> slots;
    std::unordered_map<uint64_t, pinv_status> finished;
    // enqueue and completion (host, ms after creation), device start and end of the work
    std::unordered_map<uint64_t, std::array<double, 4>> times;
    double t_origin = 0;                // host time of creation
    cudaEvent_t origin = nullptr;       // recorded at creation on the build stream
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    cudaStream_t build_stream = nullptr;
    uint64_t next_ticket = 1, lru_clock = 0;
    int64_t merge_frames = 0;  // 0: no merging; else the most frames one merged apply takes
    size_t resident_bytes = 0;
    std::vector<Fault> faults;                            // PINV_FAULT
    std::vector<std::pair<double, Request>> delayed;      // (report time, request) of delayed completions
    // statistics
    std::vector<double> latency_ms;
    uint64_t completed = 0, failed = 0, builds = 0, evictions = 0, recon_drops = 0;
    double frames = 0, t_first = 0, t_last = 0;

    void run();
    bool take_fault(int kind, int64_t key, double* ms = nullptr) {
        for (auto& f : faults)
            if (!f.used && f.kind == kind && f.key == key) {
                f.used = true;
                if (ms) *ms = f.ms;
                return true;
            }
        return false;
    }
    bool release_delayed(std::unique_lock<std::mutex>& lk);
    bool dispatch_one(std::unique_lock<std::mutex>& lk);
    bool reap(std::unique_lock<std::mutex>& lk);
    pinv_status make_resident(Registered& r, int id, bool* defer);
    void evict(Registered& v);
    void finish(const Request& q, pinv_status st, std::unique_lock<std::mutex>& lk);
};

namespace {

// Device bytes a plan keeps while resident (its build transients are not
// counted): factors, exact Gram, phase tables and, if stored, Recon.
size_t plan_footprint(const pinv_plan_desc& d, bool with_recon) {
    const double N = (double)d.n_vox, Mk = (double)d.n_samples, M = Mk * d.n_coils;
    const bool fp64 = d.precision == PINV_FP64;
    // lean plans: G^-1 (FP64), or W32 (+ the FP64 W for an FP64 residual)
    double b = fp64 ? N * N * 16.0 : N * N * 8.0;
    if (!fp64 && d.refine_residual == PINV_RESIDUAL_FP64) b += N * N * 16.0;
    if (!fp64 && d.refine_residual == PINV_RESIDUAL_TOEPLITZ) b += N * N * 24.0;  // exact Gram digits
    int recon = d.recon_mode;
    if (recon == PINV_RECON_AUTO) recon = N * M * (fp64 ? 16.0 : 8.0) <= 64.0 * (1ull << 30);
    if (recon && with_recon) b += N * M * (fp64 ? 16.0 : 8.0);
    int width = 0;
    for (int i = 0; i < d.ndim; ++i) width += d.dims[i];
    b += Mk * width * 48.0 + N * d.n_coils * 40.0 + N * 64.0;  // tables (c128, c64, double-float, transposed)
    if (d.b0_hz) b += Mk * 8.0 + N * 48.0 * std::min(Mk, 4096.0);
    return (size_t)b + (1u << 20);
}

}  // namespace

void pinv_server::finish(const Request& q, pinv_status st, std::unique_lock<std::mutex>& lk) {
    const double t = now_s();
    // the callback runs before the request counts as finished, so a waiter
    // that returns may release whatever the callback uses
    if (q.cb) {
        lk.unlock();
        q.cb(q.ticket, st, q.user);
        lk.lock();
    }
    finished[q.ticket] = st;
    times[q.ticket] = {(q.t_enqueue - t_origin) * 1e3, (t - t_origin) * 1e3, q.dev_start_ms, q.dev_end_ms};
    if (st == PINV_OK) {
        ++completed;
        frames += (double)q.frames;
        latency_ms.push_back((t - q.t_enqueue) * 1e3);
        t_last = t;
    } else {
        ++failed;
    }
    cv_done.notify_all();
}

void pinv_server::evict(Registered& v) {
    pinv_plan_destroy(v.plan);  // no request of it is in flight (inflight == 0)
    v.plan = nullptr;
    resident_bytes -= v.bytes;
    v.bytes = 0;
}

// Make plan `id` resident, building it on the build stream. Room is made in
// tiers: first the Recon of idle plans is dropped (least recently used
// first; they keep serving from their factors), then idle plans are evicted.
// A plan whose Recon does not fit is built factor-only. *defer is set when
// the plan does not fit now but will once requests in flight have finished.
pinv_status pinv_server::make_resident(Registered& r, int id, bool* defer) {
    *defer = false;
    if (r.plan) return PINV_OK;
    const size_t need_full = plan_footprint(r.desc, true), need_fac = plan_footprint(r.desc, false);
    if (need_fac > budget) return set_error(PINV_ERR_BUDGET, "plan footprint exceeds the server's HBM budget");
    auto lru_idle = [&](bool with_recon) {
        int v = -1;
        for (int i = 0; i < (int)plans.size(); ++i) {
            const Registered& c = plans[i];
            if (i == id || !c.plan || c.inflight > 0 || (with_recon && !c.plan->recon)) continue;
            if (v < 0 || c.last_use < plans[v].last_use) v = i;
        }
        return v;
    };
    while (resident_bytes + need_full > budget) {  // tier 1: idle Recons
        const int v = lru_idle(true);
        if (v < 0) break;
        const size_t freed = plans[v].plan->drop_recon();
        plans[v].bytes -= std::min(plans[v].bytes, freed);
        resident_bytes -= std::min(resident_bytes, freed);
        ++recon_drops;
    }
    while (resident_bytes + need_fac > budget) {  // tier 2: idle plans
        const int v = lru_idle(false);
        if (v < 0) break;
        evict(plans[v]);
        ++evictions;
    }
    if (resident_bytes + need_fac > budget) {
        size_t busy = 0;
        for (auto& c : plans) busy += c.inflight > 0 ? c.bytes : 0;
        *defer = busy > 0;
        return *defer ? PINV_OK : set_error(PINV_ERR_BUDGET, "no idle plan to evict within the HBM budget");
    }
    pinv_plan_desc d = r.desc;
    const bool full = resident_bytes + need_full <= budget;
    if (!full) d.recon_mode = PINV_RECON_NONE;
    if (take_fault(FAULT_ALLOC, id)) return set_error(PINV_ERR_OOM, "injected allocation failure at admission");
    pinv_plan* p = nullptr;
    pinv_status st = pinv_plan_create(&d, build_stream, &p);
    if (st != PINV_OK) return st;
    st = take_fault(FAULT_BUILD, id) ? set_error(PINV_ERR_INTERNAL, "injected build failure")
                                     : pinv_build(p, build_stream);
    if (st != PINV_OK) {
        pinv_plan_destroy(p);
        return st;
    }
    cudaError_t e = cudaEventRecord(r.ready, build_stream);
    if (e != cudaSuccess) {
        pinv_plan_destroy(p);
        return set_error(PINV_ERR_CUDA, cudaGetErrorString(e));
    }
    r.plan = p;
    r.bytes = std::max(full ? need_full : need_fac, p->bytes);
    resident_bytes += r.bytes;
    ++builds;
    return PINV_OK;
}

// Submit the oldest queued request to a free slot. Returns true if it did work.
bool pinv_server::dispatch_one(std::unique_lock<std::mutex>& lk) {
    if (queue.empty()) return false;
    Slot* slot = nullptr;
    for (auto& s : slots)
        if (!s.busy) { slot = &s; break; }
    if (!slot) return false;
    Request q = queue.front();
    Registered& r = plans[q.plan_id];
    bool defer = false;
    pinv_status st = r.failed != PINV_OK ? r.failed : make_resident(r, q.plan_id, &defer);
    if (defer) return false;  // head of the queue waits until a slot completes
    queue.pop_front();
    if (st == PINV_OK && take_fault(FAULT_DROP, (int64_t)q.ticket))
        st = set_error(PINV_ERR_INTERNAL, "request dropped (injected)");
    if (st == PINV_OK) st = apply_check(r.plan, q.data, q.image, q.frames, q.dtype);
    // requests of the same plan and element type queued behind this one join its apply
    std::vector<Request> more;
    int64_t F = q.frames;
    if (st == PINV_OK && merge_frames > 0 && faults.empty() && q.frames > 0) {
        for (auto it = queue.begin(); it != queue.end();) {
            if (it->plan_id == q.plan_id && it->dtype == q.dtype && it->frames > 0 && F + it->frames <= merge_frames &&
                apply_check(r.plan, it->data, it->image, it->frames, it->dtype) == PINV_OK) {
                F += it->frames;
                more.push_back(*it);
                it = queue.erase(it);
            } else {
                ++it;
            }
        }
    }
    if (st == PINV_OK && F > 0) {
        const size_t es = q.dtype == PINV_C128 ? 16 : 8;
        const int64_t rows = r.plan->M, n = r.plan->N;
        const size_t base = (apply_scratch_layout(r.plan, F, q.dtype, nullptr, nullptr) + 255) & ~(size_t)255;
        const size_t dbytes = more.empty() ? 0 : (((size_t)F * rows * es + 255) & ~(size_t)255);
        const size_t need = base + dbytes + (more.empty() ? 0 : (size_t)F * n * es);
        if (need > slot->scratch_bytes) {
            if (slot->scratch) cudaFree(slot->scratch);
            slot->scratch = nullptr;
            slot->scratch_bytes = 0;
            if (cudaMalloc(&slot->scratch, need) != cudaSuccess) st = set_error(PINV_ERR_OOM, "slot scratch");
            else slot->scratch_bytes = need;
        }
        if (st == PINV_OK) {
            ApplyScratch sc;
            apply_scratch_layout(r.plan, F, q.dtype, slot->scratch, &sc);
            uint8_t* dbuf = (uint8_t*)slot->scratch + base;  // merged: frames gathered here
            uint8_t* ibuf = dbuf + dbytes;                   // and their images
            const void* data = q.data;
            void* image = q.image;
            if (cudaStreamWaitEvent(slot->stream, r.ready, 0) != cudaSuccess ||
                cudaEventRecord(slot->t0, slot->stream) != cudaSuccess)
                st = set_error(PINV_ERR_CUDA, "cudaStreamWaitEvent");
            if (st == PINV_OK && !more.empty()) {
                size_t off = 0;
                auto gather = [&](const Request& m) {
                    const size_t b = (size_t)m.frames * rows * es;
                    if (cudaMemcpyAsync(dbuf + off, m.data, b, cudaMemcpyDeviceToDevice, slot->stream) != cudaSuccess)
                        st = set_error(PINV_ERR_CUDA, "merge gather");
                    off += b;
                };
                gather(q);
                for (auto& m : more) gather(m);
                data = dbuf;
                image = ibuf;
            }
            if (st == PINV_OK) st = apply_impl(r.plan, data, image, F, q.dtype, slot->stream, sc);
            if (st == PINV_OK && !more.empty()) {
                size_t off = 0;
                auto scatter = [&](const Request& m) {
                    const size_t b = (size_t)m.frames * n * es;
                    if (cudaMemcpyAsync(m.image, ibuf + off, b, cudaMemcpyDeviceToDevice, slot->stream) != cudaSuccess)
                        st = set_error(PINV_ERR_CUDA, "merge scatter");
                    off += b;
                };
                scatter(q);
                for (auto& m : more) scatter(m);
            }
        }
    }
    if (st == PINV_OK && F > 0 && cudaEventRecord(slot->t1, slot->stream) != cudaSuccess)
        st = set_error(PINV_ERR_CUDA, "cudaEventRecord");
    if (st == PINV_OK && cudaEventRecord(slot->done, slot->stream) != cudaSuccess)
        st = set_error(PINV_ERR_CUDA, "cudaEventRecord");
    if (st != PINV_OK) {
        finish(q, st, lk);
        for (auto& m : more) finish(m, st, lk);
        return true;
    }
    r.inflight++;
    r.last_use = ++lru_clock;
    slot->busy = true;
    slot->req = q;
    slot->more = std::move(more);
    return true;
}

// Complete every slot whose event has fired. Returns true if it did work.
bool pinv_server::reap(std::unique_lock<std::mutex>& lk) {
    bool any = false;
    for (auto& s : slots) {
        if (!s.busy) continue;
        const cudaError_t e = cudaEventQuery(s.done);
        if (e == cudaErrorNotReady) continue;
        s.busy = false;
        Registered& r = plans[s.req.plan_id];
        r.inflight--;
        pinv_status st = PINV_OK;
        if (e != cudaSuccess) {
            st = set_error(PINV_ERR_CUDA, cudaGetErrorString(e));
        } else if (r.failed != PINV_OK) {
            st = r.failed;
        } else if (r.plan && r.plan->st_host->not_pd_pivot != INT_MAX) {
            // the build behind this request found a non-positive pivot: later
            // requests of this encoding fail at once, and the plan is dropped
            st = r.failed = PINV_ERR_NOT_PD;
        } else if (r.plan && r.plan->st_host->timeout_site) {
            st = PINV_ERR_TIMEOUT;
        }
        if (r.failed != PINV_OK && r.plan && r.inflight == 0) evict(r);
        Request q = s.req;
        float a = 0.f, b = 0.f;
        if (st == PINV_OK && q.frames > 0 && cudaEventElapsedTime(&a, origin, s.t0) == cudaSuccess &&
            cudaEventElapsedTime(&b, origin, s.t1) == cudaSuccess) {
            q.dev_start_ms = a;
            q.dev_end_ms = b;
        }
        double ms = 0.0;
        if (st == PINV_OK && take_fault(FAULT_DELAY, (int64_t)q.ticket, &ms))
            delayed.push_back({now_s() + ms * 1e-3, q});  // reported later; the slot is free now
        else
            finish(q, st, lk);
        for (Request m : s.more) {  // merged requests: same apply, same status and device times
            m.dev_start_ms = q.dev_start_ms;
            m.dev_end_ms = q.dev_end_ms;
            finish(m, st, lk);
        }
        s.more.clear();
        any = true;
    }
    return any;
}

// Report the delayed completions whose time has come. Returns true if it did work.
bool pinv_server::release_delayed(std::unique_lock<std::mutex>& lk) {
    bool any = false;
    const double t = now_s();
    for (size_t i = 0; i < delayed.size();) {
        if (delayed[i].first <= t) {
            const Request q = delayed[i].second;
            delayed.erase(delayed.begin() + (long)i);
            finish(q, PINV_OK, lk);
            any = true;
        } else {
            ++i;
        }
    }
    return any;
}

void pinv_server::run() {
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    while (true) {
        bool work = reap(lk);
        work = release_delayed(lk) || work;
        while (dispatch_one(lk)) work = true;
        bool busy = !delayed.empty();
        for (auto& s : slots) busy = busy || s.busy;
        if (stop && !busy && queue.empty()) break;
        if (!work) {
            if (busy) cv_work.wait_for(lk, std::chrono::microseconds(50));
            else cv_work.wait(lk, [&] { return stop || !queue.empty(); });
        }
    }
}

extern "C" {

pinv_status pinv_server_create(size_t hbm_budget_bytes, int max_slots, pinv_server** out) {
    if (!out || max_slots < 1 || max_slots > 64 || hbm_budget_bytes == 0)
        return set_error(PINV_ERR_INVALID_ARG, "need out, 1 <= max_slots <= 64 and a nonzero budget");
    *out = nullptr;
    auto* sv = new pinv_server();
    sv->budget = hbm_budget_bytes;
    if (cudaGetDevice(&sv->device) != cudaSuccess ||
        cudaStreamCreateWithFlags(&sv->build_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreate(&sv->origin) != cudaSuccess) {
        delete sv;
        return set_error(PINV_ERR_CUDA, "server stream creation failed");
    }
    sv->slots.resize(max_slots);
    for (auto& s : sv->slots) {
        if (cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreate(&s.t0) != cudaSuccess || cudaEventCreate(&s.t1) != cudaSuccess) {
            delete sv;
            return set_error(PINV_ERR_CUDA, "slot stream creation failed");
        }
    }
    sv->t_origin = now_s();
    if (cudaEventRecord(sv->origin, sv->build_stream) != cudaSuccess) {
        delete sv;
        return set_error(PINV_ERR_CUDA, "server event record failed");
    }
    sv->faults = parse_faults(std::getenv("PINV_FAULT"));
    sv->worker = std::thread([sv] { sv->run(); });
    *out = sv;
    return PINV_OK;
}

pinv_status pinv_serve_register(pinv_server* sv, const pinv_plan_desc* d, int* plan_id) {
    if (!sv || !d || !plan_id) return set_error(PINV_ERR_INVALID_ARG, "null argument");
    if (d->ndim < 1 || d->ndim > 3 || d->n_vox < 1 || d->n_samples < 1 || d->n_coils < 1 || !d->traj)
        return set_error(PINV_ERR_INVALID_ARG, "bad descriptor");
    Registered r;
    r.desc = *d;
    r.desc.refine_tol = 0.0;  // fixed refinement steps: the worker never waits on a host read
    r.desc.lean = 1;          // resident plans keep only what an apply reads
    r.traj.assign(d->traj, d->traj + d->n_samples * d->ndim);
    r.desc.traj = r.traj.data();
    if (d->coil_maps) {
        r.coils.assign(d->coil_maps, d->coil_maps + 2 * d->n_vox * d->n_coils);
        r.desc.coil_maps = r.coils.data();
    }
    if (d->b0_hz) {
        if (!d->times) return set_error(PINV_ERR_INVALID_ARG, "b0_hz needs times");
        r.b0.assign(d->b0_hz, d->b0_hz + d->n_vox);
        r.times.assign(d->times, d->times + d->n_samples);
        r.desc.b0_hz = r.b0.data();
        r.desc.times = r.times.data();
    }
    if (d->voxel_index) {
        r.vox.assign(d->voxel_index, d->voxel_index + d->n_vox);
        r.desc.voxel_index = r.vox.data();
    }
    std::unique_lock<std::mutex> lk(sv->mu);
    // the event is created here, on the caller's thread, with the server's device current
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev != sv->device) cudaSetDevice(sv->device);
    const cudaError_t e = cudaEventCreateWithFlags(&r.ready, cudaEventDisableTiming);
    if (dev != sv->device) cudaSetDevice(dev);
    if (e != cudaSuccess) return set_error(PINV_ERR_CUDA, "event creation failed");
    sv->plans.push_back(std::move(r));
    // vector growth moved the owned arrays; re-point each descriptor at its own copies
    for (auto& p : sv->plans) {
        p.desc.traj = p.traj.data();
        if (!p.coils.empty()) p.desc.coil_maps = p.coils.data();
        if (!p.b0.empty()) { p.desc.b0_hz = p.b0.data(); p.desc.times = p.times.data(); }
        if (!p.vox.empty()) p.desc.voxel_index = p.vox.data();
    }
    *plan_id = (int)sv->plans.size() - 1;
    return PINV_OK;
}

pinv_status pinv_serve_enqueue(pinv_server* sv, int plan_id, const void* d_data, void* d_image, int64_t n_frames,
                               int dtype, pinv_done_cb cb, void* user, uint64_t* ticket) {
    if (!sv || !ticket) return set_error(PINV_ERR_INVALID_ARG, "null argument");
    Request q;
    q.plan_id = plan_id;
    q.data = d_data;
    q.image = d_image;
    q.frames = n_frames;
    q.dtype = dtype;
    q.cb = cb;
    q.user = user;
    q.t_enqueue = now_s();
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        if (plan_id < 0 || plan_id >= (int)sv->plans.size()) return set_error(PINV_ERR_INVALID_ARG, "unknown plan");
        if (sv->stop) return set_error(PINV_ERR_INVALID_ARG, "server is shutting down");
        q.ticket = sv->next_ticket++;
        *ticket = q.ticket;
        if (sv->t_first == 0) sv->t_first = q.t_enqueue;
        sv->queue.push_back(q);
    }
    sv->cv_work.notify_one();
    return PINV_OK;
}

pinv_status pinv_serve_poll(pinv_server* sv, uint64_t ticket, int* done, pinv_status* result) {
    if (!sv || !done) return set_error(PINV_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->finished.find(ticket);
    *done = it != sv->finished.end();
    if (*done && result) *result = it->second;
    return PINV_OK;
}

pinv_status pinv_serve_wait(pinv_server* sv, uint64_t ticket, double timeout_s, pinv_status* result) {
    if (!sv) return set_error(PINV_ERR_INVALID_ARG, "null server");
    std::unique_lock<std::mutex> lk(sv->mu);
    const bool ok = sv->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s),
                                         [&] { return sv->finished.count(ticket) > 0; });
    if (!ok) return set_error(PINV_ERR_TIMEOUT, "request not finished within the timeout");
    if (result) *result = sv->finished[ticket];
    return PINV_OK;
}

pinv_status pinv_server_set_merge(pinv_server* sv, int64_t max_frames) {
    if (!sv || max_frames < 0) return set_error(PINV_ERR_INVALID_ARG, "need a server and max_frames >= 0");
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->merge_frames = max_frames;
    return PINV_OK;
}

pinv_status pinv_serve_times(pinv_server* sv, uint64_t ticket, double* times_ms) {
    if (!sv || !times_ms) return set_error(PINV_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->times.find(ticket);
    if (it == sv->times.end()) return set_error(PINV_ERR_INVALID_ARG, "unknown or unfinished ticket");
    for (int i = 0; i < 4; ++i) times_ms[i] = it->second[i];
    return PINV_OK;
}

pinv_status pinv_server_stats(pinv_server* sv, pinv_server_stats_t* o) {
    if (!sv || !o) return set_error(PINV_ERR_INVALID_ARG, "null argument");
    std::lock_guard<std::mutex> lk(sv->mu);
    std::memset(o, 0, sizeof(*o));
    o->completed = sv->completed;
    o->failed = sv->failed;
    o->builds = sv->builds;
    o->evictions = sv->evictions;
    o->recon_drops = sv->recon_drops;
    o->frames = sv->frames;
    o->resident_bytes = sv->resident_bytes;
    for (auto& p : sv->plans) o->resident_plans += p.plan != nullptr;
    o->queued = (int)sv->queue.size();
    if (!sv->latency_ms.empty()) {
        std::vector<double> v = sv->latency_ms;
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) { return v[std::min(v.size() - 1, (size_t)(q * (double)(v.size() - 1) + 0.5))]; };
        o->p50_ms = pct(0.50);
        o->p99_ms = pct(0.99);
        o->max_ms = v.back();
        double s = 0;
        for (double x : v) s += x;
        o->mean_ms = s / (double)v.size();
        o->span_s = sv->t_last - sv->t_first;
    }
    return PINV_OK;
}

void pinv_server_destroy(pinv_server* sv) {
    if (!sv) return;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    cudaSetDevice(sv->device);
    cudaDeviceSynchronize();
    for (auto& p : sv->plans) {
        pinv_plan_destroy(p.plan);
        if (p.ready) cudaEventDestroy(p.ready);
    }
    for (auto& s : sv->slots) {
        if (s.scratch) cudaFree(s.scratch);
        if (s.done) cudaEventDestroy(s.done);
        if (s.t0) cudaEventDestroy(s.t0);
        if (s.t1) cudaEventDestroy(s.t1);
        if (s.stream) cudaStreamDestroy(s.stream);
    }
    if (sv->origin) cudaEventDestroy(sv->origin);
    if (sv->build_stream) cudaStreamDestroy(sv->build_stream);
    delete sv;
}

}  // extern "C"
