// Serving loop: resident gauge fields, HBM-budgeted admission, continuous batching.
//
// A request (field, Ns, m0, m_q, weights, nrhs right-hand sides, tolerance, precision)
// joins the batch group of its (field, Ns, m0, weights, precision): one Engine (packed
// links) plus one slot-based BatchCG on its own CUDA stream.  One worker thread runs
// the loop below; client threads only enqueue and wait:
//   1. admit queued requests, in arrival order, into free slots of their group (creating
//      the group when the budget allows); a request that does not fit waits;
//   2. for every group whose previous chunk of iterations has finished on the device
//      (an event query, never a blocking wait), read its systems' states, start the FP64
//      reliable updates of parked systems, hand finished systems back (copy x out, free the
//      slot; a request completes when all its systems are done) and launch its next chunk
//      of `k` CG iterations.  Groups run on their own streams and progress independently,
//      so a batch of small lattices is not held to the pace of a large one; streams of
//      groups with less work per iteration get a higher scheduling priority;
//   3. drop idle groups to return their memory to the budget.
// New requests therefore enter running batches between iterations, as slots and
// memory free up.  Caller buffers must stay valid until the ticket completes.
// A second thread copies finished solutions out to host buffers, so the worker never waits
// for a device-to-host copy.  Any CUDA or solver error in a group fails every request that
// has systems in it (with that status) and drops the group.  Requests can be cancelled, and a
// policy can shed requests that waited too long for admission or refuse new ones when the
// queue is full (serve_set_policy).
#include <algorithm>
#include <atomic>
#include <cstdlib>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "batch_cg.h"
#include "engine.h"

namespace odwf {

using Clock = std::chrono::steady_clock;

struct Field {
    odwf_lattice lat{};
    void* U = nullptr;  // resident external-layout links (device)
    size_t bytes = 0;
};

struct Request {
    uint64_t ticket = 0;
    odwf_request req{};
    std::vector<double> omega;
    std::vector<const void*> b;
    std::vector<void*> x;
    Clock::time_point t_submit, t_admit;
    int remaining = 0;
    int status = ODWF_PENDING;
    int iters = 0;
    double resid = 0;
    double latency_ms = 0, queue_ms = 0;
    bool admitted = false;
    bool done = false;
    bool cancel = false;  // serve_cancel of a running request: its slots stop between chunks
};

struct Group {
    std::string key;
    int field_id = 0;
    int prec = ODWF_F16;
    std::unique_ptr<Engine> eng;
    std::unique_ptr<BatchCG> cg;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_chunk = nullptr;  // end of the last launched chunk of iterations
    bool in_flight = false;
    size_t reserved = 0;
    std::vector<std::shared_ptr<Request>> slot_req;  // owner of each slot (until its copy-out is done)
    std::vector<int> slot_rhs;
    std::vector<cudaEvent_t> ev_out;  // per slot: its solution has been unpacked into the staging buffer
    bool failed = false;              // an error: requests failed, the group is dropped
    int copies = 0;                   // copy-out jobs of this group queued or running
    Clock::time_point last_used;
    int used_slots() const {
        int n = 0;
        for (auto& r : slot_req) n += r ? 1 : 0;
        return n;
    }
};

}  // namespace odwf

struct serve_handle {
    size_t budget = 0;
    size_t used = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    uint64_t next_ticket = 1;
    int device = 0;
    std::map<int, odwf::Field> fields;
    std::deque<std::shared_ptr<odwf::Request>> queue;
    std::map<uint64_t, std::shared_ptr<odwf::Request>> tickets;
    std::vector<std::unique_ptr<odwf::Group>> groups;
    std::thread worker;
    // copy-out of finished systems whose x is host memory (one job per system)
    struct CopyJob {
        odwf::Group* g;
        int slot;
        std::shared_ptr<odwf::Request> R;
        void* dst;
        const void* src;
        size_t bytes;
        int code;
        int iters;
        double resid;
    };
    std::deque<CopyJob> copy_jobs;
    std::condition_variable cv_copy;
    std::thread copier;
    bool copier_stop = false;
    // policy: requests still queued after admit_deadline_ms are shed (ODWF_ETIMEOUT); at most
    // max_queued requests wait (serve_submit answers ODWF_EBUSY beyond); <= 0 disables each
    double admit_deadline_ms = 0;
    int max_queued = 0;
    int fair = 0;  // 1: every batch at the same stream priority
    uint64_t shed = 0, refused = 0;
};

namespace odwf {

namespace {

constexpr int kMaxSlots = 16;
constexpr int kIterChunk = 8;

// Host-side failure injection for tests: with ODWF_SERVE_INJECT_ERROR=n in the environment the
// n-th chunk launch of the process reports ODWF_ECUDA instead of launching (no device fault).
long inject_at() {
    static const long n = [] {
        const char* v = std::getenv("ODWF_SERVE_INJECT_ERROR");
        return v ? std::atol(v) : 0L;
    }();
    return n;
}
std::atomic<long> g_chunks{0};

size_t per_system_bytes(size_t sites5, int prec) {
    // x staging for a host output (external layout) and a device copy of a host b
    if (prec == ODWF_F64) return sites5 * 192 * 8;
    const size_t lowb = prec == ODWF_F32 ? 96 : 52;
    // FP64 x, a device copy of a host b, x staging, FP32 r and x, five low-precision fields
    return sites5 * (192 * 3 + 96 * 2 + lowb * 5);
}

size_t group_fixed_bytes(size_t vh, size_t sites5) {
    // links (FP64, float-float, FP32-18, FP32-12 and its site-major copy), FP64 / float-float
    // temporaries, scratch
    return 8 * vh * (144 + 144 + 80 + 48 + 96) + sites5 * 192 * 6 + (1 << 20);
}

std::string group_key(const odwf_request& r, const std::vector<double>& om) {
    std::string k = std::to_string(r.field_id) + "/" + std::to_string(r.Ns) + "/" + std::to_string(r.m0) + "/" +
                    std::to_string(r.prec);
    for (double w : om) {
        char buf[40];
        snprintf(buf, sizeof(buf), "/%.17g", w);
        k += buf;
    }
    return k;
}

void complete(serve_handle* S, const std::shared_ptr<Request>& R, int status) {
    R->status = status;
    R->done = true;
    R->latency_ms = std::chrono::duration<double, std::milli>(Clock::now() - R->t_submit).count();
    S->cv_done.notify_all();
}

// Try to admit the request (all its systems at once); returns true when admitted.
bool try_admit(serve_handle* S, const std::shared_ptr<Request>& R, std::unique_lock<std::mutex>& lk) {
    const odwf_request& q = R->req;
    auto fit = S->fields.find(q.field_id);
    if (fit == S->fields.end()) {
        complete(S, R, ODWF_ENOTFOUND);
        return true;
    }
    const odwf_lattice& lat = fit->second.lat;
    const size_t vh = (size_t)lat.dims[0] * lat.dims[1] * lat.dims[2] * lat.dims[3] / 2;
    const size_t sites5 = vh * q.Ns;
    const std::string key = group_key(q, R->omega);
    Group* G = nullptr;
    for (auto& g : S->groups)
        if (g->key == key) G = g.get();
    const size_t psb = per_system_bytes(sites5, q.prec);
    if (G) {
        int free_slots = 0;
        for (auto& r : G->slot_req) free_slots += r ? 0 : 1;
        if (free_slots < q.nrhs) return false;
    } else {
        const size_t avail = S->budget > S->used ? S->budget - S->used : 0;
        const size_t fixed = group_fixed_bytes(vh, sites5);
        if (fixed + psb * q.nrhs > avail) return false;
        const int cap = (int)std::min<size_t>(kMaxSlots, std::max<size_t>(q.nrhs, (avail - fixed) / psb / 2));
        auto g = std::make_unique<Group>();
        g->key = key;
        g->field_id = q.field_id;
        g->prec = q.prec;
        g->eng = std::make_unique<Engine>();
        lk.unlock();  // device work below; the queue stays consistent (only this thread admits)
        int rc = g->eng->init(&lat, q.Ns, q.m0, q.mq, R->omega.data());
        if (!rc) {
            // less work per iteration -> higher priority (numerically lower), one level per 4x
            int least = 0, greatest = 0;
            cudaDeviceGetStreamPriorityRange(&least, &greatest);
            int prio = greatest;
            if (!S->fair)
                for (size_t w = sites5; w > (1u << 18) && prio < least; w >>= 2) ++prio;
            if (cudaStreamCreateWithPriority(&g->stream, cudaStreamNonBlocking, prio) != cudaSuccess ||
                cudaEventCreateWithFlags(&g->ev_chunk, cudaEventDisableTiming) != cudaSuccess)
                rc = ODWF_ECUDA;
        }
        if (!rc) rc = g->eng->set_gauge(fit->second.U, g->stream);
        odwf_solve_params prm;
        std::memset(&prm, 0, sizeof(prm));
        prm.tol = q.tol;
        prm.max_iter = q.max_iter;
        prm.prec = q.prec;
        prm.delta = 0.01;
        g->cg = std::make_unique<BatchCG>();
        if (!rc) rc = g->cg->init(g->eng.get(), cap, prm, g->stream);
        lk.lock();
        if (rc) {
            if (g->ev_chunk) cudaEventDestroy(g->ev_chunk);
            if (g->stream) cudaStreamDestroy(g->stream);
            complete(S, R, rc);
            return true;
        }
        g->reserved = fixed + psb * cap;
        S->used += g->reserved;
        g->slot_req.assign(cap, nullptr);
        g->slot_rhs.assign(cap, -1);
        g->ev_out.assign(cap, nullptr);
        for (auto& e : g->ev_out) cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
        G = g.get();
        S->groups.push_back(std::move(g));
    }
    // place the systems into free slots
    lk.unlock();
    int rc = ODWF_OK;
    std::vector<int> slots;
    for (int i = 0; i < (int)G->slot_req.size() && (int)slots.size() < q.nrhs; ++i)
        if (!G->slot_req[i]) slots.push_back(i);
    for (int k = 0; k < q.nrhs && !rc; ++k) {
        const double2* db = (const double2*)R->b[k];  // host data is copied per slot by admit()
        rc = G->cg->admit(slots[k], db, q.mq, G->stream, q.tol, q.max_iter);
    }
    lk.lock();
    if (rc) {
        complete(S, R, rc);
        return true;
    }
    for (int k = 0; k < q.nrhs; ++k) {
        G->slot_req[slots[k]] = R;
        G->slot_rhs[slots[k]] = k;
    }
    R->admitted = true;
    R->t_admit = Clock::now();
    R->queue_ms = std::chrono::duration<double, std::milli>(R->t_admit - R->t_submit).count();
    R->remaining = q.nrhs;
    G->last_used = Clock::now();
    return true;
}

void destroy_group(Group* g) {
    if (g->stream) cudaStreamSynchronize(g->stream);
    g->cg.reset();
    g->eng.reset();
    for (auto& e : g->ev_out)
        if (e) cudaEventDestroy(e);
    g->ev_out.clear();
    if (g->ev_chunk) cudaEventDestroy(g->ev_chunk);
    if (g->stream) cudaStreamDestroy(g->stream);
    g->ev_chunk = nullptr;
    g->stream = nullptr;
}

// One system of R finished with `code`: count it, complete R when it was the last.
void system_done(serve_handle* S, const std::shared_ptr<Request>& R, int code, int iters, double resid) {
    R->iters = std::max(R->iters, iters);
    R->resid = std::max(R->resid, resid);
    if (code && R->status == ODWF_PENDING) R->status = code;
    if (--R->remaining == 0 && !R->done) complete(S, R, R->status == ODWF_PENDING ? ODWF_OK : R->status);
}

// An error in group g: fail every request with systems in it and mark the group for dropping.
// Called with the serve lock held.
void fail_group(serve_handle* S, Group* g, int code) {
    g->failed = true;
    for (size_t i = 0; i < g->slot_req.size(); ++i) {
        auto R = g->slot_req[i];
        if (R && !R->done) complete(S, R, code);
    }
}

// Cancelled requests give up their slots (between chunks; no copy-out).  Lock released.
int drop_cancelled(serve_handle* S, Group* g) {
    BatchCG& cg = *g->cg;
    for (int i = 0; i < cg.cap; ++i) {
        std::shared_ptr<Request> R;
        {
            std::lock_guard<std::mutex> g2(S->mu);
            R = g->slot_req[i];
            if (!R || !R->cancel || !cg.active[i]) continue;
        }
        const int rc = cg.cancel(i, g->stream);
        if (rc) return rc;
        std::lock_guard<std::mutex> g2(S->mu);
        g->slot_req[i] = nullptr;
        g->slot_rhs[i] = -1;
        if (!R->done) complete(S, R, ODWF_ECANCELED);
    }
    return ODWF_OK;
}

// Hand the group's finished systems back: x into the caller's device buffer (stream-ordered),
// or into a per-slot staging buffer whose copy to the caller's host buffer the copier thread
// does; free the slot, complete requests whose systems are all done.  Lock released.
int harvest(serve_handle* S, Group* g) {
    BatchCG& cg = *g->cg;
    for (int i = 0; i < cg.cap; ++i) {
        if (!cg.active[i] || !cg.slot_finished(i)) continue;
        std::shared_ptr<Request> R;
        {
            std::lock_guard<std::mutex> g2(S->mu);
            R = g->slot_req[i];
        }
        if (!R) {
            cg.release(i);
            continue;
        }
        const int k = g->slot_rhs[i];
        void* xo = R->x[k];
        const size_t eb = g->eng->sites5() * 192;
        int rc = ODWF_OK;
        double2* dx = (double2*)xo;
        const bool host = !is_device_ptr(xo);
        if (host) dx = (double2*)g->eng->get_ws("serve.x" + std::to_string(i), eb, &rc);
        double tr = 0;
        if (!rc) rc = cg.finalize(i, dx, g->stream, &tr);  // synchronizes the group's stream
        if (rc) return rc;
        const int stt = cg.st_host[i].status;
        const int iters = cg.st_host[i].iter;
        cg.release(i);
        int code = ODWF_OK;
        if (stt == kBreakdown) code = ODWF_EBREAKDOWN;
        else if (stt != kDone) code = ODWF_ENOCONV;
        std::lock_guard<std::mutex> g2(S->mu);
        if (host && !R->done) {
            // the slot stays owned by R until the copier has read the staging buffer
            S->copy_jobs.push_back({g, i, R, xo, dx, eb, code, iters, tr});
            ++g->copies;
            S->cv_copy.notify_all();
        } else {
            g->slot_req[i] = nullptr;
            g->slot_rhs[i] = -1;
            if (!R->done) system_done(S, R, code, iters, tr);
        }
        g->last_used = Clock::now();
    }
    return ODWF_OK;
}

// Copier thread: blocking device-to-host copies of finished solutions, off the worker.
void copier_loop(serve_handle* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        S->cv_copy.wait(lk, [&] { return S->copier_stop || !S->copy_jobs.empty(); });
        if (S->copy_jobs.empty() && S->copier_stop) break;
        serve_handle::CopyJob j = S->copy_jobs.front();
        S->copy_jobs.pop_front();
        lk.unlock();
        int rc = ODWF_OK;
        if (cudaMemcpy(j.dst, j.src, j.bytes, cudaMemcpyDeviceToHost) != cudaSuccess) {
            cudaGetLastError();
            rc = ODWF_ECUDA;
        }
        lk.lock();
        --j.g->copies;
        j.g->slot_req[j.slot] = nullptr;
        j.g->slot_rhs[j.slot] = -1;
        if (!j.R->done) system_done(S, j.R, rc ? rc : j.code, j.iters, j.resid);
        S->cv_work.notify_all();
    }
}

void worker_loop(serve_handle* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        // 1. admission in arrival order (a request that does not fit yet waits; later ones
        //    for other groups may still enter).  try_admit drops the lock around device work,
        //    so iterate over a snapshot of the queue.
        std::vector<std::shared_ptr<Request>> snap(S->queue.begin(), S->queue.end());
        const auto now = Clock::now();
        for (auto& R : snap) {
            if (S->stop) break;
            const double waited = std::chrono::duration<double, std::milli>(now - R->t_submit).count();
            if (R->cancel || (S->admit_deadline_ms > 0 && waited > S->admit_deadline_ms)) {
                // cancelled while queued, or shed: waited longer than the admission deadline
                if (!R->cancel) ++S->shed;
                complete(S, R, R->cancel ? ODWF_ECANCELED : ODWF_ETIMEOUT);
                auto it = std::find(S->queue.begin(), S->queue.end(), R);
                if (it != S->queue.end()) S->queue.erase(it);
                continue;
            }
            if (try_admit(S, R, lk)) {
                auto it = std::find(S->queue.begin(), S->queue.end(), R);
                if (it != S->queue.end()) S->queue.erase(it);
            }
        }
        // drop failed groups (their requests were failed; pending copy-outs of the group are
        // abandoned first so that nothing refers to it)
        for (auto it = S->groups.begin(); it != S->groups.end();) {
            Group* g = it->get();
            if (!g->failed) {
                ++it;
                continue;
            }
            for (auto jt = S->copy_jobs.begin(); jt != S->copy_jobs.end();) {
                if (jt->g == g) {
                    --g->copies;
                    jt = S->copy_jobs.erase(jt);
                } else {
                    ++jt;
                }
            }
            if (g->copies > 0) {  // a copy the copier has taken: drop the group once it is done
                ++it;
                continue;
            }
            lk.unlock();
            destroy_group(g);
            lk.lock();
            S->used -= std::min(S->used, g->reserved);
            it = S->groups.erase(it);
        }
        bool any = false;
        for (auto& g : S->groups)
            if (g->cg && g->cg->any_running()) any = true;
        if (S->stop && !any && S->copy_jobs.empty()) break;
        if (!any) {
            // 3. drop idle groups (their memory goes back to the budget), then sleep
            for (auto it = S->groups.begin(); it != S->groups.end();) {
                Group* g = it->get();
                if (g->used_slots() == 0) {
                    lk.unlock();
                    destroy_group(g);
                    lk.lock();
                    S->used -= std::min(S->used, g->reserved);
                    it = S->groups.erase(it);
                } else {
                    ++it;
                }
            }
            if (S->queue.empty() && !S->stop) S->cv_work.wait_for(lk, std::chrono::milliseconds(50));
            else if (!S->queue.empty()) S->cv_work.wait_for(lk, std::chrono::milliseconds(1));
            continue;
        }
        // 2. per group, without blocking: harvest a finished chunk, then launch the next one
        std::vector<Group*> act;
        for (auto& g : S->groups)
            if (g->cg && g->cg->any_running()) act.push_back(g.get());
        lk.unlock();
        bool launched = false;
        NvtxRange nv_("odwf.serve.pass");
        for (Group* g : act) {
            BatchCG& cg = *g->cg;
            int rc = ODWF_OK;
            if (g->in_flight) {
                const cudaError_t q = cudaEventQuery(g->ev_chunk);
                if (q == cudaErrorNotReady) continue;
                g->in_flight = false;
                if (q != cudaSuccess) rc = cuda_fail(q, "serve: iteration chunk");
                if (!rc) rc = cg.poll(g->stream);
                if (!rc) rc = cg.service(g->stream);
                if (!rc) rc = harvest(S, g);
                if (!rc) rc = drop_cancelled(S, g);
            }
            if (!rc && cg.any_running()) {
                if (inject_at() > 0 && ++g_chunks == inject_at())
                    rc = fail(ODWF_ECUDA, "serve: injected failure of a chunk launch (ODWF_SERVE_INJECT_ERROR)");
                if (!rc) rc = cg.resume(g->stream, false);
                if (!rc) rc = cg.run_iterations(kIterChunk, g->stream);
                if (!rc) {
                    const cudaError_t e = cudaEventRecord(g->ev_chunk, g->stream);
                    if (e != cudaSuccess) rc = cuda_fail(e, "serve: cudaEventRecord");
                    else g->in_flight = true;
                }
                launched = true;
            }
            if (rc) {
                std::lock_guard<std::mutex> g2(S->mu);
                fail_group(S, g, rc);
            }
        }
        if (!launched) std::this_thread::sleep_for(std::chrono::microseconds(100));
        lk.lock();
    }
    // fail whatever is still queued, let the copier finish the groups' copy-outs, free the groups
    for (auto& R : S->queue) complete(S, R, ODWF_ETIMEOUT);
    S->queue.clear();
    while (true) {
        int copies = 0;
        for (auto& g : S->groups) copies += g->copies;
        if (!copies) break;
        S->cv_work.wait_for(lk, std::chrono::milliseconds(10));
    }
    lk.unlock();
    for (auto& g : S->groups) destroy_group(g.get());
    lk.lock();
    S->groups.clear();
    lk.unlock();
}

}  // namespace

}  // namespace odwf

using odwf::fail;

extern "C" {

int serve_create(size_t hbm_budget_bytes, serve_handle** out) {
    try {
        if (!out) return fail(ODWF_EINVAL, "serve_create: null out");
        *out = nullptr;
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return fail(ODWF_ECUDA, "serve_create: no CUDA device");
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return fail(ODWF_ECUDA, "serve_create: cudaMemGetInfo failed");
        auto* S = new serve_handle();
        S->device = dev;
        S->budget = hbm_budget_bytes ? hbm_budget_bytes : (size_t)(0.9 * (double)fr);
        S->worker = std::thread(odwf::worker_loop, S);
        S->copier = std::thread(odwf::copier_loop, S);
        *out = S;
        return ODWF_OK;
    } catch (...) {
        return fail(ODWF_ENOMEM, "serve_create: host allocation failed");
    }
}

int serve_register_gauge(serve_handle* S, int field_id, const odwf_lattice* lat, const void* U) {
    if (!S || !lat || !U) return fail(ODWF_EINVAL, "serve_register_gauge: null argument");
    for (int i = 0; i < 4; ++i)
        if (lat->dims[i] < 2 || (lat->dims[i] & 1)) return fail(ODWF_EINVAL, "serve_register_gauge: bad lattice");
    const size_t V = (size_t)lat->dims[0] * lat->dims[1] * lat->dims[2] * lat->dims[3];
    const size_t bytes = V * 4 * 9 * 16;
    std::lock_guard<std::mutex> g(S->mu);
    if (S->fields.count(field_id)) return fail(ODWF_EINVAL, "serve_register_gauge: field id already registered");
    if (S->used + bytes > S->budget) return fail(ODWF_ENOMEM, "serve_register_gauge: over the HBM budget");
    odwf::Field f;
    f.lat = *lat;
    f.bytes = bytes;
    if (cudaMalloc(&f.U, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(ODWF_ENOMEM, "serve_register_gauge: device allocation failed");
    }
    if (cudaMemcpy(f.U, U, bytes, cudaMemcpyDefault) != cudaSuccess) {
        cudaFree(f.U);
        return fail(ODWF_ECUDA, "serve_register_gauge: copy failed");
    }
    S->used += bytes;
    S->fields[field_id] = f;
    return ODWF_OK;
}

int serve_submit(serve_handle* S, const odwf_request* req, uint64_t* ticket) {
    if (!S || !req || !ticket) return fail(ODWF_EINVAL, "serve_submit: null argument");
    if (req->nrhs <= 0 || req->nrhs > odwf::kMaxSlots || !req->b || !req->x || !req->omega)
        return fail(ODWF_EINVAL, "serve_submit: need 1..16 right-hand sides and omega");
    if (req->Ns < 2 || req->Ns > 32 || (req->Ns & (req->Ns - 1)))
        return fail(ODWF_EINVAL, "serve_submit: Ns must be 2, 4, 8, 16 or 32");
    if (!(req->tol > 0) || req->max_iter <= 0 || req->prec < ODWF_F64 || req->prec > ODWF_BF16)
        return fail(ODWF_EINVAL, "serve_submit: bad tol / max_iter / prec");
    auto R = std::make_shared<odwf::Request>();
    R->req = *req;
    R->omega.assign(req->omega, req->omega + req->Ns);
    R->b.assign(req->b, req->b + req->nrhs);
    R->x.assign(req->x, req->x + req->nrhs);
    R->t_submit = odwf::Clock::now();
    std::lock_guard<std::mutex> g(S->mu);
    auto fit = S->fields.find(req->field_id);
    if (fit == S->fields.end()) return fail(ODWF_ENOTFOUND, "serve_submit: unknown field id");
    const odwf_lattice& lat = fit->second.lat;
    const size_t vh = (size_t)lat.dims[0] * lat.dims[1] * lat.dims[2] * lat.dims[3] / 2;
    const size_t need = odwf::group_fixed_bytes(vh, vh * req->Ns) +
                        odwf::per_system_bytes(vh * req->Ns, req->prec) * req->nrhs;
    size_t field_bytes = 0;
    for (auto& kv : S->fields) field_bytes += kv.second.bytes;
    if (need + field_bytes > S->budget) return fail(ODWF_ENOMEM, "serve_submit: request can never fit the HBM budget");
    if (S->max_queued > 0 && (int)S->queue.size() >= S->max_queued) {
        ++S->refused;
        return fail(ODWF_EBUSY, "serve_submit: the queue is full (serve_set_policy max_queued)");
    }
    R->ticket = S->next_ticket++;
    S->tickets[R->ticket] = R;
    S->queue.push_back(R);
    *ticket = R->ticket;
    S->cv_work.notify_all();
    return ODWF_OK;
}

int serve_poll(serve_handle* S, uint64_t ticket, int timeout_ms, odwf_result* res) {
    if (!S) return fail(ODWF_EINVAL, "serve_poll: null handle");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return fail(ODWF_ENOTFOUND, "serve_poll: unknown ticket");
    auto R = it->second;
    if (!R->done && timeout_ms > 0)
        S->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return R->done; });
    if (res) {
        res->status = R->done ? R->status : ODWF_PENDING;
        res->iters = R->iters;
        res->true_resid = R->resid;
        res->latency_ms = R->done ? R->latency_ms
                                  : std::chrono::duration<double, std::milli>(odwf::Clock::now() - R->t_submit).count();
        res->queue_ms = R->admitted ? R->queue_ms : -1.0;
    }
    return R->done ? R->status : ODWF_PENDING;
}

int serve_set_policy(serve_handle* S, double admit_deadline_ms, int max_queued, int fair) {
    if (!S) return fail(ODWF_EINVAL, "serve_set_policy: null handle");
    if (!std::isfinite(admit_deadline_ms)) return fail(ODWF_EINVAL, "serve_set_policy: non-finite deadline");
    std::lock_guard<std::mutex> g(S->mu);
    S->admit_deadline_ms = admit_deadline_ms;
    S->max_queued = max_queued;
    S->fair = fair ? 1 : 0;
    S->cv_work.notify_all();
    return ODWF_OK;
}

int serve_cancel(serve_handle* S, uint64_t ticket) {
    if (!S) return fail(ODWF_EINVAL, "serve_cancel: null handle");
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return fail(ODWF_ENOTFOUND, "serve_cancel: unknown ticket");
    auto& R = it->second;
    if (R->done) return ODWF_OK;  // already finished: its status stands
    R->cancel = true;
    if (!R->admitted) {
        auto q = std::find(S->queue.begin(), S->queue.end(), R);
        if (q != S->queue.end()) S->queue.erase(q);
        odwf::complete(S, R, ODWF_ECANCELED);
    }
    S->cv_work.notify_all();
    return ODWF_OK;
}

int serve_destroy(serve_handle* S) {
    if (!S) return fail(ODWF_EINVAL, "serve_destroy: null handle");
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->copier_stop = true;
        S->cv_copy.notify_all();
    }
    if (S->copier.joinable()) S->copier.join();
    for (auto& kv : S->fields)
        if (kv.second.U) cudaFree(kv.second.U);
    delete S;
    return ODWF_OK;
}

}  // extern "C"
