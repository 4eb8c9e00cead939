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
#include <algorithm>
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
    std::vector<std::shared_ptr<Request>> slot_req;  // owner of each slot
    std::vector<int> slot_rhs;
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
    std::string worker_error;
};

namespace odwf {

namespace {

constexpr int kMaxSlots = 16;
constexpr int kIterChunk = 8;

size_t per_system_bytes(size_t sites5, int prec) {
    if (prec == ODWF_F64) return sites5 * 192 * 7;
    const size_t lowb = prec == ODWF_F32 ? 96 : 52;
    // FP64 x, a device copy of a host b, FP32 r and x, five low-precision fields
    return sites5 * (192 * 2 + 96 * 2 + lowb * 5);
}

size_t group_fixed_bytes(size_t vh, size_t sites5) {
    return 8 * vh * (144 + 80 + 48) + sites5 * 192 * 6 + (1 << 20);  // links, FP64 temporaries, scratch
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

// Hand the group's finished systems back: copy x out, free the slot, complete requests
// whose systems are all done.  Called from the worker with the serve lock released.
void harvest(serve_handle* S, Group* g) {
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
        if (host) dx = (double2*)g->eng->get_ws("serve.x", eb, &rc);
        double tr = 0;
        if (!rc) rc = cg.finalize(i, dx, g->stream, &tr);
        if (!rc && host) {
            if (cudaMemcpyAsync(xo, dx, eb, cudaMemcpyDeviceToHost, g->stream) != cudaSuccess ||
                cudaStreamSynchronize(g->stream) != cudaSuccess)
                rc = ODWF_ECUDA;
        }
        const int stt = cg.st_host[i].status;
        const int iters = cg.st_host[i].iter;
        cg.release(i);
        std::lock_guard<std::mutex> g2(S->mu);
        g->slot_req[i] = nullptr;
        g->slot_rhs[i] = -1;
        R->iters = std::max(R->iters, iters);
        R->resid = std::max(R->resid, tr);
        int code = rc;
        if (!code && stt == kBreakdown) code = ODWF_EBREAKDOWN;
        if (!code && stt != kDone) code = ODWF_ENOCONV;
        if (code && R->status == ODWF_PENDING) R->status = code;
        if (--R->remaining == 0) complete(S, R, R->status == ODWF_PENDING ? ODWF_OK : R->status);
        g->last_used = Clock::now();
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
        for (auto& R : snap) {
            if (S->stop) break;
            if (try_admit(S, R, lk)) {
                auto it = std::find(S->queue.begin(), S->queue.end(), R);
                if (it != S->queue.end()) S->queue.erase(it);
            }
        }
        bool any = false;
        for (auto& g : S->groups)
            if (g->cg && g->cg->any_running()) any = true;
        if (S->stop && !any) break;
        if (!any) {
            // 3. drop idle groups (their memory goes back to the budget), then sleep
            for (auto it = S->groups.begin(); it != S->groups.end();) {
                Group* g = it->get();
                if (g->used_slots() == 0) {
                    lk.unlock();
                    if (g->stream) cudaStreamSynchronize(g->stream);
                    g->cg.reset();
                    g->eng.reset();
                    if (g->ev_chunk) cudaEventDestroy(g->ev_chunk);
                    if (g->stream) cudaStreamDestroy(g->stream);
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
        for (Group* g : act) {
            BatchCG& cg = *g->cg;
            if (g->in_flight) {
                const cudaError_t q = cudaEventQuery(g->ev_chunk);
                if (q == cudaErrorNotReady) continue;
                g->in_flight = false;
                if (cg.poll(g->stream)) continue;
                cg.service(g->stream);
                harvest(S, g);
            }
            if (!cg.any_running()) continue;
            cg.resume(g->stream, false);
            cg.run_iterations(kIterChunk, g->stream);
            if (cudaEventRecord(g->ev_chunk, g->stream) == cudaSuccess) g->in_flight = true;
            launched = true;
        }
        if (!launched) std::this_thread::sleep_for(std::chrono::microseconds(100));
        lk.lock();
    }
    // fail whatever is still queued
    for (auto& R : S->queue) complete(S, R, ODWF_ETIMEOUT);
    S->queue.clear();
    lk.unlock();
    for (auto& g : S->groups) {
        if (g->stream) cudaStreamSynchronize(g->stream);
        g->cg.reset();
        g->eng.reset();
        if (g->ev_chunk) cudaEventDestroy(g->ev_chunk);
        if (g->stream) cudaStreamDestroy(g->stream);
    }
    S->groups.clear();
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

int serve_destroy(serve_handle* S) {
    if (!S) return fail(ODWF_EINVAL, "serve_destroy: null handle");
    {
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
        S->cv_work.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    for (auto& kv : S->fields)
        if (kv.second.U) cudaFree(kv.second.U);
    delete S;
    return ODWF_OK;
}

}  // extern "C"
