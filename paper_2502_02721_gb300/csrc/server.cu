// Serving loop behind ipf_server_create / ipf_submit / ipf_poll.
//
// A scheduler thread keeps up to max_inflight requests on the GPU at once.
// A request is admitted when a slot is free and its footprint
// (ipf_footprint) fits in what is left of the server's HBM budget; its
// context then allocates from one device arena reserved at server creation,
// so admission and retirement never call cudaMalloc / cudaFree (no implicit
// device synchronisation while other requests run).  Each admitted request
// has its own context and streams, so the work of all in-flight requests
// overlaps on the device; the scheduler tops up every request with a slice
// of Hessenberg steps whenever its previous slice has finished, enqueues the
// projected solve and the copy of x to pinned host memory after the last
// slice, and retires the request when that copy has landed.
//
// Requests the batched step can drive (one RHS, float storage, sparse-sign
// sketch, full pivoting, a PSF on the FMA or tensor-core path or a CSR
// matrix: see batch.cu) do not step on their own streams: each takes a slot
// of the server's batch engine, and one turn of the engine advances every
// slot by steps_per_slice steps with one launch per phase per step.  When a
// slot has taken its k steps it leaves the batch and its solve runs on the
// request's stream after that turn.  b is staged in pinned host memory that
// the device reads directly, so admitting a request never waits for the GPU.
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "ipf_internal.cuh"

namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// first-fit arena over one device block; used only by the scheduler thread
struct Arena {
    char* base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_;      // offset -> length
    std::map<size_t, size_t> used_;      // offset -> length
    size_t in_use = 0;
    bool pinned = false;
    bool init(size_t bytes, bool host_pinned = false) {
        pinned = host_pinned;
        const cudaError_t e = pinned ? cudaMallocHost((void**)&base, bytes) : cudaMalloc((void**)&base, bytes);
        if (e != cudaSuccess) { base = nullptr; return false; }
        size = bytes;
        free_[0] = bytes;
        return true;
    }
    void* get(size_t bytes) {
        bytes = (bytes + 255) & ~(size_t)255;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, len = it->second;
                free_.erase(it);
                if (len > bytes) free_[off + bytes] = len - bytes;
                used_[off] = bytes;
                in_use += bytes;
                return base + off;
            }
        }
        return nullptr;
    }
    void put(void* p) {
        if (!p) return;
        const size_t off = (size_t)((char*)p - base);
        auto u = used_.find(off);
        if (u == used_.end()) return;
        size_t len = u->second;
        used_.erase(u);
        in_use -= len;
        size_t start = off;
        auto nx = free_.lower_bound(off);
        if (nx != free_.end() && nx->first == off + len) {   // merge with the next hole
            len += nx->second;
            nx = free_.erase(nx);
        }
        if (nx != free_.begin()) {                            // and with the previous one
            auto pv = std::prev(nx);
            if (pv->first + pv->second == off) {
                start = pv->first;
                len += pv->second;
                free_.erase(pv);
            }
        }
        free_[start] = len;
    }
    void release() {
        if (base) { if (pinned) cudaFreeHost(base); else cudaFree(base); }
        base = nullptr;
    }
};

void* arena_alloc(size_t bytes, void* user) { return ((Arena*)user)->get(bytes); }
void arena_free(void* p, void* user) { ((Arena*)user)->put(p); }

struct Job {
    unsigned long long ticket = 0;
    // copied request
    ipf_operator op{};
    std::vector<float> psf, sep_row, sep_col, motion, vals;
    std::vector<long long> rowptr;
    std::vector<int> colind;
    std::vector<float> b;
    float* b_pin = nullptr;                 // pinned copy of b, read by the device
    int slot = -1;                          // batch engine slot, or -1
    int cls = 0;                            // its engine (size class)
    ipf_config cfg{};
    int k = 0;
    double lambda = 0.0;
    size_t footprint = 0;
    long long n = 0;
    // runtime
    ipf_ctx* ctx = nullptr;
    float* x_dev = nullptr;                 // nrhs x n, from the device arena
    float* x_pin = nullptr;                 // nrhs x n, from the pinned arena
    std::vector<float> x;                   // result, copied out at retirement
    cudaStream_t us = nullptr;              // the request's own ordering stream
    cudaEvent_t ev = nullptr;               // completion of the last enqueued work
    int enqueued = 0;
    bool solving = false;
    // result
    ipf_status status = IPF_PENDING;
    int k_used = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;
};

}  // namespace

struct ipf_server {
    ipf_server_config cfg{};
    Arena arena;
    Arena pinned;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::unique_ptr<Job>> pending;
    std::vector<std::unique_ptr<Job>> active;
    std::map<unsigned long long, std::unique_ptr<Job>> done;
    unsigned long long next_ticket = 1;
    std::atomic<bool> stop{false};
    std::thread worker;
    size_t reserved = 0;                     // footprints of active jobs
    int device = 0;
    // the batched step: one engine (stream, work list) per size class, so a
    // small request steps in lockstep only with requests of similar work per
    // step, and the classes' launches overlap on the GPU (NULL with
    // cfg.per_request)
    static constexpr int kClasses = 3;
    ipf::BatchEngine* eng[kClasses] = {};
    std::deque<cudaEvent_t> turns[kClasses]; // engine turns in flight
    std::vector<cudaEvent_t> spare_ev;
    // statistics
    unsigned long long n_done = 0, n_rejected = 0;
    int n_batched = 0;                       // requests that took a batch slot

    void loop();
    bool admit(Job* j);
    void retire(Job* j);
};

bool ipf_server::admit(Job* j) {
    const size_t xb = sizeof(float) * (size_t)j->n * j->cfg.nrhs;
    j->x_pin = (float*)pinned.get(xb);
    if (!j->x_pin) return false;                       // wait for pinned space
    j->b_pin = (float*)pinned.get(sizeof(float) * j->b.size());
    if (!j->b_pin) {
        pinned.put(j->x_pin);
        j->x_pin = nullptr;
        return false;
    }
    memcpy(j->b_pin, j->b.data(), sizeof(float) * j->b.size());
    if (cudaStreamCreateWithFlags(&j->us, cudaStreamNonBlocking) != cudaSuccess) {
        pinned.put(j->x_pin);
        j->x_pin = nullptr;
        return false;
    }
    ipf_config c = j->cfg;
    c.alloc = arena_alloc;
    c.free = arena_free;
    c.alloc_user = &arena;
    c.stream = j->us;                                  // order against this request only
    c.profile = 0;
    // requests in flight already overlap with one another; a second stream
    // per step only adds launches and events (measured: lower capacity and
    // higher latency under load), so a request on its own streams steps on
    // one stream
    c.overlap = 0;
    if (eng[0]) {
        // steps come from the batch engine where it can, which runs the
        // products at the pivot rows beside the operator (step mode 2)
        c.use_graphs = 0;
        c.overlap = 2;
    }
    ipf_ctx* ctx = nullptr;
    // the device reads b from pinned host memory: no wait for the GPU here
    ipf_status st = ipf_create(&j->op, j->b_pin, IPF_MEM_DEVICE, &c, &ctx);
    if (st == IPF_ERR_OOM || (st == IPF_OK && !(j->x_dev = (float*)arena.get(xb)))) {
        if (ctx) ipf_destroy(ctx);
        cudaStreamDestroy(j->us);
        j->us = nullptr;
        pinned.put(j->x_pin);
        j->x_pin = nullptr;
        pinned.put(j->b_pin);
        j->b_pin = nullptr;
        return false;                                  // try again when memory frees up
    }
    j->t_admit = now_s();
    if (st != IPF_OK) {
        j->status = st;
        j->t_done = j->t_admit;
        cudaStreamDestroy(j->us);
        j->us = nullptr;
        pinned.put(j->x_pin);
        j->x_pin = nullptr;
        return true;
    }
    j->ctx = ctx;
    if (cudaEventCreateWithFlags(&j->ev, cudaEventDisableTiming) != cudaSuccess) {
        j->status = IPF_ERR_CUDA;
        retire(j);
        return true;
    }
    // a request the batched step cannot drive steps on its own stream
    // (eagerly); the others go to the engine of their size class: bytes a
    // step moves, about n s_V (k + 1) / 2 of the basis plus the operator's
    if (eng[0]) {
        const double sv = j->cfg.storage == IPF_STORE_F32 ? 4.0 : 2.0;
        double per_step = (double)j->n * sv * (j->k + 1) / 2.0 +
                          (j->op.kind == IPF_OP_CSR ? (double)j->op.nnz * 8.0 : (double)j->n * 8.0);
        j->cls = per_step < 16e6 ? 0 : per_step < 96e6 ? 1 : 2;
        j->slot = ipf::batch_add(eng[j->cls], ctx, j->k, j->us);
    }
    if (j->slot >= 0) ++n_batched;
    return true;
}

void ipf_server::retire(Job* j) {
    if (j->slot >= 0) {
        // still in the batch (an error or shutdown): drop it, and let the
        // turns that read it finish first
        ipf::batch_remove(eng[j->cls], j->slot);
        j->slot = -1;
        for (cudaEvent_t ev : turns[j->cls]) cudaEventSynchronize(ev);
    }
    if (j->ctx) {
        int kd = 0;
        ipf_status st = ipf_sync(j->ctx, &kd);
        if (j->status == IPF_PENDING || j->status == IPF_OK)
            j->status = st < 0 ? st : (kd < j->k ? IPF_BREAKDOWN : IPF_OK);
        j->k_used = kd < j->k ? kd : j->k;
        ipf_destroy(j->ctx);
        j->ctx = nullptr;
    }
    if (j->us) {
        cudaStreamSynchronize(j->us);
        if (j->x_pin && (j->status == IPF_OK || j->status == IPF_BREAKDOWN))
            j->x.assign(j->x_pin, j->x_pin + (size_t)j->n * j->cfg.nrhs);
        cudaStreamDestroy(j->us);
        j->us = nullptr;
    }
    if (j->x_dev) arena.put(j->x_dev);
    j->x_dev = nullptr;
    if (j->x_pin) pinned.put(j->x_pin);
    j->x_pin = nullptr;
    if (j->b_pin) pinned.put(j->b_pin);
    j->b_pin = nullptr;
    if (j->ev) cudaEventDestroy(j->ev);
    j->ev = nullptr;
    j->t_done = now_s();
}

void ipf_server::loop() {
    cudaSetDevice(device);
    const int slice = cfg.steps_per_slice > 0 ? cfg.steps_per_slice : 8;
    while (!stop.load()) {
        bool worked = false;
        // admit while slots and budget allow (FIFO; a request that does not fit waits)
        {
            std::unique_lock<std::mutex> lk(mu);
            while (!pending.empty() && (int)active.size() < cfg.max_inflight) {
                Job* j = pending.front().get();
                if (reserved + j->footprint > cfg.hbm_budget_bytes && !active.empty()) break;
                std::unique_ptr<Job> up = std::move(pending.front());
                pending.pop_front();
                lk.unlock();
                const bool ok = admit(up.get());
                lk.lock();
                if (!ok) {
                    if (active.empty()) {                    // nothing will free memory: give up on it
                        up->status = IPF_ERR_OOM;
                        up->t_admit = up->t_done = now_s();
                        ++n_done;
                        done[up->ticket] = std::move(up);
                        cv.notify_all();
                        continue;
                    }
                    pending.push_front(std::move(up));       // retry when memory frees up
                    break;
                }
                worked = true;
                if (up->status != IPF_PENDING) {
                    ++n_done;
                    done[up->ticket] = std::move(up);
                    cv.notify_all();
                } else {
                    reserved += up->footprint;
                    active.push_back(std::move(up));
                }
            }
        }
        // one turn of each size class's engine (at most two in flight per
        // class); slots that have taken their k steps leave the batch, and
        // their solves (below) follow that turn on their own streams
        for (int cl = 0; cl < kClasses && eng[cl]; ++cl) {
            std::deque<cudaEvent_t>& tq = turns[cl];
            while (!tq.empty() && cudaEventQuery(tq.front()) == cudaSuccess) {
                spare_ev.push_back(tq.front());
                tq.pop_front();
            }
            if (ipf::batch_used(eng[cl]) == 0 || tq.size() >= 2) continue;
            cudaEvent_t ev = nullptr;
            if (!spare_ev.empty()) {
                ev = spare_ev.back();
                spare_ev.pop_back();
            } else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
                ev = nullptr;
            }
            const cudaError_t e = ev ? ipf::batch_run(eng[cl], slice, ev) : cudaErrorMemoryAllocation;
            worked = true;
            if (ev) tq.push_back(ev);
            for (auto& up : active) {
                Job* j = up.get();
                if (j->slot < 0 || j->cls != cl) continue;
                if (e != cudaSuccess) {
                    ipf::batch_remove(eng[cl], j->slot);
                    j->slot = -1;
                    j->status = IPF_ERR_CUDA;
                    j->enqueued = j->k;
                    continue;
                }
                if (ipf::batch_steps(eng[cl], j->slot) < j->k) continue;
                ipf::batch_remove(eng[cl], j->slot);
                j->slot = -1;
                cudaStreamWaitEvent(j->us, ev, 0);
                ipf::ctx_steps_taken(j->ctx, j->k);
                j->enqueued = j->k;
            }
        }
        // top up every in-flight request whose previous work has finished
        for (size_t a = 0; a < active.size();) {
            Job* j = active[a].get();
            if (j->slot >= 0) { ++a; continue; }         // advanced by the batch engine
            if (j->status < 0 && !j->solving) {
                retire(j);
                std::lock_guard<std::mutex> lk(mu);
                reserved -= j->footprint;
                ++n_done;
                done[j->ticket] = std::move(active[a]);
                active.erase(active.begin() + a);
                cv.notify_all();
                continue;
            }
            const bool idle = j->enqueued == 0 || cudaEventQuery(j->ev) == cudaSuccess;
            if (!idle) { ++a; continue; }
            worked = true;
            if (j->solving) {
                retire(j);
                std::lock_guard<std::mutex> lk(mu);
                reserved -= j->footprint;
                ++n_done;
                done[j->ticket] = std::move(active[a]);
                active.erase(active.begin() + a);
                cv.notify_all();
                continue;
            }
            ipf_status st = IPF_OK;
            int kq = 0;
            if (j->enqueued < j->k) {
                const int todo = j->k - j->enqueued < slice ? j->k - j->enqueued : slice;
                st = ipf_step(j->ctx, todo, &kq);
                j->enqueued += todo;
            } else {
                st = ipf_solve(j->ctx, j->k, &j->lambda, 1, j->x_dev, IPF_MEM_DEVICE, nullptr);
                if (st == IPF_OK) {
                    // ipf_solve leaves the request's stream waiting for the solve
                    const size_t xb = sizeof(float) * (size_t)j->n * j->cfg.nrhs;
                    if (cudaMemcpyAsync(j->x_pin, j->x_dev, xb, cudaMemcpyDeviceToHost, j->us) != cudaSuccess)
                        st = IPF_ERR_CUDA;
                }
                j->solving = true;
            }
            if (st < 0) {
                j->status = st;
                retire(j);
                j->status = st;
                std::lock_guard<std::mutex> lk(mu);
                reserved -= j->footprint;
                ++n_done;
                done[j->ticket] = std::move(active[a]);
                active.erase(active.begin() + a);
                cv.notify_all();
                continue;
            }
            cudaEventRecord(j->ev, j->us);
            ++a;
        }
        if (!worked) {
            std::unique_lock<std::mutex> lk(mu);
            cv.wait_for(lk, std::chrono::microseconds(active.empty() ? 2000 : 50));
        }
    }
}

extern "C" {

ipf_status ipf_server_create(const ipf_server_config* cfg, ipf_server** out) {
    if (!out || !cfg) return IPF_ERR_ARG;
    *out = nullptr;
    if (cfg->max_inflight < 1 || cfg->max_inflight > 64) return IPF_ERR_ARG;
    std::unique_ptr<ipf_server> s(new ipf_server());
    s->cfg = *cfg;
    if (cudaGetDevice(&s->device) != cudaSuccess) return IPF_ERR_CUDA;
    if (s->cfg.hbm_budget_bytes == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return IPF_ERR_CUDA;
        s->cfg.hbm_budget_bytes = fr / 10 * 8;
    }
    if (!s->arena.init(s->cfg.hbm_budget_bytes)) return IPF_ERR_OOM;
    if (s->cfg.pinned_bytes == 0) s->cfg.pinned_bytes = (size_t)1 << 30;
    if (!s->pinned.init(s->cfg.pinned_bytes, true)) {
        s->arena.release();
        return IPF_ERR_OOM;
    }
    for (int cl = 0; cl < ipf_server::kClasses && !s->cfg.per_request; ++cl) {
        if (!(s->eng[cl] = ipf::batch_create())) {
            for (int c2 = 0; c2 < cl; ++c2) ipf::batch_destroy(s->eng[c2]);
            s->arena.release();
            s->pinned.release();
            return IPF_ERR_CUDA;
        }
    }
    ipf_server* raw = s.release();
    raw->worker = std::thread([raw] { raw->loop(); });
    *out = raw;
    return IPF_OK;
}

ipf_status ipf_submit(ipf_server* s, const ipf_request* rq, unsigned long long* ticket) {
    if (!s || !rq || !ticket || !rq->b) return IPF_ERR_ARG;
    const ipf_operator& op = rq->op;
    if (op.mem != IPF_MEM_HOST && op.mem != IPF_MEM_DEVICE) return IPF_ERR_ARG;
    if (rq->k < 1 || rq->k > rq->cfg.k_max || !(rq->lambda >= 0.0)) return IPF_ERR_ARG;
    std::unique_ptr<Job> j(new Job());
    j->op = op;
    j->cfg = rq->cfg;
    j->k = rq->k;
    j->lambda = rq->lambda;
    j->n = op.kind == IPF_OP_CSR ? op.cols : (long long)op.rows * op.cols;
    if (j->n < 1 || j->cfg.nrhs < 1 || j->cfg.nrhs > 32) return IPF_ERR_ARG;
    // copy what the request points at: host arrays of the operator and b
    auto cp = [](const float* p, size_t cnt, std::vector<float>& dst) -> const float* {
        if (!p) return nullptr;
        dst.assign(p, p + cnt);
        return dst.data();
    };
    if (op.mem == IPF_MEM_HOST) {
        if (op.kind == IPF_OP_PSF2D) {
            if (!op.psf || op.ph <= 0 || op.pw <= 0) return IPF_ERR_ARG;
            j->op.psf = cp(op.psf, (size_t)op.ph * op.pw, j->psf);
        } else if (op.kind == IPF_OP_PSF2D_SEP_MOTION) {
            if (!op.sep_row || !op.sep_col || !op.motion || op.slen <= 0 || op.mlen <= 0) return IPF_ERR_ARG;
            j->op.sep_row = cp(op.sep_row, op.slen, j->sep_row);
            j->op.sep_col = cp(op.sep_col, op.slen, j->sep_col);
            j->op.motion = cp(op.motion, (size_t)op.mlen * op.mlen, j->motion);
        } else if (op.kind == IPF_OP_CSR) {
            if (!op.rowptr || op.rows <= 0 || op.nnz < 0) return IPF_ERR_ARG;
            j->rowptr.assign(op.rowptr, op.rowptr + op.rows + 1);
            j->op.rowptr = j->rowptr.data();
            if (op.nnz > 0) {
                if (!op.colind || !op.vals) return IPF_ERR_ARG;
                j->colind.assign(op.colind, op.colind + op.nnz);
                j->op.colind = j->colind.data();
                j->op.vals = cp(op.vals, (size_t)op.nnz, j->vals);
            }
        } else {
            return IPF_ERR_ARG;
        }
    } else if (op.kind != IPF_OP_CSR) {
        // device PSF arrays are small: bring them to the host so the request is self-contained
        if (op.kind == IPF_OP_PSF2D) {
            j->psf.resize((size_t)op.ph * op.pw);
            if (cudaMemcpy(j->psf.data(), op.psf, j->psf.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
                return IPF_ERR_CUDA;
            j->op.psf = j->psf.data();
        } else {
            j->sep_row.resize(op.slen);
            j->sep_col.resize(op.slen);
            j->motion.resize((size_t)op.mlen * op.mlen);
            if (cudaMemcpy(j->sep_row.data(), op.sep_row, op.slen * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
                cudaMemcpy(j->sep_col.data(), op.sep_col, op.slen * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
                cudaMemcpy(j->motion.data(), op.motion, j->motion.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
                return IPF_ERR_CUDA;
            j->op.sep_row = j->sep_row.data();
            j->op.sep_col = j->sep_col.data();
            j->op.motion = j->motion.data();
        }
        j->op.mem = IPF_MEM_HOST;
    }
    j->b.assign(rq->b, rq->b + (size_t)j->n * j->cfg.nrhs);
    ipf_config fc = j->cfg;
    // + arena rounding (256 bytes per allocation) and the x buffer
    j->footprint = ipf_footprint(&j->op, &fc) + sizeof(float) * (size_t)j->n * fc.nrhs + (64 << 10);
    if (j->footprint > s->cfg.hbm_budget_bytes || sizeof(float) * (size_t)j->n * fc.nrhs > s->cfg.pinned_bytes) {
        std::lock_guard<std::mutex> lk(s->mu);
        ++s->n_rejected;
        return IPF_ERR_REJECTED;
    }
    j->t_submit = now_s();
    std::lock_guard<std::mutex> lk(s->mu);
    j->ticket = s->next_ticket++;
    *ticket = j->ticket;
    s->pending.push_back(std::move(j));
    s->cv.notify_all();
    return IPF_OK;
}

ipf_status ipf_poll(ipf_server* s, unsigned long long ticket, ipf_result* res, float* x_out) {
    if (!s || !res) return IPF_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->done.find(ticket);
    if (it == s->done.end()) {
        if (ticket == 0 || ticket >= s->next_ticket) return IPF_ERR_ARG;
        res->status = IPF_PENDING;
        return IPF_PENDING;
    }
    Job* j = it->second.get();
    res->status = j->status;
    res->k_used = j->k_used;
    res->t_submit = j->t_submit;
    res->t_admit = j->t_admit;
    res->t_done = j->t_done;
    if (x_out && !j->x.empty()) memcpy(x_out, j->x.data(), sizeof(float) * j->x.size());
    const ipf_status st = j->status;
    s->done.erase(it);
    return st;
}

ipf_status ipf_server_batch_stats(ipf_server* s, int* batched, long long* graph_turns, long long* eager_turns,
                                  long long* captures) {
    if (!s) return IPF_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (batched) *batched = s->n_batched;
    long long g = 0, e = 0, c = 0;
    for (auto* en : s->eng) {
        long long g1 = 0, e1 = 0, c1 = 0;
        if (en) ipf::batch_counters(en, &g1, &e1, &c1);
        g += g1;
        e += e1;
        c += c1;
    }
    if (graph_turns) *graph_turns = g;
    if (eager_turns) *eager_turns = e;
    if (captures) *captures = c;
    return IPF_OK;
}

ipf_status ipf_server_stats(ipf_server* s, int* inflight, int* queued, size_t* hbm_in_use) {
    if (!s) return IPF_ERR_ARG;
    std::lock_guard<std::mutex> lk(s->mu);
    if (inflight) *inflight = (int)s->active.size();
    if (queued) *queued = (int)s->pending.size();
    if (hbm_in_use) *hbm_in_use = s->reserved;
    return IPF_OK;
}

void ipf_server_destroy(ipf_server* s) {
    if (!s) return;
    s->stop.store(true);
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (auto& j : s->active) s->retire(j.get());
    s->active.clear();
    s->done.clear();
    s->pending.clear();
    cudaDeviceSynchronize();
    for (auto& tq : s->turns)
        for (cudaEvent_t ev : tq) cudaEventDestroy(ev);
    for (cudaEvent_t ev : s->spare_ev) cudaEventDestroy(ev);
    for (auto* e : s->eng) ipf::batch_destroy(e);
    s->arena.release();
    s->pinned.release();
    delete s;
}

}  // extern "C"
