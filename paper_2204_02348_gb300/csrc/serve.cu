// Serving loop: continuous batching of reconstruction requests under a fixed HBM budget.
//
// One scheduler thread per server owns the device work.  Submitted requests wait in an arrival-ordered queue;
// a request is admitted as soon as a stream slot is free and the budget arena (one device allocation,
// first-fit with coalescing) can hold its reservation: input frames (the rows holding the windows), the
// requested outputs and the generic path's scratch for one chunk of frames.  A request that does not fit lets
// later ones that do fit go first (no head-of-line blocking), until it has waited DH_SERVER_MAX_WAIT_MS or
// been passed DH_SERVER_MAX_BYPASS times; from then on nothing is admitted before it, so it cannot starve.  An admitted request is queued on its slot's stream as host-to-device copy,
// reconstruction (the same kernels as dh_process_batch, with the handle's device-resident plan and the
// request's own scratch), and device-to-host copies of its outputs, chunk after chunk, followed by an event.
// The scheduler polls the events, releases the reservation and the slot of every finished request, records
// its submit-to-completion latency and wakes its waiters.  Requests that arrive while others are on the device
// are admitted as soon as memory and a slot free up, so their work overlaps on the GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <set>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "runtime.hpp"

namespace dh {
namespace {

constexpr size_t kAlign = 256;
constexpr int kMaxSlots = 64;

size_t align_up(size_t v) { return (v + kAlign - 1) & ~(kAlign - 1); }

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// First-fit allocator over [0, size) with coalescing of freed ranges.
class Arena {
  public:
    explicit Arena(size_t size) : size_(size) {
        if (size) free_[0] = size;
    }
    bool alloc(size_t bytes, size_t* off) {
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes;
                const size_t start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                used_ += bytes;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t used() const { return used_; }

  private:
    size_t size_, used_ = 0;
    std::map<size_t, size_t> free_;
};

struct Req {
    uint64_t id = 0;
    dh_request r{};
    Handle* H = nullptr;
    int chunk = 1;                 // frames per chunk
    size_t b_frames = 0, b_fields = 0, b_coefs = 0, b_scratch = 0, bytes = 0;
    size_t off = 0;
    int status = DH_SUCCESS;
    bool done = false;
    double t_submit = 0, t_admit = 0, t_done = 0;
    int bypassed = 0;              // later requests admitted while this one did not fit
    std::string why;
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;      // after the request's last copy (timing)
    cudaEvent_t ev0 = nullptr;     // before its first copy (timing)
    std::vector<cudaEvent_t> kev;  // pairs around each chunk's kernels (timing), grown as needed
    int kpairs = 0;                // pairs used by the current request
    Req* req = nullptr;
};

}  // namespace
}  // namespace dh

struct dh_server_s {
    int dev = 0;
    unsigned char* base = nullptr;
    size_t budget = 0;
    dh::Arena* arena = nullptr;
    std::vector<dh::Slot> slots;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<dh::Req*> queue;
    std::unordered_map<uint64_t, dh::Req*> reqs;
    uint64_t next_id = 1;
    std::thread th;
    bool stop = false;
    // statistics
    long long submitted = 0, completed = 0, failed = 0, frames = 0, bypassed = 0;
    std::vector<double> lat_ms, wait_ms, kernel_ms, span_ms;
    double t_first = -1, t_last = 0;
    size_t peak_bytes = 0;
    int inflight = 0, peak_inflight = 0;
    int max_bypass = DH_SERVER_MAX_BYPASS, max_wait_ms = DH_SERVER_MAX_WAIT_MS;
};

namespace dh {
namespace {

std::mutex g_servers_mu;
std::set<dh_server_s*> g_servers;

bool valid(dh_server_s* s) {
    std::lock_guard<std::mutex> lk(g_servers_mu);
    return g_servers.count(s) != 0;
}

void finish(dh_server_s* S, Req* r, double t, const Slot* sl = nullptr) {
    r->done = true;
    r->t_done = t;
    if (r->status == DH_SUCCESS) {
        S->completed += 1;
        S->frames += r->r.batch;
        S->lat_ms.push_back(1e3 * (r->t_done - r->t_submit));
        S->wait_ms.push_back(1e3 * (r->t_admit - r->t_submit));
        S->t_last = std::max(S->t_last, t);
        if (sl) {
            // device times from the slot's timing events (all complete: the last one has been reached)
            float span = 0.f, k = 0.f, ktot = 0.f;
            if (cudaEventElapsedTime(&span, sl->ev0, sl->ev) == cudaSuccess) S->span_ms.push_back(span);
            bool ok = true;
            for (int i = 0; i < sl->kpairs && ok; ++i) {
                ok = cudaEventElapsedTime(&k, sl->kev[2 * i], sl->kev[2 * i + 1]) == cudaSuccess;
                ktot += k;
            }
            if (ok) S->kernel_ms.push_back(ktot);
        }
    } else {
        S->failed += 1;
    }
}

// A timing event pair of a slot for one more chunk (created on first use).
bool chunk_events(Slot& sl, cudaEvent_t* a, cudaEvent_t* b) {
    while ((int)sl.kev.size() < 2 * (sl.kpairs + 1)) {
        cudaEvent_t e = nullptr;
        if (cudaEventCreate(&e) != cudaSuccess) return false;
        sl.kev.push_back(e);
    }
    *a = sl.kev[2 * sl.kpairs];
    *b = sl.kev[2 * sl.kpairs + 1];
    sl.kpairs += 1;
    return true;
}

// Queue one admitted request on its slot's stream (called with the server lock held).
void launch(dh_server_s* S, Req* r, Slot& sl) {
    Handle* H = r->H;
    int rc;
    {
        std::lock_guard<std::mutex> hl(H->mu);
        rc = ensure_plan(H);
    }
    sl.kpairs = 0;
    cudaEventRecord(sl.ev0, sl.st);
    if (rc) {
        r->status = rc;
        r->why = "plan: " + std::string(dh_last_error());
        cudaEventRecord(sl.ev, sl.st);
        return;
    }
    const dhk::Plan& P = H->plan;
    unsigned char* base = S->base + r->off;
    unsigned char* d_frames = base;
    unsigned char* d_fields = r->b_fields ? base + r->b_frames : nullptr;
    unsigned char* d_coefs = r->b_coefs ? base + r->b_frames + r->b_fields : nullptr;
    unsigned char* d_scratch = r->b_scratch ? base + r->b_frames + r->b_fields + r->b_coefs : nullptr;
    const size_t esz = r->r.dtype == DH_DTYPE_U16 ? 2 : 4;
    // only the rows holding the windows are uploaded; the kernels run on a plan of the cropped frames
    int row0 = 0, rows = 0;
    window_rows(P, &row0, &rows);
    dhk::Plan Pc = P;
    Pc.height = rows;
    for (int p = 0; p < P.pols; ++p) Pc.pol[p].oy -= row0;
    const size_t full_bytes = (size_t)P.width * P.height * esz;
    const size_t frame_bytes = (size_t)P.width * rows * esz;
    const size_t field_bytes = (size_t)P.pols * P.my * P.m * 8;
    const size_t coef_bytes = (size_t)P.pols * P.modes_out * 8;
    for (int f0 = 0; f0 < r->r.batch && rc == DH_SUCCESS; f0 += r->chunk) {
        const int n = std::min(r->chunk, r->r.batch - f0);
        cudaError_t e = cudaMemcpy2DAsync(d_frames, frame_bytes,
                                          (const unsigned char*)r->r.h_frames + f0 * full_bytes + (size_t)row0 * P.width * esz,
                                          full_bytes, frame_bytes, n, cudaMemcpyHostToDevice, sl.st);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "request frames upload");
            break;
        }
        cudaEvent_t ka = nullptr, kb = nullptr;
        const bool timed = chunk_events(sl, &ka, &kb);
        if (timed) cudaEventRecord(ka, sl.st);
        rc = process_plan(H, Pc, d_frames, r->r.dtype, n, d_fields, d_coefs, d_scratch, r->b_scratch, sl.st);
        if (timed) cudaEventRecord(kb, sl.st);
        if (rc) break;
        if (d_fields) {
            e = cudaMemcpyAsync((unsigned char*)r->r.h_fields + f0 * field_bytes, d_fields, n * field_bytes,
                                cudaMemcpyDeviceToHost, sl.st);
            if (e != cudaSuccess) rc = cuda_fail(e, "request fields download");
        }
        if (d_coefs && rc == DH_SUCCESS) {
            e = cudaMemcpyAsync((unsigned char*)r->r.h_coefs + f0 * coef_bytes, d_coefs, n * coef_bytes,
                                cudaMemcpyDeviceToHost, sl.st);
            if (e != cudaSuccess) rc = cuda_fail(e, "request coefficients download");
        }
    }
    if (rc) {
        r->status = rc;
        r->why = dh_last_error();
    }
    cudaEventRecord(sl.ev, sl.st);
}

void scheduler(dh_server_s* S) {
    cudaSetDevice(S->dev);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        // completions
        for (Slot& sl : S->slots) {
            if (!sl.req) continue;
            const cudaError_t q = cudaEventQuery(sl.ev);
            if (q == cudaErrorNotReady) continue;
            Req* r = sl.req;
            if (q != cudaSuccess && r->status == DH_SUCCESS) {
                r->status = DH_ERROR_CUDA;
                r->why = cudaGetErrorString(q);
            }
            S->arena->release(r->off, r->bytes);
            sl.req = nullptr;
            S->inflight -= 1;
            finish(S, r, now_s(), &sl);
            S->cv_done.notify_all();
        }
        // admissions in arrival order; a request that does not fit lets later ones that fit go first, until it
        // has waited or been passed enough (then nothing is admitted before it)
        if (!S->stop) {
            const double tnow = now_s();
            auto it = S->queue.begin();
            while (it != S->queue.end()) {
                Slot* free_slot = nullptr;
                for (Slot& sl : S->slots)
                    if (!sl.req) {
                        free_slot = &sl;
                        break;
                    }
                if (!free_slot) break;
                Req* r = *it;
                size_t off = 0;
                if (!S->arena->alloc(r->bytes, &off)) {
                    if (r->bypassed >= S->max_bypass || 1e3 * (tnow - r->t_submit) >= S->max_wait_ms) break;
                    ++it;
                    continue;
                }
                // every earlier request still queued is passed by this one
                for (auto jt = S->queue.begin(); jt != it; ++jt) (*jt)->bypassed += 1;
                if (it != S->queue.begin()) S->bypassed += 1;
                it = S->queue.erase(it);
                r->off = off;
                r->t_admit = tnow;
                free_slot->req = r;
                S->inflight += 1;
                S->peak_inflight = std::max(S->peak_inflight, S->inflight);
                S->peak_bytes = std::max(S->peak_bytes, S->arena->used());
                launch(S, r, *free_slot);
            }
        }
        if (S->stop) {
            while (!S->queue.empty()) {
                Req* r = S->queue.front();
                S->queue.pop_front();
                r->status = DH_ERROR_ERROR;
                r->why = "server destroyed before the request was admitted";
                finish(S, r, now_s());
            }
            S->cv_done.notify_all();
            if (S->inflight == 0) break;
        }
        if (S->inflight > 0) {
            lk.unlock();
            std::this_thread::sleep_for(std::chrono::microseconds(20));
            lk.lock();
        } else {
            S->cv_work.wait_for(lk, std::chrono::milliseconds(5));
        }
    }
}

}  // namespace
}  // namespace dh

using namespace dh;

extern "C" {

int dh_server_create(size_t hbm_budget, int max_inflight, dh_server* out) {
    if (!out) return fail(DH_ERROR_NULLPOINTER, "out is null");
    if (max_inflight < 1 || max_inflight > kMaxSlots) return fail(DH_ERROR_INVALIDARGUMENT, "max_inflight must be in 1..64");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
    dh_server_s* S = new dh_server_s();
    S->dev = dev;
    S->budget = hbm_budget & ~(kAlign - 1);
    if (S->budget) {
        e = cudaMalloc(&S->base, S->budget);
        if (e != cudaSuccess) {
            delete S;
            return fail(DH_ERROR_MEMORYALLOCATION, std::string("server budget: ") + cudaGetErrorString(e));
        }
    }
    S->arena = new Arena(S->budget);
    S->slots.resize(max_inflight);
    for (Slot& sl : S->slots) {
        e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreate(&sl.ev);
        if (e == cudaSuccess) e = cudaEventCreate(&sl.ev0);
        if (e != cudaSuccess) {
            for (Slot& s2 : S->slots) {
                if (s2.st) cudaStreamDestroy(s2.st);
                if (s2.ev) cudaEventDestroy(s2.ev);
                if (s2.ev0) cudaEventDestroy(s2.ev0);
            }
            if (S->base) cudaFree(S->base);
            delete S->arena;
            delete S;
            return cuda_fail(e, "server streams");
        }
    }
    {
        std::lock_guard<std::mutex> lk(g_servers_mu);
        g_servers.insert(S);
    }
    S->th = std::thread(scheduler, S);
    *out = S;
    return DH_SUCCESS;
}

int dh_server_set_admission(dh_server s, int max_bypass, int max_wait_ms) {
    if (!valid(s)) return fail(DH_ERROR_INVALIDHANDLE, "invalid server");
    if (max_bypass < 0 || max_wait_ms < 0) return fail(DH_ERROR_INVALIDARGUMENT, "admission limits must be >= 0");
    std::lock_guard<std::mutex> lk(s->mu);
    s->max_bypass = max_bypass;
    s->max_wait_ms = max_wait_ms;
    return DH_SUCCESS;
}

int dh_server_submit(dh_server s, const dh_request* r, uint64_t* ticket) {
    if (!valid(s)) return fail(DH_ERROR_INVALIDHANDLE, "invalid server");
    if (!r || !ticket || !r->h_frames) return fail(DH_ERROR_NULLPOINTER, "null request, ticket or frames");
    if (r->dtype != DH_DTYPE_U16 && r->dtype != DH_DTYPE_F32) return fail(DH_ERROR_INVALIDARGUMENT, "bad dtype");
    if (r->batch < 1) return fail(DH_ERROR_INVALIDDIMENSION, "request batch must be >= 1");
    Handle* H = get_handle(r->geometry);
    if (!H) return fail(DH_ERROR_INVALIDHANDLE, "request geometry handle is invalid");
    Geometry g;
    std::string why;
    int rc;
    {
        std::lock_guard<std::mutex> hl(H->mu);
        rc = build_geometry(H->s, &g, &why);
        if (rc == DH_SUCCESS) rc = ensure_plan(H);
    }
    if (rc) return rc == DH_ERROR_CUDA || rc == DH_ERROR_MEMORYALLOCATION ? rc : fail(rc, why.empty() ? dh_last_error() : why);
    const dhk::Plan P = H->plan;
    Req* q = new Req();
    q->r = *r;
    q->H = H;
    const size_t esz = r->dtype == DH_DTYPE_U16 ? 2 : 4;
    int row0 = 0, rows = 0;
    window_rows(P, &row0, &rows);
    const size_t frame = (size_t)P.width * rows * esz;   // the uploaded rows of one frame
    const size_t field = r->h_fields ? (size_t)P.pols * P.my * P.m * 8 : 0;
    const size_t coef = (r->h_coefs && P.modes) ? (size_t)P.pols * P.modes_out * 8 : 0;
    // the fused path needs no scratch; frames staged in the arena are 256-byte aligned, so only the row pitch
    // decides whether tensor copies apply
    const bool fused = fused_allowed(H, P) && fused_layout_ok(P, r->dtype);
    const size_t scratch = (fused ? 0 : split_window_bytes(P) * P.pols) + (coef ? basis_scratch_bytes(P) : 0);
    const size_t per_frame = frame + field + coef + scratch;
    const size_t cap = std::max(s->budget / 2, per_frame);
    if (align_up(frame) + align_up(field) + align_up(coef) + align_up(scratch) > s->budget) {
        delete q;
        return fail(DH_ERROR_MEMORYALLOCATION, "one frame of this request does not fit the server's HBM budget");
    }
    int chunk = (int)std::min<size_t>((size_t)r->batch, std::max<size_t>(1, cap / per_frame));
    for (;; --chunk) {
        q->b_frames = align_up(chunk * frame);
        q->b_fields = align_up(chunk * field);
        q->b_coefs = align_up(chunk * coef);
        q->b_scratch = align_up(chunk * scratch);
        q->bytes = q->b_frames + q->b_fields + q->b_coefs + q->b_scratch;
        if (q->bytes <= s->budget || chunk == 1) break;
    }
    q->chunk = chunk;
    if (!r->h_coefs || !P.modes) q->r.h_coefs = nullptr;
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) {
        delete q;
        return fail(DH_ERROR_ERROR, "server is shutting down");
    }
    q->id = s->next_id++;
    q->t_submit = now_s();
    if (s->t_first < 0) s->t_first = q->t_submit;
    s->submitted += 1;
    s->reqs[q->id] = q;
    s->queue.push_back(q);
    *ticket = q->id;
    s->cv_work.notify_one();
    return DH_SUCCESS;
}

int dh_server_wait(dh_server s, uint64_t ticket, int timeout_ms) {
    if (!valid(s)) return fail(DH_ERROR_INVALIDHANDLE, "invalid server");
    std::unique_lock<std::mutex> lk(s->mu);
    auto it = s->reqs.find(ticket);
    if (it == s->reqs.end()) return fail(DH_ERROR_INVALIDARGUMENT, "unknown or already collected ticket");
    Req* r = it->second;
    auto pred = [&] { return r->done; };
    if (timeout_ms < 0) {
        s->cv_done.wait(lk, pred);
    } else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) {
        return fail(DH_ERROR_TIMEOUT, "request still running");
    }
    const int st = r->status;
    const std::string why = r->why;
    s->reqs.erase(it);
    delete r;
    if (st != DH_SUCCESS) return fail(st, why);
    return DH_SUCCESS;
}

int dh_server_stats(dh_server s, dh_stats* out) {
    if (!valid(s)) return fail(DH_ERROR_INVALIDHANDLE, "invalid server");
    if (!out) return fail(DH_ERROR_NULLPOINTER, "out is null");
    std::lock_guard<std::mutex> lk(s->mu);
    dh_stats st{};
    st.submitted = s->submitted;
    st.completed = s->completed;
    st.failed = s->failed;
    st.frames = s->frames;
    auto pct = [](std::vector<double> l, double p) {
        if (l.empty()) return 0.0;
        std::sort(l.begin(), l.end());
        const size_t i = (size_t)std::ceil(p * l.size()) - 1;
        return l[std::min(i, l.size() - 1)];
    };
    if (!s->lat_ms.empty()) {
        st.p50_ms = pct(s->lat_ms, 0.50);
        st.p99_ms = pct(s->lat_ms, 0.99);
        st.max_ms = pct(s->lat_ms, 1.0);
    }
    st.wait_p50_ms = pct(s->wait_ms, 0.50);
    st.wait_p99_ms = pct(s->wait_ms, 0.99);
    st.kernel_p50_ms = pct(s->kernel_ms, 0.50);
    st.kernel_p99_ms = pct(s->kernel_ms, 0.99);
    st.span_p50_ms = pct(s->span_ms, 0.50);
    st.span_p99_ms = pct(s->span_ms, 0.99);
    for (double k : s->kernel_ms) st.kernel_ms_total += k;
    st.bypassed = s->bypassed;
    st.frames_per_s = (s->frames > 0 && s->t_last > s->t_first) ? s->frames / (s->t_last - s->t_first) : 0.0;
    st.budget_bytes = s->budget;
    st.peak_bytes = s->peak_bytes;
    st.max_inflight = (int)s->slots.size();
    st.peak_inflight = s->peak_inflight;
    *out = st;
    return DH_SUCCESS;
}

int dh_server_destroy(dh_server s) {
    {
        std::lock_guard<std::mutex> lk(g_servers_mu);
        if (!g_servers.count(s)) return fail(DH_ERROR_INVALIDHANDLE, "invalid server");
        g_servers.erase(s);
    }
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_work.notify_all();
    if (s->th.joinable()) s->th.join();
    for (Slot& sl : s->slots) {
        if (sl.st) cudaStreamSynchronize(sl.st);
        if (sl.st) cudaStreamDestroy(sl.st);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.ev0) cudaEventDestroy(sl.ev0);
        for (cudaEvent_t e : sl.kev) cudaEventDestroy(e);
    }
    for (auto& kv : s->reqs) delete kv.second;
    if (s->base) cudaFree(s->base);
    delete s->arena;
    delete s;
    return DH_SUCCESS;
}

}  // extern "C"
