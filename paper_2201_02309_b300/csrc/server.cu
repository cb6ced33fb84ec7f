// Serving loop for the reconstruction operator (Sec. II steps 1-7 per
// request): requests of different geometries, volume sizes and precisions
// arrive on the host at any time.  A worker thread admits them as CUDA-stream
// slots and device memory free up (continuous batching: a request that
// arrives while others run starts as soon as a slot and its bytes are free,
// without waiting for a batch boundary), so the copies and kernels of
// several requests overlap on the device.  Plans stay on the device in a
// cache keyed by geometry.  The paper has no serving component; this is the
// operator's deployment form.
//
// Device memory: one arena (a single allocation made when the server starts)
// holds every running request's view window, volume and workspace; a
// first-fit sub-allocator hands out 256-byte aligned blocks.  A request is
// admitted only when its block fits ("admission by HBM").  Plans live
// outside the arena, in a cache with its own byte budget: when a new plan
// pushes the cache over budget, idle plans are evicted least recently used
// first.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "common.cuh"

namespace kats {

// ----------------------------------------------------------------- arena
// First-fit allocator of offsets in [0, size).  Blocks are rounded up to 256
// bytes; a freed block merges with free neighbours.  Host logic only.
class Arena {
public:
    explicit Arena(int64_t size) : size_(size)
    {
        if (size_ > 0) free_[0] = size_;
    }

    int64_t alloc(int64_t bytes)
    {
        if (bytes <= 0) bytes = 1;
        bytes = (bytes + 255) / 256 * 256;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            const int64_t off = it->first, rest = it->second - bytes;
            free_.erase(it);
            if (rest > 0) free_[off + bytes] = rest;
            used_[off] = bytes;
            in_use_ += bytes;
            if (in_use_ > peak_) peak_ = in_use_;
            return off;
        }
        return -1;
    }

    bool release(int64_t off)
    {
        auto u = used_.find(off);
        if (u == used_.end()) return false;
        const int64_t bytes = u->second;
        used_.erase(u);
        in_use_ -= bytes;
        int64_t start = off, len = bytes;
        auto next = free_.lower_bound(off);
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                start = prev->first;
                len += prev->second;
                free_.erase(prev);
            }
        }
        if (next != free_.end() && next->first == off + bytes) {
            len += next->second;
            free_.erase(next);
        }
        free_[start] = len;
        return true;
    }

    int64_t largest_free() const
    {
        int64_t m = 0;
        for (const auto &f : free_) m = f.second > m ? f.second : m;
        return m;
    }
    int64_t size() const { return size_; }
    int64_t in_use() const { return in_use_; }
    int64_t peak() const { return peak_; }

private:
    int64_t size_, in_use_ = 0, peak_ = 0;
    std::map<int64_t, int64_t> free_, used_;  // offset -> bytes
};

// ----------------------------------------------------------------- server
namespace {

enum ReqState { kPending = 0, kRunning = 1, kDone = 2 };

struct PlanEntry {
    kats_plan *plan = nullptr;
    int64_t bytes = 0;
    int users = 0;  // running requests holding the plan
    uint64_t last_use = 0;
    std::string key;
};

struct Request {
    uint64_t id = 0;
    kats_geometry g{};
    std::string key;
    const float *sino = nullptr;
    float *vol = nullptr;
    int precision = KATS_PREC_FP32;
    ReqState state = kPending;
    int status = KATS_OK;
    std::string error;
    int slot = -1, plan_hit = 0;
    bool plan_seen = false;
    int64_t off = -1, bytes = 0;
    PlanEntry *plan = nullptr;
    int bypassed = 0;  // later requests admitted ahead of this one while it was first in line
    double t_submit = 0, t_admit = 0, t_done = 0;
    float gpu_ms = 0;
};

struct Slot {
    cudaStream_t st = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int *h_status = nullptr;  // pinned copy of the plan's device status word after the request
    Request *req = nullptr;
};

std::string geometry_key(const kats_geometry &g)
{
    return std::string(reinterpret_cast<const char *>(&g), sizeof(g));
}

}  // namespace

struct Server {
    kats_server_config cfg{};
    int device = 0;
    char *base = nullptr;
    Arena arena{0};
    std::vector<Slot> slots;
    std::unordered_map<std::string, PlanEntry *> plans;
    int64_t plan_bytes = 0;
    uint64_t use_clock = 0, next_id = 1;
    std::deque<Request *> pending;
    std::unordered_map<uint64_t, Request *> all;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    kats_server_stats st{};

    double now_ms() const
    {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
    int running() const
    {
        int n = 0;
        for (const Slot &s : slots) n += s.req != nullptr;
        return n;
    }
    int free_slot() const
    {
        for (size_t i = 0; i < slots.size(); ++i)
            if (!slots[i].req) return (int)i;
        return -1;
    }

    void complete(Request *r, int status, const std::string &err)
    {
        r->state = kDone;
        r->status = status;
        r->error = err;
        r->t_done = now_ms();
        if (status == KATS_OK)
            st.completed++;
        else
            st.failed++;
        cv_done.notify_all();
    }

    void drop_pending(Request *r)
    {
        for (auto it = pending.begin(); it != pending.end(); ++it)
            if (*it == r) {
                pending.erase(it);
                return;
            }
    }

    // Finished slot: release its memory and plan, record times.
    void retire(Slot &s, int status, const std::string &err)
    {
        Request *r = s.req;
        cudaEventElapsedTime(&r->gpu_ms, s.ev0, s.ev1);
        arena.release(r->off);
        r->plan->users--;
        r->plan->last_use = ++use_clock;
        s.req = nullptr;
        complete(r, status, err);
    }

    bool poll_completions()
    {
        bool progress = false;
        for (Slot &s : slots) {
            if (!s.req) continue;
            const cudaError_t q = cudaEventQuery(s.ev1);
            if (q == cudaErrorNotReady) continue;
            progress = true;
            if (q != cudaSuccess) {
                retire(s, KATS_ECUDA, std::string("request stream: ") + cudaGetErrorString(q));
                continue;
            }
            if (*s.h_status != 0) {
                // a bounded wait in the request's kernels gave up (the word is shared by the
                // plan's concurrent requests, so each of them that saw it reports it)
                cudaMemsetAsync(reinterpret_cast<const Plan *>(s.req->plan->plan)->dev_status, 0, sizeof(int), s.st);
                retire(s, KATS_ETIMEOUT, "a bounded device wait gave up during the request");
            } else {
                retire(s, KATS_OK, "");
            }
        }
        return progress;
    }

    // Idle plans leave, least recently used first, while the cache is over budget.
    void evict_over_budget(std::unique_lock<std::mutex> &lk, const PlanEntry *keep)
    {
        std::vector<PlanEntry *> victims;
        while (plan_bytes > cfg.plan_cache_bytes) {
            PlanEntry *v = nullptr;
            for (auto &kv : plans)
                if (kv.second != keep && kv.second->users == 0 && (!v || kv.second->last_use < v->last_use))
                    v = kv.second;
            if (!v) break;
            plans.erase(v->key);
            plan_bytes -= v->bytes;
            st.plan_evictions++;
            victims.push_back(v);
        }
        if (victims.empty()) return;
        lk.unlock();  // freeing device memory may wait for the device
        for (PlanEntry *v : victims) {
            katsevich_plan_destroy(v->plan);
            delete v;
        }
        lk.lock();
    }

    // The request's plan, built (outside the lock) on a cache miss; null if
    // the geometry is invalid or the build failed (the request is then done).
    PlanEntry *ensure_plan(Request *r, std::unique_lock<std::mutex> &lk)
    {
        auto f = plans.find(r->key);
        if (f != plans.end()) {
            if (!r->plan_seen) {
                r->plan_seen = true;
                r->plan_hit = 1;
                st.plan_hits++;
            }
            f->second->last_use = ++use_clock;
            return f->second;
        }
        lk.unlock();
        kats_plan *kp = nullptr;
        const int rc = katsevich_plan(&r->g, &kp);
        const std::string err = rc ? katsevich_last_error() : "";
        kats_plan_info info{};
        if (!rc) katsevich_plan_info(kp, &info);
        lk.lock();
        if (rc) {
            drop_pending(r);
            complete(r, rc, err);
            return nullptr;
        }
        PlanEntry *pe = new PlanEntry();
        pe->plan = kp;
        pe->bytes = info.plan_bytes;
        pe->last_use = ++use_clock;
        pe->key = r->key;
        plans[r->key] = pe;
        plan_bytes += pe->bytes;
        st.plan_misses++;
        r->plan_seen = true;
        evict_over_budget(lk, pe);
        return pe;
    }

    bool launch(Request *r, PlanEntry *pe, int64_t off, int64_t bytes, int k)
    {
        Slot &s = slots[(size_t)k];
        r->state = kRunning;
        r->slot = k;
        r->off = off;
        r->bytes = bytes;
        r->plan = pe;
        r->t_admit = now_ms();
        pe->users++;
        s.req = r;
        int rc = cudaEventRecord(s.ev0, s.st) == cudaSuccess ? KATS_OK : KATS_ECUDA;
        const Plan &p = *reinterpret_cast<const Plan *>(pe->plan);
        *s.h_status = 0;
        if (!rc) rc = recon_one_host(p, r->precision, r->sino, r->vol, base + off, s.st);
        if (!rc && cudaMemcpyAsync(s.h_status, p.dev_status, sizeof(int), cudaMemcpyDeviceToHost, s.st) != cudaSuccess)
            rc = KATS_ECUDA;
        if (!rc && cudaEventRecord(s.ev1, s.st) != cudaSuccess) rc = KATS_ECUDA;
        if (rc) {
            const std::string err = katsevich_last_error();
            cudaStreamSynchronize(s.st);  // nothing of the request may still use its block
            cudaEventRecord(s.ev1, s.st);
            cudaStreamSynchronize(s.st);
            retire(s, rc, err);
            return false;
        }
        const int n = running();
        if (n > st.max_running) st.max_running = n;
        return true;
    }

    // Admit pending requests in arrival order while slots and memory allow.
    // A request whose block does not fit waits; later requests may go ahead
    // of the first one in line at most cfg.max_bypass times, after which
    // admission waits for it (no starvation of large requests).
    bool admit(std::unique_lock<std::mutex> &lk)
    {
        bool progress = false;
        size_t i = 0;
        while (i < pending.size() && !stop) {
            const int k = free_slot();
            if (k < 0) break;
            Request *head = pending.front();
            Request *r = pending[i];
            if (r != head && head->bypassed >= cfg.max_bypass) break;
            PlanEntry *pe = ensure_plan(r, lk);
            if (!pe) {
                progress = true;
                i = 0;  // r left the queue; restart from the (possibly new) head
                continue;
            }
            if (free_slot() < 0) break;  // the lock was released while the plan was built
            const int64_t bytes = (int64_t)host_item_bytes(*reinterpret_cast<const Plan *>(pe->plan), r->precision);
            if (bytes > arena.size()) {
                drop_pending(r);
                st.refused++;
                char msg[160];
                snprintf(msg, sizeof msg, "the request needs %lld device bytes; the server's arena holds %lld",
                         (long long)bytes, (long long)arena.size());
                complete(r, KATS_ENOMEM, msg);
                progress = true;
                i = 0;
                continue;
            }
            const int64_t off = arena.alloc(bytes);
            if (off < 0) {
                ++i;  // waits for memory; a later, smaller request may fit
                continue;
            }
            pending.erase(pending.begin() + (std::ptrdiff_t)i);
            if (r != head) head->bypassed++;
            launch(r, pe, off, bytes, free_slot());
            progress = true;
            i = 0;
        }
        return progress;
    }

    void run()
    {
        cudaSetDevice(device);
        std::unique_lock<std::mutex> lk(mu);
        for (;;) {
            bool progress = poll_completions();
            if (stop) {
                if (running() == 0) break;
            } else {
                progress = admit(lk) || progress;
            }
            if (!progress) cv_work.wait_for(lk, std::chrono::microseconds(50));
        }
        while (!pending.empty()) {
            Request *r = pending.front();
            pending.pop_front();
            complete(r, KATS_EINVAL, "the server stopped before the request was admitted");
        }
    }
};

}  // namespace kats

using namespace kats;

struct kats_server {
    Server s;
};
struct kats_arena {
    Arena a;
    explicit kats_arena(int64_t n) : a(n) {}
};

extern "C" {

int katsevich_arena_create(int64_t bytes, kats_arena **out)
{
    if (!out || bytes <= 0) {
        set_error("katsevich_arena_create: need a positive size and an output pointer");
        return KATS_EINVAL;
    }
    *out = new kats_arena(bytes);
    return KATS_OK;
}

int64_t katsevich_arena_alloc(kats_arena *a, int64_t bytes) { return a ? a->a.alloc(bytes) : -1; }

int katsevich_arena_free(kats_arena *a, int64_t offset)
{
    if (!a || !a->a.release(offset)) {
        set_error("katsevich_arena_free: offset %lld is not an allocated block", (long long)offset);
        return KATS_EINVAL;
    }
    return KATS_OK;
}

int64_t katsevich_arena_largest_free(const kats_arena *a) { return a ? a->a.largest_free() : -1; }
int64_t katsevich_arena_in_use(const kats_arena *a) { return a ? a->a.in_use() : -1; }
void katsevich_arena_destroy(kats_arena *a) { delete a; }

int katsevich_server_create(const kats_server_config *cfg, kats_server **out)
{
    if (!cfg || !out) {
        set_error("null config or output pointer");
        return KATS_EINVAL;
    }
    *out = nullptr;
    if (cfg->slots < 1 || cfg->slots > 64 || cfg->arena_bytes <= 0 || cfg->plan_cache_bytes < 0 ||
        cfg->max_bypass < 0) {
        set_error("server config: need 1 <= slots <= 64, arena_bytes > 0, plan_cache_bytes >= 0, max_bypass >= 0");
        return KATS_EINVAL;
    }
    kats_server *srv = new kats_server();
    Server &s = srv->s;
    s.cfg = *cfg;
    cudaError_t e = cudaGetDevice(&s.device);
    if (e == cudaSuccess) e = dev_malloc((void **)&s.base, (size_t)cfg->arena_bytes);
    if (e != cudaSuccess) {
        const int rc = cuda_fail(e, "server arena allocation");
        delete srv;
        return rc;
    }
    s.arena = Arena(cfg->arena_bytes);
    s.slots.resize((size_t)cfg->slots);
    for (Slot &sl : s.slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreate(&sl.ev0);
        if (e == cudaSuccess) e = cudaEventCreate(&sl.ev1);
        if (e == cudaSuccess) e = cudaHostAlloc((void **)&sl.h_status, sizeof(int), cudaHostAllocDefault);
    }
    if (e != cudaSuccess) {
        const int rc = cuda_fail(e, "server streams");
        for (Slot &sl : s.slots) {
            if (sl.st) cudaStreamDestroy(sl.st);
            if (sl.ev0) cudaEventDestroy(sl.ev0);
            if (sl.ev1) cudaEventDestroy(sl.ev1);
            if (sl.h_status) cudaFreeHost(sl.h_status);
        }
        cudaFree(s.base);
        delete srv;
        return rc;
    }
    s.st.slots = cfg->slots;
    s.st.arena_bytes = cfg->arena_bytes;
    s.worker = std::thread([&s] { s.run(); });
    *out = srv;
    return KATS_OK;
}

int katsevich_server_submit(kats_server *srv, const kats_geometry *g, const float *host_sino, float *host_vol,
                            int precision, uint64_t *ticket)
{
    if (!srv || !g || !host_sino || !host_vol || !ticket) {
        set_error("null server, geometry, buffer or ticket pointer");
        return KATS_EINVAL;
    }
    if (precision != KATS_PREC_FP32 && precision != KATS_PREC_BF16 && precision != KATS_PREC_FP16) {
        set_error("unknown precision %d", precision);
        return KATS_EINVAL;
    }
    Server &s = srv->s;
    Request *r = new Request();
    r->g = *g;
    r->key = geometry_key(*g);
    r->sino = host_sino;
    r->vol = host_vol;
    r->precision = precision;
    {
        std::lock_guard<std::mutex> lk(s.mu);
        if (s.stop) {
            delete r;
            set_error("the server is stopping");
            return KATS_EINVAL;
        }
        r->id = s.next_id++;
        r->t_submit = s.now_ms();
        s.all[r->id] = r;
        s.pending.push_back(r);
        s.st.submitted++;
    }
    s.cv_work.notify_one();
    *ticket = r->id;
    return KATS_OK;
}

int katsevich_server_wait(kats_server *srv, uint64_t ticket, int64_t timeout_ms, kats_request_stats *stats)
{
    if (!srv) {
        set_error("null server");
        return KATS_EINVAL;
    }
    Server &s = srv->s;
    std::unique_lock<std::mutex> lk(s.mu);
    auto f = s.all.find(ticket);
    if (f == s.all.end()) {
        set_error("unknown ticket %llu", (unsigned long long)ticket);
        return KATS_EINVAL;
    }
    Request *r = f->second;
    const int64_t limit = timeout_ms < 0 ? 0 : timeout_ms;
    if (!s.cv_done.wait_for(lk, std::chrono::milliseconds(limit), [r] { return r->state == kDone; })) {
        set_error("request %llu has not finished after %lld ms (it keeps running; wait again)",
                  (unsigned long long)ticket, (long long)limit);
        return KATS_ETIMEOUT;
    }
    if (stats) {
        stats->status = r->status;
        stats->slot = r->slot;
        stats->plan_hit = r->plan_hit;
        stats->bypassed = r->bypassed;
        stats->t_submit_ms = r->t_submit;
        stats->t_admit_ms = r->t_admit;
        stats->t_done_ms = r->t_done;
        stats->gpu_ms = r->gpu_ms;
        stats->device_bytes = r->bytes;
    }
    const int rc = r->status;
    if (rc) set_error("%s", r->error.c_str());
    s.all.erase(f);
    delete r;
    return rc;
}

int katsevich_server_stats(kats_server *srv, kats_server_stats *out)
{
    if (!srv || !out) {
        set_error("null server or output pointer");
        return KATS_EINVAL;
    }
    Server &s = srv->s;
    std::lock_guard<std::mutex> lk(s.mu);
    s.st.arena_peak_bytes = s.arena.peak();
    s.st.arena_in_use_bytes = s.arena.in_use();
    s.st.plan_cache_used_bytes = s.plan_bytes;
    s.st.plans_cached = (int64_t)s.plans.size();
    s.st.pending = (int32_t)s.pending.size();
    s.st.running = s.running();
    *out = s.st;
    return KATS_OK;
}

void katsevich_server_destroy(kats_server *srv)
{
    if (!srv) return;
    Server &s = srv->s;
    {
        std::lock_guard<std::mutex> lk(s.mu);
        s.stop = true;
    }
    s.cv_work.notify_all();
    if (s.worker.joinable()) s.worker.join();
    for (auto &kv : s.all) delete kv.second;
    for (auto &kv : s.plans) {
        katsevich_plan_destroy(kv.second->plan);
        delete kv.second;
    }
    for (Slot &sl : s.slots) {
        cudaStreamDestroy(sl.st);
        cudaEventDestroy(sl.ev0);
        cudaEventDestroy(sl.ev1);
        cudaFreeHost(sl.h_status);
    }
    cudaFree(s.base);
    delete srv;
}

}  // extern "C"
