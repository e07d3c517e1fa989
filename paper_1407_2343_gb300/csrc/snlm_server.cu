// Native serving loop (declared in include/snlm.h, snlm_server_*): continuous
// batching of denoise requests that arrive over time, with no counterpart in the
// paper. The caller submits requests (host images and host result buffers, each
// with an arrival time on the server's clock) and drains the server; the calling
// thread then runs the loop:
//
//  1. arrivals join a FIFO queue when their time has come;
//  2. on every free stream a launch is formed from the front of the queue, as long
//     as its device footprint fits in the server's slab: a request of at least
//     solo_pixels pixels (or a lone request on an idle GPU) runs alone through the
//     per-image path, otherwise the consecutive small requests at the front become
//     one batch plan (the launch over their tile units). The launch
//     copies its inputs in, runs, and copies its results out to the callers' host
//     buffers, all on its stream, then records an event;
//  3. launches whose event has completed are retired: completion time, status,
//     their slab memory returned.
// Streams run concurrently, so requests admitted while others are on the GPU
// overlap with them. In plain mode the same loop serves one request at a time
// through the per-image path and waits for each (the per-request baseline).
#include <string.h>

#include <algorithm>
#include <chrono>
#include <iterator>
#include <map>
#include <thread>
#include <vector>

#include "../../include/snlm.h"
#include "snlm_host.h"

namespace {

// First-fit allocator over one device slab; offsets are 256-byte aligned.
struct Slab {
    char *base = nullptr;
    size_t size = 0;
    std::map<size_t, size_t> free_;   // offset -> bytes

    bool init(size_t bytes)
    {
        bytes = snlm::align_up(bytes, 256);
        if (cudaMalloc(&base, bytes) != cudaSuccess) {
            cudaGetLastError();
            base = nullptr;
            return false;
        }
        size = bytes;
        free_[0] = bytes;
        return true;
    }
    void *alloc(size_t bytes)
    {
        bytes = snlm::align_up(bytes ? bytes : 1, 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                const size_t off = it->first, rest = it->second - bytes;
                free_.erase(it);
                if (rest)
                    free_[off + bytes] = rest;
                return base + off;
            }
        }
        return nullptr;
    }
    size_t largest_free() const
    {
        size_t m = 0;
        for (const auto &e : free_)
            m = std::max(m, e.second);
        return m;
    }
    void release(void *p, size_t bytes)
    {
        bytes = snlm::align_up(bytes ? bytes : 1, 256);
        size_t off = (size_t)(static_cast<char *>(p) - base);
        auto next = free_.lower_bound(off);
        if (next != free_.end() && off + bytes == next->first) {
            bytes += next->second;
            next = free_.erase(next);
        }
        if (next != free_.begin()) {
            auto prev = std::prev(next);
            if (prev->first + prev->second == off) {
                prev->second += bytes;
                return;
            }
        }
        free_[off] = bytes;
    }
    ~Slab()
    {
        if (base)
            cudaFree(base);
    }
};

struct Req {
    snlm_serve_request r;
    double t_done = -1.0;
    int launch = -1;
};

struct Alloc {
    void *p;
    size_t bytes;
};

struct Launch {
    int stream = -1;
    cudaEvent_t done = nullptr;
    std::vector<int> members;
    std::vector<Alloc> mem;
    snlm_batch_plan *plan = nullptr;
};

size_t in_bytes(const snlm_serve_request &r) { return (size_t)r.H * r.W * snlm::dtype_size(r.dtype); }
size_t out_bytes(const snlm_serve_request &r) { return (size_t)r.H * r.W * sizeof(float); }
size_t footprint(const snlm_serve_request &r)
{
    return snlm::align_up(in_bytes(r), 256) + snlm::align_up(out_bytes(r), 256) +
           snlm::align_up(snlm_workspace_bytes(r.H, r.W, r.order), 256);
}

}  // namespace

struct snlm_server {
    snlm_server_config cfg;
    int device = 0;
    Slab slab;
    std::vector<cudaStream_t> streams;
    std::vector<char> busy;
    std::vector<char> high;       // stream created with the device's highest priority
    int *status = nullptr;        // pinned: the failure word of each stream's batch launch
    std::vector<Req> reqs;
    std::vector<int> order;       // submitted ids by arrival time
    size_t next = 0;              // next entry of `order` not yet arrived
    std::vector<int> queue;       // arrived, not launched (FIFO)
    std::vector<Launch> inflight;
    std::chrono::steady_clock::time_point t0;
    bool started = false;
    size_t used = 0;
    snlm_server_stats st;

    double clock() const
    {
        return started ? std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() : 0.0;
    }
};

namespace {

void release_launch(snlm_server *s, Launch &L)
{
    for (const Alloc &a : L.mem)
        s->slab.release(a.p, a.bytes);
    L.mem.clear();
    if (L.plan)
        snlm_batch_plan_destroy(L.plan);
    L.plan = nullptr;
    if (L.done)
        cudaEventDestroy(L.done);
    L.done = nullptr;
}

// Allocate a request's input and output, copy the input in. False if the slab
// has no room (nothing allocated then).
bool stage_request(snlm_server *s, Launch &L, const snlm_serve_request &r, cudaStream_t st, void **d_in,
                   float **d_out)
{
    void *a = s->slab.alloc(in_bytes(r));
    if (!a)
        return false;
    void *b = s->slab.alloc(out_bytes(r));
    if (!b) {
        s->slab.release(a, in_bytes(r));
        return false;
    }
    L.mem.push_back({a, in_bytes(r)});
    L.mem.push_back({b, out_bytes(r)});
    const size_t es = snlm::dtype_size(r.dtype);
    // a dense image goes as one linear copy; only a pitched one needs the 2-D form
    // (one row per copy-engine line)
    if (r.pitch == r.W)
        cudaMemcpyAsync(a, r.img, in_bytes(r), cudaMemcpyHostToDevice, st);
    else
        cudaMemcpy2DAsync(a, (size_t)r.W * es, r.img, (size_t)r.pitch * es, (size_t)r.W * es, (size_t)r.H,
                          cudaMemcpyHostToDevice, st);
    *d_in = a;
    *d_out = static_cast<float *>(b);
    return true;
}

// Launch one request alone (per-image path). Returns SNLM_OK, or SNLM_ERR_NOMEM
// when it does not fit now (nothing launched), or another error.
int launch_solo(snlm_server *s, int id, int si, Launch &L)
{
    const snlm_serve_request &r = s->reqs[id].r;
    cudaStream_t st = s->streams[si];
    const size_t wsb = snlm_workspace_bytes(r.H, r.W, r.order);
    void *ws = s->slab.alloc(wsb);
    if (!ws)
        return SNLM_ERR_NOMEM;
    L.mem.push_back({ws, wsb});
    void *d_in = nullptr;
    float *d_out = nullptr;
    if (!stage_request(s, L, r, st, &d_in, &d_out)) {
        release_launch(s, L);
        return SNLM_ERR_NOMEM;
    }
    const int rc = snlm_denoise_ws(d_in, r.dtype, r.H, r.W, r.W, r.S, r.K, r.h, r.profile, r.order, r.sigma,
                                   r.beta, d_out, ws, wsb, nullptr, st);
    if (rc != SNLM_OK) {
        cudaStreamSynchronize(st);
        release_launch(s, L);
        return rc;
    }
    cudaMemcpyAsync(r.out, d_out, out_bytes(r), cudaMemcpyDeviceToHost, st);
    L.members.push_back(id);
    return SNLM_OK;
}

snlm_request batch_request(const snlm_serve_request &r, const void *d_in, float *d_out)
{
    snlm_request q;
    q.img = d_in;
    q.out = d_out;
    q.dtype = r.dtype;
    q.H = r.H;
    q.W = r.W;
    q.pitch = r.W;
    q.S = r.S;
    q.K = r.K;
    q.h = r.h;
    q.profile = r.profile;
    q.order = r.order;
    q.sigma = r.sigma;
    q.beta = r.beta;
    return q;
}

// Scratch of a batch plan over the given requests (host only: the plan is built
// on placeholder pointers and discarded). 0 on failure.
size_t batch_scratch(const std::vector<snlm_request> &proto, size_t k, int ctas_per_sm)
{
    snlm_batch_config bc;
    bc.ctas_per_sm = ctas_per_sm;
    bc.queue_order = 0;
    bc.spin_limit_us = 0;
    bc.fail_job = -1;
    snlm_batch_plan *plan = nullptr;
    if (snlm_batch_plan_create(proto.data(), (int)k, &bc, &plan) != SNLM_OK)
        return 0;
    const size_t b = snlm_batch_plan_workspace_bytes(plan);
    snlm_batch_plan_destroy(plan);
    return b;
}

// Launch the longest prefix of `ids` that fits in the largest free block of the
// slab as one batch plan; `n_ok` receives its length. SNLM_ERR_NOMEM (nothing
// staged, nothing launched) when not even one request fits now.
int launch_batch(snlm_server *s, const std::vector<int> &ids, int si, Launch &L, int *n_ok)
{
    cudaStream_t st = s->streams[si];
    *n_ok = 0;
    // size first, on placeholder pointers: inputs + outputs + the plan's scratch
    std::vector<snlm_request> proto;
    for (int id : ids)
        proto.push_back(batch_request(s->reqs[id].r, reinterpret_cast<const void *>(256),
                                      reinterpret_cast<float *>(256)));
    const size_t avail = s->slab.largest_free();
    size_t k = 0, io = 0;
    for (; k < ids.size(); ++k) {
        const snlm_serve_request &r = s->reqs[ids[k]].r;
        const size_t add = snlm::align_up(in_bytes(r), 256) + snlm::align_up(out_bytes(r), 256) +
                           snlm::align_up(snlm_workspace_bytes(r.H, r.W, r.order), 256) * 2;
        if (io + add > avail)
            break;
        io += add;
    }
    while (k > 0) {
        size_t need = snlm::align_up(batch_scratch(proto, k, s->cfg.ctas_per_sm), 256);
        for (size_t i = 0; i < k; ++i) {
            const snlm_serve_request &r = s->reqs[ids[i]].r;
            need += snlm::align_up(in_bytes(r), 256) + snlm::align_up(out_bytes(r), 256);
        }
        if (need <= avail)
            break;
        --k;
    }
    if (k == 0)
        return SNLM_ERR_NOMEM;
    // stage (every allocation fits: their total is at most the largest free block)
    std::vector<snlm_request> br;
    for (size_t i = 0; i < k; ++i) {
        const snlm_serve_request &r = s->reqs[ids[i]].r;
        void *d_in = nullptr;
        float *d_out = nullptr;
        if (!stage_request(s, L, r, st, &d_in, &d_out)) {
            cudaStreamSynchronize(st);
            release_launch(s, L);
            return SNLM_ERR_NOMEM;
        }
        br.push_back(batch_request(r, d_in, d_out));
    }
    snlm_batch_config bc;
    bc.ctas_per_sm = s->cfg.ctas_per_sm;
    bc.queue_order = 0;
    bc.spin_limit_us = 0;
    bc.fail_job = -1;
    snlm_batch_plan *plan = nullptr;
    int rc = snlm_batch_plan_create(br.data(), (int)br.size(), &bc, &plan);
    size_t wsb = 0;
    void *ws = nullptr;
    if (rc == SNLM_OK) {
        L.plan = plan;
        wsb = snlm_batch_plan_workspace_bytes(plan);
        ws = s->slab.alloc(wsb);
        if (!ws)
            rc = SNLM_ERR_NOMEM;
    }
    if (rc == SNLM_OK) {
        L.mem.push_back({ws, wsb});
        rc = snlm_batch_plan_upload(plan, ws, wsb, st);
    }
    if (rc == SNLM_OK)
        rc = snlm_batch_plan_launch(plan, st);
    // the run's failure word lands in pinned memory behind it on the stream: read once
    // the launch's event has completed, without a blocking readback in the loop
    if (rc == SNLM_OK)
        rc = snlm_batch_plan_status_async(plan, &s->status[si], st);
    if (rc != SNLM_OK) {
        cudaStreamSynchronize(st);
        release_launch(s, L);
        return rc;
    }
    for (size_t i = 0; i < br.size(); ++i) {
        const snlm_serve_request &r = s->reqs[ids[i]].r;
        cudaMemcpyAsync(r.out, br[i].out, out_bytes(r), cudaMemcpyDeviceToHost, st);
        L.members.push_back(ids[i]);
    }
    *n_ok = (int)br.size();
    return SNLM_OK;
}

// A free stream, of the high-priority half for small launches and of the
// low-priority half for large ones when one is free, else any free stream.
int free_stream(const snlm_server *s, bool small)
{
    int any = -1;
    for (size_t i = 0; i < s->busy.size(); ++i)
        if (!s->busy[i]) {
            if ((s->high[i] != 0) == small)
                return (int)i;
            if (any < 0)
                any = (int)i;
        }
    return any;
}

long long pixels(const snlm_serve_request &r) { return (long long)r.H * r.W; }

// Form and start launches on the free streams. Returns true if something started.
bool start_launches(snlm_server *s, int *err)
{
    bool any = false;
    const bool plain = s->cfg.mode == SNLM_SERVE_PLAIN;
    while (!s->queue.empty()) {
        const int front = s->queue.front();
        const snlm_serve_request &fr = s->reqs[front].r;
        // small launches take the high-priority streams; so does a large one that
        // starts on an idle GPU, so that requests arriving after it do not preempt it
        // (at low load that is what keeps the large requests' latency at the plain
        // path's); a large launch that joins running work yields to later small ones
        const int si = free_stream(s, pixels(fr) < s->cfg.solo_pixels || s->inflight.empty());
        if (si < 0 || (plain && !s->inflight.empty()))
            break;
        Launch L;
        L.stream = si;
        int launched = 0;
        const bool solo = plain || fr.K < 1 || pixels(fr) >= s->cfg.solo_pixels ||
                          (s->queue.size() == 1 && s->inflight.empty());
        int rc = SNLM_ERR_NOMEM;
        if (!solo) {
            std::vector<int> ids;
            for (size_t q = 0; q < s->queue.size() && (int)ids.size() < s->cfg.max_batch; ++q) {
                const snlm_serve_request &r = s->reqs[s->queue[q]].r;
                if (r.K < 1 || pixels(r) >= s->cfg.solo_pixels)
                    break;                              // keep arrival order
                ids.push_back(s->queue[q]);
            }
            int n_ok = 0;
            rc = launch_batch(s, ids, si, L, &n_ok);
            launched = n_ok;
        }
        if (solo || (rc == SNLM_ERR_NOMEM && s->inflight.empty())) {
            // alone (or, when even a batch of one does not fit an idle GPU, through
            // the per-image path, whose scratch is smaller)
            rc = launch_solo(s, front, si, L);
            launched = 1;
        }
        if (rc == SNLM_ERR_NOMEM) {
            if (s->inflight.empty())
                *err = SNLM_ERR_NOMEM;                  // cannot fit even with the GPU idle
            break;                                      // else wait for memory
        }
        if (rc != SNLM_OK) {
            *err = rc;
            return any;
        }
        cudaEventCreateWithFlags(&L.done, cudaEventDisableTiming);
        cudaEventRecord(L.done, s->streams[si]);
        for (int id : L.members)
            s->reqs[id].launch = s->st.launches;
        s->st.launches += 1;
        s->st.max_batch = std::max(s->st.max_batch, launched);
        s->queue.erase(s->queue.begin(), s->queue.begin() + launched);
        s->busy[si] = 1;
        s->inflight.push_back(std::move(L));
        s->st.max_inflight = std::max(s->st.max_inflight, (int)s->inflight.size());
        s->st.max_used_bytes = std::max(s->st.max_used_bytes, (long long)(s->slab.size - [&] {
                                                                   size_t f = 0;
                                                                   for (auto &e : s->slab.free_)
                                                                       f += e.second;
                                                                   return f;
                                                               }()));
        any = true;
    }
    return any;
}

bool retire(snlm_server *s, int *err)
{
    bool any = false;
    for (size_t i = 0; i < s->inflight.size();) {
        Launch &L = s->inflight[i];
        const cudaError_t q = cudaEventQuery(L.done);
        if (q == cudaErrorNotReady) {
            ++i;
            continue;
        }
        const double t = s->clock();
        if (q != cudaSuccess) {
            cudaGetLastError();
            *err = SNLM_ERR_CUDA;
        } else if (L.plan && *static_cast<volatile int *>(&s->status[L.stream]) != 0) {
            *err = SNLM_ERR_TIMEOUT;
        }
        for (int id : L.members) {
            s->reqs[id].t_done = t;
            s->st.images += 1;
        }
        s->busy[L.stream] = 0;
        release_launch(s, L);
        s->inflight.erase(s->inflight.begin() + (long)i);
        any = true;
    }
    return any;
}

}  // namespace

extern "C" {

int snlm_server_create(const snlm_server_config *cfg, snlm_server **out)
{
    if (!out)
        return SNLM_ERR_ARG;
    *out = nullptr;
    snlm_server_config c;
    c.mode = SNLM_SERVE_BATCHED;
    c.mem_budget = 0;
    c.streams = 4;
    c.max_batch = 256;
    c.solo_pixels = 1 << 20;
    c.ctas_per_sm = 0;
    if (cfg)
        c = *cfg;
    if ((c.mode != SNLM_SERVE_BATCHED && c.mode != SNLM_SERVE_PLAIN) || c.streams < 1 || c.streams > 64 ||
        c.max_batch < 1 || c.solo_pixels < 1)
        return SNLM_ERR_ARG;
    if (c.mode == SNLM_SERVE_PLAIN)
        c.streams = 1;
    // every kernel a request can reach is loaded now, not by its first launch inside
    // the loop
    if (snlm_preload(nullptr) != SNLM_OK)
        return SNLM_ERR_CUDA;
    snlm_server *s = new snlm_server();
    s->cfg = c;
    memset(&s->st, 0, sizeof(s->st));
    cudaGetDevice(&s->device);
    size_t budget = (size_t)std::max(0LL, c.mem_budget);
    if (budget == 0) {
        size_t fr = 0, tot = 0;
        if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
            cudaGetLastError();
            delete s;
            return SNLM_ERR_CUDA;
        }
        budget = fr / 2;
    }
    if (!s->slab.init(budget)) {
        delete s;
        return SNLM_ERR_NOMEM;
    }
    s->st.budget_bytes = (long long)s->slab.size;
    void *words = nullptr;
    if (cudaHostAlloc(&words, (size_t)c.streams * sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        delete s;
        return SNLM_ERR_NOMEM;
    }
    s->status = static_cast<int *>(words);
    memset(s->status, 0, (size_t)c.streams * sizeof(int));
    s->streams.resize((size_t)c.streams);
    s->busy.assign((size_t)c.streams, 0);
    s->high.assign((size_t)c.streams, 0);
    // batched mode: the first half of the streams (at least one) get the device's
    // highest priority and carry the small launches, so that the block scheduler
    // dispatches their CTAs ahead of the pending CTAs of a large request's pass
    int least = 0, greatest = 0;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) {
        cudaGetLastError();
        least = greatest = 0;
    }
    const int n_high = c.mode == SNLM_SERVE_PLAIN ? 0 : std::max(1, c.streams / 2);
    for (size_t i = 0; i < s->streams.size(); ++i) {
        s->high[i] = (int)i < n_high;
        if (cudaStreamCreateWithPriority(&s->streams[i], cudaStreamNonBlocking, s->high[i] ? greatest : least) !=
            cudaSuccess) {
            cudaGetLastError();
            s->streams[i] = nullptr;
        }
    }
    *out = s;
    return SNLM_OK;
}

int snlm_server_submit(snlm_server *s, const snlm_serve_request *reqs, int n, int *ids)
{
    if (!s || (n > 0 && !reqs) || n < 0)
        return SNLM_ERR_ARG;
    for (int i = 0; i < n; ++i) {
        const snlm_serve_request &r = reqs[i];
        int rc = snlm::check_common(r.H, r.W, r.S, r.K, r.h, r.profile, r.order, r.sigma);
        if (rc != SNLM_OK)
            return rc;
        if (!r.img || !r.out || !snlm::valid_dtype(r.dtype) || r.pitch < r.W || !(r.t_arrival >= 0.0))
            return SNLM_ERR_ARG;
        if (footprint(r) + (1u << 20) > s->slab.size)
            return SNLM_ERR_NOMEM;                       // could never be admitted
    }
    for (int i = 0; i < n; ++i) {
        Req q;
        q.r = reqs[i];
        s->reqs.push_back(q);
        const int id = (int)s->reqs.size() - 1;
        if (ids)
            ids[i] = id;
        // keep `order` sorted by arrival among the not-yet-arrived entries
        auto pos = std::upper_bound(s->order.begin() + (long)s->next, s->order.end(), id, [&](int a, int b) {
            return s->reqs[a].r.t_arrival < s->reqs[b].r.t_arrival;
        });
        s->order.insert(pos, id);
    }
    return SNLM_OK;
}

int snlm_server_drain(snlm_server *s)
{
    if (!s)
        return SNLM_ERR_ARG;
    if (!s->started) {
        s->t0 = std::chrono::steady_clock::now();
        s->started = true;
    }
    int err = SNLM_OK;
    const auto h0 = std::chrono::steady_clock::now();
    double idle = 0.0;
    while (s->next < s->order.size() || !s->queue.empty() || !s->inflight.empty()) {
        const auto i0 = std::chrono::steady_clock::now();
        const double now = s->clock();
        while (s->next < s->order.size() && s->reqs[s->order[s->next]].r.t_arrival <= now)
            s->queue.push_back(s->order[s->next++]);
        bool progress = start_launches(s, &err);
        progress |= retire(s, &err);
        if (err != SNLM_OK)
            break;
        const auto i1 = std::chrono::steady_clock::now();
        s->st.max_iter_s = std::max(s->st.max_iter_s, std::chrono::duration<double>(i1 - i0).count());
        if (!progress) {
            // Nothing to do until an arrival or a completion: poll again after yielding
            // the core. The loop never sleeps: a timed sleep overshot by up to ~10 ms on
            // the shared host, which over a 2000-request schedule set the p99 of the
            // lightly loaded points (17 ms at 0.2x of capacity).
            std::this_thread::yield();
            const double y = std::chrono::duration<double>(std::chrono::steady_clock::now() - i1).count();
            idle += y;
            s->st.max_yield_s = std::max(s->st.max_yield_s, y);
            s->st.yields_over_1ms += y > 1e-3 ? 1 : 0;
        }
    }
    if (err != SNLM_OK) {
        // wait for what is in flight, release it, and report
        for (auto &L : s->inflight) {
            cudaStreamSynchronize(s->streams[L.stream]);
            s->busy[L.stream] = 0;
            release_launch(s, L);
        }
        s->inflight.clear();
        cudaGetLastError();
    }
    s->st.wall_s = s->clock();
    s->st.host_busy_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - h0).count() - idle;
    return err;
}

int snlm_server_result(const snlm_server *s, int id, double *t_done, int *launch)
{
    if (!s || id < 0 || id >= (int)s->reqs.size())
        return SNLM_ERR_ARG;
    if (t_done)
        *t_done = s->reqs[(size_t)id].t_done;
    if (launch)
        *launch = s->reqs[(size_t)id].launch;
    return SNLM_OK;
}

int snlm_server_get_stats(const snlm_server *s, snlm_server_stats *out)
{
    if (!s || !out)
        return SNLM_ERR_ARG;
    *out = s->st;
    return SNLM_OK;
}

double snlm_server_clock(const snlm_server *s) { return s ? s->clock() : 0.0; }

void snlm_server_destroy(snlm_server *s)
{
    if (!s)
        return;
    for (auto &L : s->inflight) {
        cudaStreamSynchronize(s->streams[L.stream]);
        release_launch(s, L);
    }
    for (auto st : s->streams)
        if (st)
            cudaStreamDestroy(st);
    if (s->status)
        cudaFreeHost(s->status);
    delete s;
}

}  // extern "C"
