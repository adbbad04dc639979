// Serving: resident scenes and a continuous-batching render loop on one GPU.
//
// The server allocates, once at create time, one device pool split into a scene region (splat
// sets copied in by darb_serve_add_scene, bump-allocated) and `slots` equal batch slots.  Every
// slot owns a stream plus kGroupStreams group streams.  A worker thread repeats: (1) for every
// free slot, take pending requests in FIFO order while their workspace fits the slot (admission
// by free memory) and at most max_batch, group them by (scene, kernel), and enqueue one
// darb_render_batch per group, the groups forked over the slot's group streams so that one
// group's compositing overlaps the next group's sorts, then joined back into the slot stream,
// which copies the per-view statuses and instance counts to pinned host memory and records the
// slot's completion event; (2) retire every batch whose event has completed, in any order: a
// view that overflowed its capacity goes back to the head of the queue once with the capacity
// its instance count asks for, every other view completes its ticket.  Because slots have their
// own streams, a batch formed while others render is on the device at once, and the batches'
// kernels overlap.  Each request's capacity comes from the largest instances-per-pixel ratio
// seen so far for its scene (or the configured guess), times a margin.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "validate.h"

namespace darb {
namespace {

using Clock = std::chrono::steady_clock;

constexpr int kMaxSlots = DARB_MAX_SERVE_SLOTS;
constexpr int kDefaultSlots = 2;
constexpr int kGroupStreams = 4;
constexpr uint64_t kPageAlign = 4096;

uint64_t align_up(uint64_t x, uint64_t a) { return (x + a - 1) / a * a; }

struct Scene {
    darb_splats splats;  // device pointers into the scene region
    double max_ratio = 0.0;  // largest instances per pixel seen (0 = none yet)
};

struct Pending {
    uint64_t ticket;
    darb_request req;
    Clock::time_point submitted;
    uint32_t attempts;
    uint64_t capacity;
};

struct Ticket {
    bool done = false;
    darb_result result{};
};

struct Batch {
    std::vector<Pending> items;
    Clock::time_point launched;
    cudaEvent_t done = nullptr;
    int slot = 0;
    uint64_t id = 0;
};

}  // namespace
}  // namespace darb

struct darb_server {
    darb_serve_cfg cfg{};
    int device = 0;
    int slots = 0;
    unsigned char *pool = nullptr;
    uint64_t scene_bytes = 0, scene_used = 0, slot_bytes = 0;
    unsigned char *slot_base[darb::kMaxSlots] = {};
    bool slot_busy[darb::kMaxSlots] = {};
    uint32_t *host_words[darb::kMaxSlots] = {};  // pinned: [max_batch] statuses then [max_batch] counts
    cudaStream_t stream[darb::kMaxSlots] = {};    // slot streams (stream[0] also copies scenes in)
    cudaStream_t group_stream[darb::kMaxSlots][darb::kGroupStreams] = {};
    cudaEvent_t begin[darb::kMaxSlots] = {};      // timed: the slot stream reached the batch ...
    cudaEvent_t events[darb::kMaxSlots] = {};     // ... and finished it (blocking-sync)
    cudaEvent_t join[darb::kMaxSlots][darb::kGroupStreams] = {};
    cudaEvent_t epoch = nullptr;                  // device time zero of gpu_begin_us / gpu_end_us
    uint64_t next_batch = 1;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    bool stop = false;
    std::vector<darb::Scene> scenes;
    std::deque<darb::Pending> pending;
    std::unordered_map<uint64_t, darb::Ticket> tickets;
    uint64_t next_ticket = 1;
    std::deque<darb::Batch> inflight;
    std::thread worker;
};

namespace darb {
namespace {

size_t scene_splat_bytes(int n, int sh_degree) {
    const size_t N = (size_t)n, K = (size_t)(sh_degree + 1) * (sh_degree + 1);
    return align_up(12 * N, 256) * 2 + align_up(16 * N, 256) + align_up(4 * N, 256) + align_up(12 * K * N, 256);
}

darb_batch_params group_params(const darb_server *S, int n_views, uint64_t capacity) {
    darb_batch_params p{};
    p.n_views = n_views;
    p.tile = S->cfg.tile;
    p.depth = S->cfg.depth;
    p.max_ctas = 0;
    p.capacity = capacity;
    return p;
}

// Device words of a slot (statuses and counts of up to max_batch views) come first.
uint64_t slot_header_bytes(const darb_server *S) { return align_up(8ull * (uint64_t)S->cfg.max_batch, 256); }

uint64_t capacity_for(const darb_server *S, const darb_request &r) {
    const Scene &sc = S->scenes[(size_t)r.scene_id];
    const double px = (double)r.cam.width * (double)r.cam.height;
    const double ratio = sc.max_ratio > 0.0 ? sc.max_ratio * S->cfg.capacity_margin : S->cfg.capacity_per_pixel;
    const double c = std::max((double)S->cfg.capacity_min, ratio * px);
    return (uint64_t)std::min(c, (double)kMaxCapacity);
}

// Workspace bytes of one request rendered alone (the admission test at submit time).
bool single_need(const darb_server *S, const darb_request &r, uint64_t capacity, size_t *bytes) {
    const darb_batch_params p = group_params(S, 1, capacity);
    return darb_render_batch_workspace_size(S->scenes[(size_t)r.scene_id].splats.n, &r.cam, &p, bytes) == DARB_OK;
}

struct GroupPlan {
    int scene, kernel;
    std::vector<int> idx;  // indices into the batch's items
    uint64_t capacity = 0;
    size_t bytes = 0;
};

// Plans the groups of a candidate batch; returns the slot bytes it needs.
size_t plan_groups(const darb_server *S, const std::vector<Pending> &items, std::vector<GroupPlan> &groups) {
    groups.clear();
    std::map<std::pair<int, int>, size_t> where;
    for (size_t i = 0; i < items.size(); ++i) {
        const auto key = std::make_pair(items[i].req.scene_id, items[i].req.kernel);
        auto it = where.find(key);
        if (it == where.end()) {
            where[key] = groups.size();
            groups.push_back(GroupPlan{key.first, key.second, {}, 0, 0});
            it = where.find(key);
        }
        GroupPlan &g = groups[it->second];
        g.idx.push_back((int)i);
        g.capacity = std::max(g.capacity, items[i].capacity);
    }
    size_t total = slot_header_bytes(S);
    for (GroupPlan &g : groups) {
        std::vector<darb_camera> cams;
        for (int i : g.idx) cams.push_back(items[(size_t)i].req.cam);
        const darb_batch_params p = group_params(S, (int)cams.size(), g.capacity);
        size_t b = 0;
        if (darb_render_batch_workspace_size(S->scenes[(size_t)g.scene].splats.n, cams.data(), &p, &b) != DARB_OK)
            return SIZE_MAX;
        g.bytes = align_up(b, 256);
        total += g.bytes;
    }
    return total;
}

struct BatchTimes {
    uint64_t id = 0;
    double gpu_begin_us = 0.0, gpu_end_us = 0.0;
};

void complete(darb_server *S, const Pending &p, int32_t status, uint32_t M, uint32_t batch_size,
              Clock::time_point launched, Clock::time_point now, const BatchTimes &bt = BatchTimes{}) {
    Ticket &t = S->tickets[p.ticket];
    t.done = true;
    t.result.status = status;
    t.result.num_instances = M;
    t.result.attempts = p.attempts;
    t.result.batch_size = batch_size;
    t.result.queue_us = std::chrono::duration<double, std::micro>(launched - p.submitted).count();
    t.result.latency_us = std::chrono::duration<double, std::micro>(now - p.submitted).count();
    t.result.batch_id = bt.id;
    t.result.gpu_begin_us = bt.gpu_begin_us;
    t.result.gpu_end_us = bt.gpu_end_us;
}

// Forms and enqueues one batch into a free slot (lock held).  Returns false if nothing was launched.
bool launch_batch(darb_server *S, int slot) {
    std::vector<Pending> items;
    std::vector<GroupPlan> groups;
    while (!S->pending.empty() && (int)items.size() < S->cfg.max_batch) {
        items.push_back(S->pending.front());
        if (plan_groups(S, items, groups) > S->slot_bytes) {
            items.pop_back();
            break;
        }
        S->pending.pop_front();
    }
    if (items.empty()) return false;
    plan_groups(S, items, groups);
    unsigned char *base = S->slot_base[slot];
    uint32_t *d_status = reinterpret_cast<uint32_t *>(base);
    uint32_t *d_count = d_status + S->cfg.max_batch;
    size_t off = slot_header_bytes(S);
    cudaStream_t ms = S->stream[slot];
    int32_t fail = DARB_OK;
    // fork: the group streams start after the slot stream reaches this batch
    if (cudaEventRecord(S->begin[slot], ms) != cudaSuccess) fail = DARB_ERR_CUDA;
    const int used = std::min<int>((int)groups.size(), kGroupStreams);
    for (int g = 0; g < used && fail == DARB_OK; ++g)
        if (cudaStreamWaitEvent(S->group_stream[slot][g], S->begin[slot], 0) != cudaSuccess) fail = DARB_ERR_CUDA;
    int view_no = 0;
    std::vector<int> order;  // item index of each view, in launch order
    for (size_t gi = 0; gi < groups.size() && fail == DARB_OK; ++gi) {
        const GroupPlan &g = groups[gi];
        std::vector<darb_camera> cams;
        std::vector<darb_image> outs;
        for (int i : g.idx) {
            cams.push_back(items[(size_t)i].req.cam);
            outs.push_back(darb_image{items[(size_t)i].req.image, nullptr, nullptr, nullptr});
            order.push_back(i);
        }
        darb_kernel_params kp{};
        darb_kernel_defaults(g.kernel, &kp);
        const darb_batch_params p = group_params(S, (int)cams.size(), g.capacity);
        const darb_status st =
            darb_render_batch(&S->scenes[(size_t)g.scene].splats, cams.data(), &kp, &p, base + off, g.bytes, outs.data(),
                              d_count + view_no, d_status + view_no,
                              reinterpret_cast<darb_stream>(S->group_stream[slot][gi % kGroupStreams]));
        if (st != DARB_OK) fail = st;
        off += g.bytes;
        view_no += (int)cams.size();
    }
    // join: the slot stream continues once every group stream has finished its groups
    for (int g = 0; g < used; ++g) {
        if (cudaEventRecord(S->join[slot][g], S->group_stream[slot][g]) != cudaSuccess ||
            cudaStreamWaitEvent(ms, S->join[slot][g], 0) != cudaSuccess)
            fail = fail == DARB_OK ? DARB_ERR_CUDA : fail;
    }
    Batch b;
    b.slot = slot;
    b.launched = Clock::now();
    b.done = S->events[slot];
    b.id = S->next_batch++;
    if (fail != DARB_OK) {
        // nothing of this batch may still write into the slot when it is reused
        for (int g = 0; g < used; ++g) cudaStreamSynchronize(S->group_stream[slot][g]);
        cudaStreamSynchronize(ms);
        for (const Pending &p : items) complete(S, p, fail, 0, (uint32_t)items.size(), b.launched, Clock::now());
        S->cv_done.notify_all();
        return true;
    }
    // items reordered into launch order, so view v of the slot is b.items[v]
    for (int i : order) b.items.push_back(items[(size_t)i]);
    const size_t words = (size_t)S->cfg.max_batch;
    cudaMemcpyAsync(S->host_words[slot], d_status, words * 4, cudaMemcpyDeviceToHost, ms);
    cudaMemcpyAsync(S->host_words[slot] + words, d_count, words * 4, cudaMemcpyDeviceToHost, ms);
    if (cudaEventRecord(b.done, ms) != cudaSuccess) {
        for (const Pending &p : b.items)
            complete(S, p, DARB_ERR_CUDA, 0, (uint32_t)b.items.size(), b.launched, Clock::now());
        S->cv_done.notify_all();
        return true;
    }
    S->slot_busy[slot] = true;
    S->inflight.push_back(std::move(b));
    return true;
}

// Retires a completed batch (lock held; q is the status of its completion event).
void retire(darb_server *S, const Batch &b, cudaError_t q) {
    const Clock::time_point now = Clock::now();
    BatchTimes bt;
    bt.id = b.id;
    float ms0 = 0.0f, ms1 = 0.0f;
    if (q == cudaSuccess && cudaEventElapsedTime(&ms0, S->epoch, S->begin[b.slot]) == cudaSuccess &&
        cudaEventElapsedTime(&ms1, S->epoch, b.done) == cudaSuccess) {
        bt.gpu_begin_us = 1e3 * (double)ms0;
        bt.gpu_end_us = 1e3 * (double)ms1;
    }
    const uint32_t *hs = S->host_words[b.slot];
    const uint32_t *hc = hs + S->cfg.max_batch;
    std::vector<Pending> retry;
    for (size_t v = 0; v < b.items.size(); ++v) {
        const Pending &p = b.items[v];
        const int32_t status = q == cudaSuccess ? (int32_t)hs[v] : (int32_t)DARB_ERR_CUDA;
        const uint32_t M = q == cudaSuccess ? hc[v] : 0;
        if (status == DARB_OK || status == DARB_ERR_CAPACITY) {
            Scene &sc = S->scenes[(size_t)p.req.scene_id];
            const double ratio = (double)M / ((double)p.req.cam.width * (double)p.req.cam.height);
            sc.max_ratio = std::max(sc.max_ratio, ratio);
        }
        if (status == DARB_ERR_CAPACITY && p.attempts == 1) {
            Pending r = p;
            r.attempts = 2;
            r.capacity = std::min<uint64_t>((uint64_t)((double)M * 1.05) + 1024, kMaxCapacity);
            size_t need = 0;
            if (single_need(S, r.req, r.capacity, &need) && need + slot_header_bytes(S) <= S->slot_bytes) {
                retry.push_back(r);
                continue;
            }
        }
        complete(S, p, status, M, (uint32_t)b.items.size(), b.launched, now, bt);
    }
    for (auto it = retry.rbegin(); it != retry.rend(); ++it) S->pending.push_front(*it);
    S->slot_busy[b.slot] = false;
    S->cv_done.notify_all();
}

// Retires every in-flight batch whose work has completed (lock held).  Returns the number retired.
int retire_ready(darb_server *S) {
    int n = 0;
    for (auto it = S->inflight.begin(); it != S->inflight.end();) {
        const cudaError_t q = cudaEventQuery(it->done);
        if (q == cudaErrorNotReady) {
            ++it;
            continue;
        }
        retire(S, *it, q);
        it = S->inflight.erase(it);
        ++n;
    }
    return n;
}

// Blocks (lock released) until the oldest in-flight batch has finished, then retires it.
void wait_oldest(darb_server *S, std::unique_lock<std::mutex> &lock) {
    cudaEvent_t ev = S->inflight.front().done;  // only this thread changes `inflight`
    lock.unlock();
    cudaEventSynchronize(ev);
    lock.lock();
    retire_ready(S);
}

void worker_loop(darb_server *S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lock(S->mu);
    for (;;) {
        bool progress = retire_ready(S) > 0;
        for (int s = 0; s < S->slots; ++s)
            if (!S->slot_busy[s] && !S->pending.empty()) progress |= launch_batch(S, s);
        if (S->stop && S->pending.empty() && S->inflight.empty()) break;
        if (progress) continue;
        if (!S->inflight.empty()) {
            if (S->pending.empty())
                S->cv_work.wait_for(lock, std::chrono::microseconds(50));  // new request or a batch finishing
            else
                wait_oldest(S, lock);  // every slot busy: wait for the oldest batch
        } else if (!S->pending.empty()) {
            // an empty slot that cannot take the head request (admission is checked at submit,
            // so this is a request whose retry grew past the slot): fail it
            const Pending p = S->pending.front();
            S->pending.pop_front();
            const auto now = Clock::now();
            complete(S, p, DARB_ERR_ADMISSION, 0, 0, now, now);
            S->cv_done.notify_all();
        } else {
            S->cv_work.wait(lock, [&] { return S->stop || !S->pending.empty(); });
        }
    }
}

}  // namespace
}  // namespace darb

using namespace darb;

extern "C" {

darb_status darb_serve_create(const darb_serve_cfg *cfg, darb_server **out) {
    if (!cfg || !out || !valid_tile(cfg->tile) || cfg->max_batch < 1 || cfg->max_batch > DARB_MAX_BATCH_VIEWS ||
        cfg->depth < 1 || cfg->depth > 8 || cfg->scene_bytes == 0 || cfg->slots < 0 || cfg->slots > kMaxSlots ||
        !(cfg->capacity_per_pixel > 0.0f) || !(cfg->capacity_margin >= 1.0f) || cfg->capacity_min < 1)
        return DARB_ERR_INVALID_ARG;
    const int slots = cfg->slots == 0 ? kDefaultSlots : cfg->slots;
    if (cfg->workspace_bytes < (uint64_t)slots * kPageAlign) return DARB_ERR_INVALID_ARG;
    darb_server *S = new darb_server();
    S->cfg = *cfg;
    S->slots = slots;
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        delete S;
        return DARB_ERR_CUDA;
    }
    S->scene_bytes = align_up(cfg->scene_bytes, kPageAlign);
    S->slot_bytes = cfg->workspace_bytes / (uint64_t)slots / kPageAlign * kPageAlign;
    const uint64_t total = S->scene_bytes + (uint64_t)slots * S->slot_bytes;
    bool ok = cudaMalloc(&S->pool, total) == cudaSuccess;
    ok = ok && cudaEventCreate(&S->epoch) == cudaSuccess;
    for (int s = 0; s < slots && ok; ++s) {
        S->slot_base[s] = S->pool + S->scene_bytes + s * S->slot_bytes;
        ok = cudaStreamCreateWithFlags(&S->stream[s], cudaStreamNonBlocking) == cudaSuccess;
        for (int g = 0; g < kGroupStreams && ok; ++g) {
            ok = cudaStreamCreateWithFlags(&S->group_stream[s][g], cudaStreamNonBlocking) == cudaSuccess;
            ok = ok && cudaEventCreateWithFlags(&S->join[s][g], cudaEventDisableTiming) == cudaSuccess;
        }
        ok = ok && cudaEventCreate(&S->begin[s]) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&S->events[s], cudaEventBlockingSync) == cudaSuccess;
        ok = ok && cudaMallocHost(&S->host_words[s], 8ull * (uint64_t)cfg->max_batch) == cudaSuccess;
    }
    ok = ok && cudaEventRecord(S->epoch, S->stream[0]) == cudaSuccess &&
         cudaEventSynchronize(S->epoch) == cudaSuccess;
    if (!ok) {
        darb_serve_destroy(S);
        cudaGetLastError();
        return DARB_ERR_CUDA;
    }
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return DARB_OK;
}

darb_status darb_serve_add_scene(darb_server *S, const darb_splats *splats, int32_t *scene_id) {
    if (!S || !valid_splats(splats) || splats->n == 0 || !scene_id) return DARB_ERR_INVALID_ARG;
    const int n = splats->n;
    const size_t need = scene_splat_bytes(n, splats->sh_degree);
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->scene_used + need > S->scene_bytes) return DARB_ERR_ADMISSION;
    unsigned char *b = S->pool + S->scene_used;
    const size_t N = (size_t)n, K = (size_t)(splats->sh_degree + 1) * (splats->sh_degree + 1);
    darb_splats d{};
    size_t o = 0;
    d.means = reinterpret_cast<float *>(b + o);
    o += align_up(12 * N, 256);
    d.scales = reinterpret_cast<float *>(b + o);
    o += align_up(12 * N, 256);
    d.quats = reinterpret_cast<float *>(b + o);
    o += align_up(16 * N, 256);
    d.opacities = reinterpret_cast<float *>(b + o);
    o += align_up(4 * N, 256);
    d.sh = reinterpret_cast<float *>(b + o);
    d.n = n;
    d.sh_degree = splats->sh_degree;
    const struct {
        const float *dst, *src;
        size_t bytes;
    } copies[] = {{d.means, splats->means, 12 * N},
                  {d.scales, splats->scales, 12 * N},
                  {d.quats, splats->quats, 16 * N},
                  {d.opacities, splats->opacities, 4 * N},
                  {d.sh, splats->sh, 12 * K * N}};
    for (const auto &c : copies)
        if (cudaMemcpyAsync(const_cast<float *>(c.dst), c.src, c.bytes, cudaMemcpyDeviceToDevice, S->stream[0]) !=
            cudaSuccess)
            return DARB_ERR_CUDA;
    if (cudaStreamSynchronize(S->stream[0]) != cudaSuccess) return DARB_ERR_CUDA;
    S->scene_used += align_up(need, 256);
    S->scenes.push_back(Scene{d, 0.0});
    *scene_id = (int32_t)S->scenes.size() - 1;
    return DARB_OK;
}

// Validates and queues one request (lock held).
darb_status enqueue(darb_server *S, const darb_request *r, uint64_t *ticket) {
    if (!r || !ticket || !valid_camera(&r->cam) || !r->image || r->kernel < 0 || r->kernel >= kNumKernels - 1)
        return DARB_ERR_INVALID_ARG;
    if (S->stop) return DARB_ERR_INVALID_ARG;
    if (r->scene_id < 0 || r->scene_id >= (int32_t)S->scenes.size()) return DARB_ERR_NOT_FOUND;
    Pending p;
    p.req = *r;
    p.submitted = Clock::now();
    p.attempts = 1;
    p.capacity = capacity_for(S, *r);
    size_t need = 0;
    if (!single_need(S, *r, p.capacity, &need) || need + slot_header_bytes(S) > S->slot_bytes)
        return DARB_ERR_ADMISSION;  // could never fit, even alone in an empty slot
    p.ticket = S->next_ticket++;
    S->tickets[p.ticket] = Ticket{};
    S->pending.push_back(p);
    *ticket = p.ticket;
    return DARB_OK;
}

darb_status darb_serve_submit(darb_server *S, const darb_request *r, uint64_t *ticket) {
    if (!S) return DARB_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(S->mu);
    const darb_status st = enqueue(S, r, ticket);
    if (st == DARB_OK) S->cv_work.notify_one();
    return st;
}

darb_status darb_serve_submit_many(darb_server *S, const darb_request *requests, int32_t count, uint64_t *tickets,
                                   int32_t *submitted) {
    if (!S || !requests || !tickets || !submitted || count < 0) return DARB_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> lock(S->mu);
    darb_status st = DARB_OK;
    int32_t k = 0;
    for (; k < count; ++k) {
        st = enqueue(S, &requests[k], &tickets[k]);
        if (st != DARB_OK) break;
    }
    *submitted = k;
    if (k > 0) S->cv_work.notify_one();
    return st;
}

darb_status darb_serve_poll(darb_server *S, uint64_t ticket, int32_t timeout_ms, darb_result *result) {
    if (!S || !result) return DARB_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lock(S->mu);
    auto it = S->tickets.find(ticket);
    if (it == S->tickets.end()) return DARB_ERR_NOT_FOUND;
    if (!it->second.done) {
        const auto until = Clock::now() + std::chrono::milliseconds(std::max(0, timeout_ms));
        S->cv_done.wait_until(lock, until, [&] {
            const auto f = S->tickets.find(ticket);
            return f == S->tickets.end() || f->second.done;
        });
        it = S->tickets.find(ticket);
        if (it == S->tickets.end()) return DARB_ERR_NOT_FOUND;  // collected by another poller
        if (!it->second.done) return DARB_ERR_TIMEOUT;
    }
    *result = it->second.result;
    S->tickets.erase(it);
    return DARB_OK;
}

void darb_serve_destroy(darb_server *S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lock(S->mu);
        S->stop = true;
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    for (int s = 0; s < kMaxSlots; ++s) {
        if (S->events[s]) cudaEventDestroy(S->events[s]);
        if (S->begin[s]) cudaEventDestroy(S->begin[s]);
        if (S->host_words[s]) cudaFreeHost(S->host_words[s]);
        for (int g = 0; g < kGroupStreams; ++g) {
            if (S->join[s][g]) cudaEventDestroy(S->join[s][g]);
            if (S->group_stream[s][g]) cudaStreamDestroy(S->group_stream[s][g]);
        }
        if (S->stream[s]) cudaStreamDestroy(S->stream[s]);
    }
    if (S->epoch) cudaEventDestroy(S->epoch);
    if (S->pool) cudaFree(S->pool);
    delete S;
}

}  // extern "C"
