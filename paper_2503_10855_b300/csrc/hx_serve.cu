// hx_serve.cu -- the serving engine: admission against a device-memory
// budget, continuous batching into the batched kernel, completion tracking.
//
// Hercules's host backend runs independent calls as concurrent tasks and
// awaits each at its first use (Sec. 4.5); a runner sizes a call's backing
// memory from its dynamic constants before running it (Sec. 4.2, 4.6).  A
// server does the same for a stream of requests: it sizes each request from
// its arguments, admits it when the device-memory budget allows, and keeps
// the device busy with steps that mix every admitted request's next piece of
// work, so requests that arrive while others run overlap with them.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "hx_batch.cuh"

namespace hx {
namespace {

double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Per-request device workspace, kept from admission to completion so that a
// request's work can be split over several steps: tile partials, histogram
// or residual accumulator, and the block progress words of a stencil request
// that runs several sweeps in one step (zero between uses).
constexpr size_t kWsPartials = kMrMaxTiles;
constexpr size_t kWsAccWords = kHiBins;
constexpr size_t kWsProgWords = 4096;
constexpr size_t kWsBytes = ((kWsPartials * sizeof(float2) + (kWsAccWords + kWsProgWords) * 4) + 255) & ~(size_t)255;
// Continuous mode: at most this many fresh requests run as standalone calls
// instead of a batched step (hx_server_config.direct_max = 0).
constexpr int kDefaultDirectMax = 4;
// Continuous mode: a fresh stencil request whose sweep moves at least this
// many bytes runs as its standalone call (hx_server_config.direct_sweep_bytes
// = 0).  A 16 MiB sweep (a 1448 x 1448 grid) fills the device on its own.
constexpr int64_t kDefaultDirectSweepBytes = (int64_t)16 << 20;
static_assert(kMaxStepSweeps <= (int)kWsAccWords, "a request's workspace holds one maximum per sweep");

struct Req {
    uint64_t id = 0;
    hx_task task{};
    double arrival = 0.0;
    double latency = -1.0;
    size_t footprint = 0;
    BInst inst{};            // described at admission
    int64_t partials = 0, acc_words = 0;
    int ws = -1;             // workspace slot
    int sweep = 0;           // stencil: current sweep
    int64_t issued = 0;      // tiles (chunks) of the current pass already put in a step
    bool admitted = false, issued_all = false, done = false;
    hx_status status = HX_OK;
};

struct Slot {   // staging for one step: descriptors and prefix sums, pinned host + device copy
    char *h = nullptr;
    char *d = nullptr;
    size_t bytes = 0;
    cudaEvent_t ev = nullptr;
    bool busy = false;
};

struct Step {
    int64_t record = -1;       // index into the server's timeline, or -1
    cudaEvent_t ev = nullptr;
    int slot = -1;             // continuous mode: staging slot to release
    std::vector<Req *> finishing;
    std::vector<Req *> members;   // continuous mode: every request with work in the step
};

}  // namespace
}  // namespace hx

struct hx_server {
    hx_ctx *ctx = nullptr;
    hx_server_config cfg{};
    cudaStream_t stream = nullptr;
    std::mutex mu;
    std::condition_variable cv_sched, cv_compl, cv_done;
    std::deque<hx::Req *> queue;              // submitted, not yet admitted
    std::vector<hx::Req *> active;            // admitted, not fully issued
    std::unordered_map<uint64_t, std::unique_ptr<hx::Req>> reqs;
    std::deque<hx::Step> steps;               // issued, not yet completed (in stream order)
    std::vector<hx::Slot> slots;
    std::vector<cudaEvent_t> free_events;     // per-launch mode
    char *ws_pool = nullptr;                  // continuous mode: max_inflight workspace slots (+ run counter)
    unsigned int *err_h = nullptr;            // host-mapped error word of the steps' bounded waits
    unsigned int *err_d = nullptr;
    bool stall_next = false;                  // test hook: stall the next multi-sweep step (hx_debug_server_stall)
    long long stall_wait_ns = 0;
    uint64_t failed_at_drain = 0;             // stats.failed when the last drain returned
    unsigned int *ctrl = nullptr;
    std::vector<int> free_ws;
    // completions not yet reported to cfg.on_done: (id, status, latency)
    std::vector<std::tuple<uint64_t, hx_status, double>> to_report;
    bool reporting = false;                   // the completion thread is calling on_done
    uint64_t next_id = 1;
    size_t used = 0;
    int inflight = 0;
    bool issuing = false;                     // standalone launches in progress without the lock
    bool stop = false;
    hx_server_stats stats{};
    double created = 0.0;                     // timeline origin (steady clock)
    std::vector<hx_server_step_record> timeline;   // one record per issued step (the first kTimelineMax)
    std::thread sched, compl_thr;
};

namespace hx {
namespace {

void admit_locked(hx_server *s) {
    const size_t budget = s->cfg.hbm_budget_bytes;
    while (!s->queue.empty()) {
        Req *r = s->queue.front();
        const bool fits = budget == 0 || s->used + r->footprint <= budget;
        if (s->inflight > 0 && (!fits || s->inflight >= s->cfg.max_inflight)) break;
        s->queue.pop_front();
        describe_instance(s->ctx, r->task, &r->inst, &r->partials, &r->acc_words);
        if (s->cfg.mode == HX_SERVE_CONTINUOUS) {
            r->ws = s->free_ws.back();
            s->free_ws.pop_back();
            char *w = s->ws_pool + (size_t)r->ws * kWsBytes;
            r->inst.partials = reinterpret_cast<float2 *>(w);
            r->inst.acc = reinterpret_cast<unsigned int *>(w + kWsPartials * sizeof(float2));
        }
        r->admitted = true;
        s->used += r->footprint;
        s->inflight += 1;
        s->stats.admitted += 1;
        s->stats.footprint_in_flight = s->used;
        s->stats.peak_footprint = std::max(s->stats.peak_footprint, s->used);
        s->active.push_back(r);
    }
}

constexpr size_t kTimelineMax = (size_t)1 << 16;

// Queues an issued step and records it in the timeline (called with the
// lock held).
void push_step_locked(hx_server *s, Step &&step, int direct) {
    if (s->timeline.size() < kTimelineMax) {
        step.record = (int64_t)s->timeline.size();
        const size_t n = std::max(step.members.size(), step.finishing.size());
        s->timeline.push_back({now_s() - s->created, -1.0, (int32_t)n, direct});
    }
    s->steps.push_back(std::move(step));
}

// Outputs of requests with no device work (empty map->reduce or histogram):
// written by small async writes on the server's stream.
cudaError_t write_trivial(cudaStream_t st, const hx_task &t) {
    cudaError_t e = cudaSuccess;
    if (t.kind == HX_TASK_MAP_REDUCE) {
        e = cudaMemsetAsync(t.u.mr.sum, 0, sizeof(float), st);
        if (e == cudaSuccess && t.u.mr.sum64) e = cudaMemsetAsync(t.u.mr.sum64, 0, sizeof(double), st);
    } else if (t.kind == HX_TASK_HISTOGRAM) {
        e = cudaMemsetAsync(t.u.hi.bins, 0, 256 * sizeof(uint32_t), st);
        if (e == cudaSuccess && t.u.hi.scan) e = cudaMemsetAsync(t.u.hi.scan, 0, 256 * sizeof(uint32_t), st);
    }
    return e;
}

void fail_requests_locked(hx_server *s, std::vector<Req *> &rs, hx_status st) {
    for (Req *r : rs) {
        if (r->done) continue;
        r->status = st;
        r->issued_all = true;
        r->done = true;
        r->latency = now_s() - r->arrival;
        if (s->cfg.on_done) s->to_report.emplace_back(r->id, st, r->latency);
        s->used -= r->footprint;
        s->inflight -= 1;
        if (r->ws >= 0) {
            // the request's final combine may never run: clear its
            // accumulators (ordered after its steps already on the stream)
            // before the slot serves another request
            char *w = s->ws_pool + (size_t)r->ws * kWsBytes;
            cudaMemsetAsync(w + kWsPartials * sizeof(float2), 0, (kWsAccWords + kWsProgWords) * 4, s->stream);
            s->free_ws.push_back(r->ws);
        }
        r->ws = -1;
        s->stats.failed += 1;
        s->stats.completed += 1;
    }
    s->stats.footprint_in_flight = s->used;
    s->cv_done.notify_all();
    s->cv_compl.notify_all();
}

// Bytes of traffic one tile (histogram: one chunk) of an instance moves.
int64_t tile_bytes(const BInst &I) {
    if (I.kind == kKindMap) return 12 * I.plan.tile_elems;
    if (I.kind == kKindStencil) return 8 * 128 * kBatchStRows;
    return kBHiTile;
}

// The request's whole work as its standalone call on the server's stream.
hx_status launch_standalone(hx_server *s, const hx_task &t) {
    if (t.kind == HX_TASK_MAP_REDUCE)
        return hx_map_reduce(s->ctx, t.u.mr.x, t.u.mr.y, t.u.mr.out, t.u.mr.a, t.u.mr.n, t.u.mr.sum, t.u.mr.sum64,
                             (hx_stream_t)s->stream);
    if (t.kind == HX_TASK_STENCIL2D)
        return hx_stencil2d(s->ctx, t.u.st.u0, t.u.st.u1, t.u.st.nx, t.u.st.ny, t.u.st.iters, t.u.st.resid, nullptr,
                            (hx_stream_t)s->stream);
    return hx_histogram(s->ctx, t.u.hi.v, t.u.hi.n, t.u.hi.bins, t.u.hi.scan, (hx_stream_t)s->stream);
}

cudaEvent_t take_event(hx_server *s) {
    cudaEvent_t ev = nullptr;
    if (!s->free_events.empty()) {
        ev = s->free_events.back();
        s->free_events.pop_back();
    } else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
        ev = nullptr;
    }
    return ev;
}

// Issues each of `rs` (admitted requests that have not started) as its
// standalone call on the server's stream, with its own completion event --
// no descriptor upload, no batched launch and final combine.  Results are the
// same bits either way.
void issue_direct_locked(hx_server *s, const std::vector<Req *> &rs, std::unique_lock<std::mutex> &lk) {
    // The launches run with the lock released (a stencil request is 20 or
    // more launches): the completion thread and submitters are not held up.
    // The requests are no longer in `active`, and only this thread issues.
    s->issuing = true;
    for (Req *r : rs) {
        r->issued_all = true;
        s->stats.launches += 1;
        cudaEvent_t ev = take_event(s);
        const hx_task t = r->task;
        lk.unlock();
        hx_status st = ev ? launch_standalone(s, t) : HX_ERR_CUDA;
        if (st == HX_OK && cudaEventRecord(ev, s->stream) != cudaSuccess) st = HX_ERR_CUDA;
        lk.lock();
        std::vector<Req *> one{r};
        if (st != HX_OK) {
            if (ev) s->free_events.push_back(ev);
            fail_requests_locked(s, one, st);
            continue;
        }
        Step step;
        step.ev = ev;
        step.finishing = one;
        step.members = one;
        push_step_locked(s, std::move(step), 1);
        s->cv_compl.notify_one();
    }
    s->issuing = false;
    s->cv_compl.notify_all();
}

bool fresh(const Req *r) { return r->issued == 0 && r->sweep == 0 && !r->issued_all; }

// Continuous mode: build one step out of the next slice of every admitted
// request (at most its share of step_target_bytes, and at least
// step_quantum_bytes, of traffic), upload its descriptors and prefix sums,
// launch.  A stencil slice stays within one sweep, except that a stencil
// request at a sweep boundary whose sweep is below the direct-issue size
// takes up to cfg.max_step_sweeps of its remaining sweeps: the step's
// persistent launch runs them one after another (bounded waits between an
// instance's sweeps, see hx_batch.cuh), so a small stencil request needs one
// step instead of one per sweep.
bool issue_step_locked(hx_server *s, std::unique_lock<std::mutex> &lk) {
    // low load: when at most cfg.direct_max requests wait and none has
    // started, each runs as its standalone call (the shortest path for a
    // request that has the device nearly to itself)
    if ((int)s->active.size() <= s->cfg.direct_max && std::all_of(s->active.begin(), s->active.end(), fresh)) {
        std::vector<Req *> all;
        all.swap(s->active);
        issue_direct_locked(s, all, lk);
        return true;
    }
    // a stencil request with large sweeps runs as its standalone call at any
    // load: in batched steps it would advance one sweep per step
    bool issued_direct = false;
    if (s->cfg.direct_sweep_bytes > 0) {
        std::vector<Req *> big, rest;
        for (Req *r : s->active)
            (r->task.kind == HX_TASK_STENCIL2D && fresh(r) && r->inst.tiles > 0 && r->task.u.st.iters > 0 &&
                     8 * (int64_t)r->task.u.st.nx * r->task.u.st.ny >= s->cfg.direct_sweep_bytes
                 ? big
                 : rest)
                .push_back(r);
        if (!big.empty()) {
            s->active.swap(rest);
            issue_direct_locked(s, big, lk);
            issued_direct = true;
            if (s->active.empty()) return true;
        }
    }
    int slot = -1;
    for (size_t i = 0; i < s->slots.size(); ++i)
        if (!s->slots[i].busy) { slot = (int)i; break; }
    if (slot < 0 || (int)s->steps.size() >= s->cfg.max_steps_in_flight) return issued_direct;
    Slot &sl = s->slots[slot];
    // Staging layout, uploaded with one copy: descriptors, then the CTA
    // prefix (n + 1 entries), the run prefix (one entry per pair + 1) and,
    // when some request runs several sweeps, the pair list.
    BInst *insts = reinterpret_cast<BInst *>(sl.h);
    std::vector<uint32_t> cpv;
    cpv.reserve(s->active.size() + 1);
    std::vector<std::pair<uint32_t, int>> multi;   // (instance, sweeps) of requests running several sweeps
    const size_t max_extra = (size_t)s->cfg.max_step_requests;   // pairs beyond the first pass
    const int64_t multi_below = s->cfg.direct_sweep_bytes > 0 ? s->cfg.direct_sweep_bytes : kDefaultDirectSweepBytes;
    size_t extra = 0;
    uint32_t n = 0;
    uint64_t c = 0;
    int64_t multi_blocks = 0;
    Step step;
    // Slice size: the step aims at step_target_bytes of traffic shared by the
    // requests in it, but each gets at least step_quantum_bytes.
    size_t n_work = 0;
    for (Req *r : s->active) n_work += (!r->issued_all && r->inst.tiles > 0) ? 1 : 0;
    n_work = std::min<size_t>(std::max<size_t>(n_work, 1), (size_t)s->cfg.max_step_requests);
    const size_t quantum = std::max(s->cfg.step_quantum_bytes, s->cfg.step_target_bytes / n_work);
    for (Req *r : s->active) {
        if (r->issued_all) continue;
        if (r->inst.tiles == 0) {                     // nothing to run on the device
            if (write_trivial(s->stream, r->task) != cudaSuccess) r->status = HX_ERR_CUDA;
            r->issued_all = true;
            step.finishing.push_back(r);
            step.members.push_back(r);
            continue;
        }
        if ((int)n >= s->cfg.max_step_requests) continue;
        BInst I = r->inst;
        I.sweep0 = I.kind == kKindStencil ? r->sweep : 0;
        int sweeps = 1;
        if (I.kind == kKindStencil && r->issued == 0 && s->cfg.max_step_sweeps > 1 &&
            8 * (int64_t)I.nx * I.ny < multi_below && I.tiles <= (int64_t)kWsProgWords) {
            sweeps = std::min({I.iters - r->sweep, s->cfg.max_step_sweeps, kMaxStepSweeps});
            if (extra + (size_t)(sweeps - 1) > max_extra) sweeps = 1;
        }
        if (sweeps > 1) {
            I.t_first = 0;
            I.t_count = I.tiles;
            I.n_sweeps = sweeps;
            I.done = I.acc + kWsAccWords;   // the workspace's progress words
        } else {
            const int64_t q = std::max<int64_t>(1, (int64_t)quantum / tile_bytes(I));
            I.t_first = r->issued;
            I.t_count = std::min<int64_t>(q, I.tiles - r->issued);
        }
        if (c + inst_ctas(I) > 0xffffffffull) continue;
        cpv.push_back((uint32_t)c);
        c += inst_ctas(I);
        if (sweeps > 1) {
            multi.emplace_back(n, sweeps);
            extra += (size_t)(sweeps - 1);
            multi_blocks += I.tiles;
        }
        insts[n++] = I;
        step.members.push_back(r);
        if (sweeps > 1) {
            r->sweep += sweeps;
            if (r->sweep < I.iters) continue;
            r->issued_all = true;
            step.finishing.push_back(r);
            continue;
        }
        r->issued += I.t_count;
        if (r->issued == I.tiles) {
            r->issued = 0;
            if (I.kind == kKindStencil && ++r->sweep < I.iters) continue;
            r->issued_all = true;
            step.finishing.push_back(r);
        }
    }
    if (n == 0 && step.finishing.empty()) return issued_direct;
    cpv.push_back((uint32_t)c);
    // Several sweeps: runs as short as keep about two per resident warp in a
    // sweep (at most kMultiSweepRun blocks), as the batch planner does; the
    // pair list is every instance's first pass in order, then each later
    // sweep of the multi-sweep instances in instance order.
    if (!multi.empty()) {
        const int64_t warps = (int64_t)s->ctx->num_sms * s->ctx->batch_ctas_per_sm[1][0] * (kBatchThreads / kWarp);
        const int run = (int)std::max<int64_t>(1, std::min<int64_t>(kMultiSweepRun, multi_blocks / (2 * warps)));
        for (const auto &m : multi) insts[m.first].run_len = run;
    }
    std::vector<uint32_t> pairs, rpv;
    for (uint32_t i = 0; i < n; ++i) pairs.push_back(make_pair(i, 0u));
    int max_sweeps = 1;
    for (const auto &m : multi) max_sweeps = std::max(max_sweeps, m.second);
    for (int ph = 1; ph < max_sweeps; ++ph)
        for (const auto &m : multi)
            if (ph < m.second) pairs.push_back(make_pair(m.first, (uint32_t)ph));
    uint64_t w = 0;
    for (uint32_t pr : pairs) {
        rpv.push_back((uint32_t)w);
        w += inst_runs(insts[pr & (kMaxPairInstances - 1u)]);
    }
    rpv.push_back((uint32_t)w);
    const bool use_pairs = !multi.empty();
    BatchSync sync{s->err_d, kDefaultWaitNs};
    if (use_pairs && s->stall_next) {   // test hook: one instance's waits can never be satisfied
        insts[multi.front().first].stall = 1;
        sync.limit_ns = s->stall_wait_ns;
        s->stall_next = false;
    }
    const size_t off_cta = ((size_t)n * sizeof(BInst) + 15) & ~(size_t)15;
    const size_t off_run = off_cta + (((size_t)(n + 1) * 4 + 15) & ~(size_t)15);
    const size_t off_pairs = off_run + ((rpv.size() * 4 + 15) & ~(size_t)15);
    const size_t bytes = use_pairs ? off_pairs + pairs.size() * 4 : off_run + rpv.size() * 4;
    memcpy(sl.h + off_cta, cpv.data(), (n + 1) * 4);
    memcpy(sl.h + off_run, rpv.data(), rpv.size() * 4);
    if (use_pairs) memcpy(sl.h + off_pairs, pairs.data(), pairs.size() * 4);
    s->active.erase(std::remove_if(s->active.begin(), s->active.end(), [](Req *r) { return r->issued_all; }),
                    s->active.end());
    hx_status st = HX_OK;
    if (n > 0) {
        cudaError_t e = w > 0xffffffffull ? cudaErrorInvalidValue
                                          : cudaMemcpyAsync(sl.d, sl.h, bytes, cudaMemcpyHostToDevice, s->stream);
        if (e != cudaSuccess) st = cuda_fail(e, "server: step upload");
        if (st == HX_OK)
            st = launch_batch_round(s->ctx, reinterpret_cast<const BInst *>(sl.d), n,
                                    reinterpret_cast<const uint32_t *>(sl.d + off_cta),
                                    reinterpret_cast<const uint32_t *>(sl.d + off_run),
                                    use_pairs ? reinterpret_cast<const uint32_t *>(sl.d + off_pairs) : nullptr,
                                    use_pairs ? (uint32_t)pairs.size() : n, (uint32_t)c, (uint32_t)w, 0, s->ctrl,
                                    sync, s->stream);
        s->stats.launches += 1;
    }
    if (st == HX_OK && cudaEventRecord(sl.ev, s->stream) != cudaSuccess) st = HX_ERR_CUDA;
    if (st != HX_OK) {
        // every request with work in the failed step fails, finished or not:
        // a sliced request missing this slice would compute a wrong result
        fail_requests_locked(s, step.members, st);
        s->active.erase(std::remove_if(s->active.begin(), s->active.end(), [](Req *r) { return r->done; }),
                        s->active.end());
        return true;
    }
    sl.busy = true;
    step.ev = sl.ev;
    step.slot = slot;
    push_step_locked(s, std::move(step), 0);
    s->cv_compl.notify_one();
    return true;
}

// Per-launch mode: each admitted request as its own standalone call(s).  A
// stencil request is 20 or more launches, so the launches run with the lock
// released: the completion thread (which takes the lock between events) and
// submitters are not held up by a backlog being issued.  The requests taken
// from `active` are reachable from this thread only until their step is
// queued.
bool issue_per_launch(hx_server *s, std::unique_lock<std::mutex> &lk) {
    if (s->active.empty()) return false;
    std::vector<Req *> batch;
    batch.swap(s->active);
    s->issuing = true;
    for (Req *r : batch) {
        const hx_task t = r->task;
        cudaEvent_t ev = take_event(s);
        s->stats.launches += 1;
        r->issued_all = true;
        lk.unlock();
        hx_status st = ev ? launch_standalone(s, t) : HX_ERR_CUDA;
        if (st == HX_OK && cudaEventRecord(ev, s->stream) != cudaSuccess) st = HX_ERR_CUDA;
        lk.lock();
        std::vector<Req *> one{r};
        if (st != HX_OK) {
            if (ev) s->free_events.push_back(ev);
            fail_requests_locked(s, one, st);
        } else {
            Step step;
            step.ev = ev;
            step.finishing = one;
            push_step_locked(s, std::move(step), 1);
            s->cv_compl.notify_one();
        }
    }
    s->issuing = false;
    s->cv_compl.notify_all();
    return true;
}

void scheduler_main(hx_server *s) {
    cudaSetDevice(s->ctx->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        admit_locked(s);
        if (s->stop && s->queue.empty() && s->active.empty()) break;
        bool issued = false;
        if (!s->active.empty())
            issued = s->cfg.mode == HX_SERVE_CONTINUOUS ? issue_step_locked(s, lk) : issue_per_launch(s, lk);
        if (!issued) s->cv_sched.wait_for(lk, std::chrono::microseconds(200));
    }
    s->cv_compl.notify_all();
}

// Reports the collected completions to cfg.on_done with the lock released.
void report_unlocked(hx_server *s, std::unique_lock<std::mutex> &lk) {
    if (s->to_report.empty()) return;
    std::vector<std::tuple<uint64_t, hx_status, double>> batch;
    batch.swap(s->to_report);
    s->reporting = true;
    lk.unlock();
    for (const auto &d : batch) s->cfg.on_done(s->cfg.on_done_user, std::get<0>(d), std::get<1>(d), std::get<2>(d));
    lk.lock();
    s->reporting = false;
    s->cv_done.notify_all();
}

void completer_main(hx_server *s) {
    cudaSetDevice(s->ctx->device);
    std::unique_lock<std::mutex> lk(s->mu);
    for (;;) {
        while (s->steps.empty()) {
            report_unlocked(s, lk);
            if (s->stop && s->queue.empty() && s->active.empty() && !s->issuing && s->to_report.empty()) return;
            if (!s->steps.empty()) break;
            s->cv_compl.wait_for(lk, std::chrono::milliseconds(5));
        }
        cudaEvent_t ev = s->steps.front().ev;
        lk.unlock();
        const cudaError_t e = cudaEventSynchronize(ev);
        const double t = now_s();
        lk.lock();
        Step step = std::move(s->steps.front());
        s->steps.pop_front();
        if (step.record >= 0) s->timeline[(size_t)step.record].done_s = t - s->created;
        // a wait between two sweeps that ran out of time invalidates every
        // request that had work in the step (they complete with the error)
        if (s->err_h && e == cudaSuccess && __atomic_exchange_n(s->err_h, 0u, __ATOMIC_ACQ_REL) != 0u)
            for (Req *r : step.members) r->status = HX_ERR_TIMEOUT;
        for (Req *r : step.finishing) {
            if (e != cudaSuccess) r->status = HX_ERR_CUDA;
            if (r->status != HX_OK) s->stats.failed += 1;
            r->latency = t - r->arrival;
            r->done = true;
            s->used -= r->footprint;
            s->inflight -= 1;
            if (r->ws >= 0) s->free_ws.push_back(r->ws);
            r->ws = -1;
            s->stats.completed += 1;
            if (s->cfg.on_done) s->to_report.emplace_back(r->id, r->status, r->latency);
        }
        s->stats.footprint_in_flight = s->used;
        if (step.slot >= 0) s->slots[step.slot].busy = false;
        else s->free_events.push_back(step.ev);
        s->cv_sched.notify_all();
        s->cv_done.notify_all();
        report_unlocked(s, lk);
    }
}

hx_status submit_at(hx_server *s, const hx_task *task, double arrival, uint64_t *req_id) {
    if (!s || !task) return fail(HX_ERR_INVALID, "hx_server_submit: NULL argument");
    hx_status st = validate_task(*task, 0, "hx_server_submit");
    if (st != HX_OK) return st;
    auto r = std::make_unique<Req>();
    r->task = *task;
    r->arrival = arrival;
    r->footprint = task_footprint(*task);
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) return fail(HX_ERR_INVALID, "hx_server_submit: server is stopping");
    r->id = s->next_id++;
    if (req_id) *req_id = r->id;
    s->queue.push_back(r.get());
    s->reqs[r->id] = std::move(r);
    s->stats.submitted += 1;
    s->cv_sched.notify_one();
    return HX_OK;
}

}  // namespace
}  // namespace hx

extern "C" {

hx_status hx_server_create(hx_ctx *ctx, const hx_server_config *cfg, hx_server **out) {
    using namespace hx;
    if (!ctx || !cfg || !out) return fail(HX_ERR_INVALID, "hx_server_create: NULL argument");
    *out = nullptr;
    if (cfg->mode != HX_SERVE_CONTINUOUS && cfg->mode != HX_SERVE_PER_LAUNCH)
        return fail(HX_ERR_INVALID, "hx_server_create: unknown mode");
    if (cfg->max_inflight < 0 || cfg->max_inflight > 16384 || cfg->max_steps_in_flight < 0 ||
        cfg->max_steps_in_flight > 64 || cfg->max_step_requests < 0 || cfg->max_step_requests > 65536 ||
        cfg->direct_max < -1 || cfg->direct_max > 65536 || cfg->direct_sweep_bytes < -1 ||
        cfg->max_step_sweeps < 0 || cfg->max_step_sweeps > kMaxStepSweeps)
        return fail(HX_ERR_INVALID, "hx_server_create: bad limits");
    DeviceGuard g(ctx->device);
    hx_server *s = new (std::nothrow) hx_server();
    if (!s) return fail(HX_ERR_NOMEM, "hx_server_create: host allocation failed");
    s->ctx = ctx;
    s->cfg = *cfg;
    s->created = now_s();
    if (s->cfg.max_inflight == 0) s->cfg.max_inflight = 4096;
    if (s->cfg.hbm_budget_bytes == 0) s->cfg.hbm_budget_bytes = ctx->hbm_budget;
    if (s->cfg.max_steps_in_flight == 0) s->cfg.max_steps_in_flight = 4;
    if (s->cfg.max_step_requests == 0) s->cfg.max_step_requests = 4096;
    if (s->cfg.step_quantum_bytes == 0) s->cfg.step_quantum_bytes = (size_t)32 << 20;
    if (s->cfg.step_target_bytes == 0) s->cfg.step_target_bytes = (size_t)512 << 20;
    if (s->cfg.direct_max == 0) s->cfg.direct_max = kDefaultDirectMax;
    if (s->cfg.direct_sweep_bytes == 0) s->cfg.direct_sweep_bytes = kDefaultDirectSweepBytes;
    if (s->cfg.max_step_sweeps == 0) s->cfg.max_step_sweeps = kMaxStepSweeps;
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete s;
        return cuda_fail(e, "hx_server_create: stream");
    }
    if (s->cfg.mode == HX_SERVE_CONTINUOUS) {
        auto align = [](size_t v) { return (v + 255) & ~(size_t)255; };
        const size_t K = (size_t)s->cfg.max_step_requests;
        s->slots.resize((size_t)s->cfg.max_steps_in_flight + 1);
        for (Slot &sl : s->slots) {
            // descriptors, CTA prefix, run prefix and pair list (at most K
            // first passes and K later sweeps)
            sl.bytes = align(K * sizeof(BInst)) + align((K + 1) * 4) + align((2 * K + 1) * 4) + align(2 * K * 4);
            if (e == cudaSuccess) e = cudaMallocHost(&sl.h, sl.bytes);
            if (e == cudaSuccess) e = cudaMalloc(&sl.d, sl.bytes);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.ev, cudaEventDisableTiming);
        }
        const size_t pool = (size_t)s->cfg.max_inflight * kWsBytes;
        if (e == cudaSuccess) e = cudaMalloc(&s->ws_pool, pool + 256);
        if (e == cudaSuccess) e = cudaMemset(s->ws_pool, 0, pool + 256);
        s->ctrl = reinterpret_cast<unsigned int *>(s->ws_pool + pool);
        for (int i = s->cfg.max_inflight - 1; i >= 0; --i) s->free_ws.push_back(i);
        if (e == cudaSuccess) e = cudaHostAlloc(reinterpret_cast<void **>(&s->err_h), 64, cudaHostAllocMapped);
        if (e == cudaSuccess) {
            *s->err_h = 0u;
            e = cudaHostGetDevicePointer(reinterpret_cast<void **>(&s->err_d), s->err_h, 0);
        }
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        for (Slot &sl : s->slots) {
            if (sl.h) cudaFreeHost(sl.h);
            if (sl.d) cudaFree(sl.d);
            if (sl.ev) cudaEventDestroy(sl.ev);
        }
        if (s->ws_pool) cudaFree(s->ws_pool);
        if (s->err_h) cudaFreeHost(s->err_h);
        cudaStreamDestroy(s->stream);
        delete s;
        return cuda_fail(e, "hx_server_create: staging");
    }
    s->sched = std::thread(scheduler_main, s);
    s->compl_thr = std::thread(completer_main, s);
    *out = s;
    return HX_OK;
}

void hx_server_destroy(hx_server *s) {
    if (!s) return;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->stop = true;
    }
    s->cv_sched.notify_all();
    s->cv_compl.notify_all();
    if (s->sched.joinable()) s->sched.join();
    if (s->compl_thr.joinable()) s->compl_thr.join();
    hx::DeviceGuard g(s->ctx->device);
    cudaStreamSynchronize(s->stream);
    hx::release_slot(s->ctx, (hx_stream_t)s->stream);
    for (hx::Slot &sl : s->slots) {
        if (sl.h) cudaFreeHost(sl.h);
        if (sl.d) cudaFree(sl.d);
        if (sl.ev) cudaEventDestroy(sl.ev);
    }
    for (cudaEvent_t ev : s->free_events) cudaEventDestroy(ev);
    if (s->ws_pool) cudaFree(s->ws_pool);
    if (s->err_h) cudaFreeHost(s->err_h);
    cudaStreamDestroy(s->stream);
    delete s;
}

hx_status hx_server_submit(hx_server *s, const hx_task *task, uint64_t *req_id) {
    return hx::submit_at(s, task, hx::now_s(), req_id);
}

hx_status hx_server_poll(hx_server *s, uint64_t req_id, double *latency_s) {
    if (!s) return hx::fail(HX_ERR_INVALID, "hx_server_poll: server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    auto it = s->reqs.find(req_id);
    if (it == s->reqs.end()) return hx::fail(HX_ERR_INVALID, "hx_server_poll: unknown request id");
    const hx::Req &r = *it->second;
    if (!r.done) return HX_ERR_BUSY;
    if (latency_s) *latency_s = r.latency;
    if (r.status != HX_OK) return hx::fail(r.status, "hx_server_poll: the request's launch failed");
    return HX_OK;
}

hx_status hx_server_drain(hx_server *s, double timeout_s) {
    if (!s) return hx::fail(HX_ERR_INVALID, "hx_server_drain: server is NULL");
    std::unique_lock<std::mutex> lk(s->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::duration<double>(timeout_s);
    // every request completed, and every completion reported to on_done
    auto settled = [s] { return s->stats.completed >= s->stats.submitted && s->to_report.empty() && !s->reporting; };
    while (!settled()) {
        if (s->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && !settled())
            return hx::fail(HX_ERR_TIMEOUT, "hx_server_drain: requests still pending at the timeout");
    }
    const bool new_failures = s->stats.failed > s->failed_at_drain;
    s->failed_at_drain = s->stats.failed;
    return new_failures ? hx::fail(HX_ERR_CUDA, "hx_server_drain: some requests' launches failed") : HX_OK;
}

hx_status hx_debug_server_stall(hx_server *s, int64_t wait_limit_ns) {
    if (!s || wait_limit_ns < 0) return hx::fail(HX_ERR_INVALID, "hx_debug_server_stall: bad arguments");
    if (s->cfg.mode != HX_SERVE_CONTINUOUS)
        return hx::fail(HX_ERR_INVALID, "hx_debug_server_stall: continuous mode only");
    std::lock_guard<std::mutex> lk(s->mu);
    s->stall_next = true;
    s->stall_wait_ns = wait_limit_ns;
    return HX_OK;
}

hx_status hx_server_get_timeline(hx_server *s, hx_server_step_record *out, int32_t max, int32_t *n) {
    if (!s || !n || max < 0 || (max > 0 && !out)) return hx::fail(HX_ERR_INVALID, "hx_server_get_timeline: bad arguments");
    std::lock_guard<std::mutex> lk(s->mu);
    const size_t k = std::min(s->timeline.size(), (size_t)max);
    std::copy(s->timeline.begin(), s->timeline.begin() + k, out);
    *n = (int32_t)s->timeline.size();
    return HX_OK;
}

hx_status hx_server_get_stats(hx_server *s, hx_server_stats *out) {
    if (!s || !out) return hx::fail(HX_ERR_INVALID, "hx_server_get_stats: NULL argument");
    std::lock_guard<std::mutex> lk(s->mu);
    *out = s->stats;
    return HX_OK;
}

hx_status hx_server_run_trace(hx_server *s, const hx_task *tasks, const double *arrival_s, int32_t n,
                              double timeout_s, double *latency_s, double *makespan_s) {
    using namespace hx;
    if (!s || n < 0 || (n > 0 && (!tasks || !arrival_s || !latency_s)))
        return fail(HX_ERR_INVALID, "hx_server_run_trace: bad arguments");
    for (int i = 0; i < n; ++i) {
        hx_status st = validate_task(tasks[i], i, "hx_server_run_trace");
        if (st != HX_OK) return st;
        if (i > 0 && arrival_s[i] < arrival_s[i - 1])
            return fail(HX_ERR_INVALID, "hx_server_run_trace: arrival times must be non-decreasing");
    }
    std::vector<uint64_t> ids(n);
    const double t0 = now_s() + 1e-3;
    for (int i = 0; i < n; ++i) {
        const double target = t0 + arrival_s[i];
        for (;;) {
            const double left = target - now_s();
            if (left <= 0.0) break;
            if (left > 3e-4) std::this_thread::sleep_for(std::chrono::microseconds(100));
        }
        hx_status st = submit_at(s, &tasks[i], target, &ids[i]);
        if (st != HX_OK) return st;
    }
    const double last = n ? t0 + arrival_s[n - 1] : t0;
    hx_status st = hx_server_drain(s, std::max(0.0, last - now_s()) + timeout_s);
    double end = t0;
    {
        std::lock_guard<std::mutex> lk(s->mu);
        for (int i = 0; i < n; ++i) {
            auto it = s->reqs.find(ids[i]);
            if (it == s->reqs.end()) continue;
            latency_s[i] = it->second->done ? it->second->latency : -1.0;
            if (it->second->done) end = std::max(end, it->second->arrival + it->second->latency);
            if (it->second->done) s->reqs.erase(it);
        }
    }
    if (makespan_s) *makespan_s = end - t0;
    return st;
}

}  // extern "C"
