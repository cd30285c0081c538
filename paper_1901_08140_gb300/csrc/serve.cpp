// serve.cpp -- the serving form of the C ABI: a request loop with
// continuous batching (bz_server_create, bz_submit, bz_poll, bz_cancel).
//
// Requests (a compiled mixture and a swarm configuration) are queued in
// arrival order.  A worker thread owns S launch slots (one non-blocking CUDA
// stream each).  Whenever a slot is free it takes the request at the head of
// the queue and, in arrival order, further queued requests of its step-kernel
// class (precision, feature instance, field paths, channel tables staged or
// not), looking past requests of other classes -- as many as fit the
// device-memory admission budget, up to a group cap -- and runs them together
// as one batched persistent launch on that slot (bz_create_batch/bz_launch_batch);
// a spawn-mode request (an avalanche) runs alone as its own persistent
// launch (bz_run_swarm).  Running launches are polled without blocking, so
// requests that arrive while others are on the GPU are admitted as soon as a
// slot and memory free up, and their work overlaps on the device.  A
// request's results depend only on its own configuration (counter-based
// random numbers keyed by the swarm seed and the particle ids, one step
// kernel for every launch form, requests grouped by kernel class), so they
// are the same alone and in the mix.
//
// In simulated mode (opts.simulate = n > 0) no device is touched: a launch
// completes after n polls of the worker and reports zero tallies except the
// counts of electrons and real collisions, which lets the scheduling --
// admission, grouping, ordering, cancellation -- be tested on a host
// without a GPU.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "bz.h"
#include "bz_impl.h"

namespace {

enum State { QUEUED, RUNNING, DONE, CANCELLED };

struct Req {
    uint64_t id;
    const bz_mixture *mix;
    bz_swarm_config cfg;
    double bytes;
    int key;        // step-kernel class: requests of one launch share it
    bool alone;     // spawn mode: its own launch
    State state;
    double t_submit, t_admit, t_done;
    uint64_t launch;
    int32_t group_size;
    bz_status status;
    bz_tallies tallies;
};

struct Launch {
    std::vector<uint64_t> ids;
    double bytes;
    bz_batch *batch;
    bz_swarm *swarm;
    int polls_left;  // simulated mode
};

}  // namespace

struct bz_server {
    bz_ctx *ctx;
    bz_server_opts opts;
    std::vector<cudaStream_t> streams;
    std::vector<Launch> slot;       // per slot; empty ids = free
    std::mutex mu;
    std::condition_variable cv;
    std::deque<uint64_t> queue;
    std::unordered_map<uint64_t, Req> reqs;
    uint64_t next_id = 1;
    bool stop = false;
    bool paused = false;  // admission held (bz_server_pause); running launches go on
    std::thread worker;
    std::chrono::steady_clock::time_point t0;
    bz_server_stats st;
};

namespace {

double now_s(const bz_server *s)
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - s->t0).count();
}

// Device bytes a request holds while it runs: the per-electron results of
// its swarm (x, y, z, t and the two energy sums in FP64, the velocity and nu'
// in FP32, seven 32-bit counters: 92 bytes) for every electron slot, the
// birth records of created electrons (40 bytes each) in spawn mode, and 2 MiB
// of per-swarm tally scratch and parameters.
double request_bytes(const bz_swarm_config &c)
{
    const double n = (double)c.n_electrons;
    if (!c.spawn) return 92.0 * n + (double)(2u << 20);
    const double cap = c.pop_cap ? (double)c.pop_cap : 64.0 * n;
    return 92.0 * cap + 40.0 * (cap - n) + (double)(2u << 20);
}

// Step-kernel class of a request (requests of one batched launch share it):
// precision, the feature instance, and whether the lean instance carries the
// magnetic field's paths.
int kernel_key(const bz_mixture *mix, const bz_swarm_config &c, bool simulated)
{
    const bool ext = simulated ? (c.trial_mode == BZ_TRIAL_VARIABLE || c.trial_mode == BZ_TRIAL_BINNED ||
                                  c.gas_temperature_K > 0.0)
                               : bz::needs_feature_instance(mix, &c);
    const bool bf = ext || c.b_T > 0.0;
    // a batch stages channel tables only if every mixture does; one that would
    // stage them alone then searches the cumulative table in L2 instead, which
    // can choose differently where a draw falls within FP32 rounding of a
    // channel boundary -- so such requests form a class of their own
    const bool ch = !simulated && mix && bz::stages_channels(mix, c.precision);
    return (c.precision == 64 ? 4 : 0) | (ext ? 2 : 0) | (bf ? 1 : 0) | (ch ? 8 : 0);
}

// Results of a finished launch (lock held): every request of the launch gets
// its tallies and status, unless it was cancelled meanwhile.
void finish(bz_server *s, Launch &L, const std::vector<bz_tallies> &t, const std::vector<bz_status> &stat)
{
    const double tn = now_s(s);
    for (size_t i = 0; i < L.ids.size(); ++i) {
        auto it = s->reqs.find(L.ids[i]);
        if (it == s->reqs.end()) continue;
        Req &r = it->second;
        if (r.state == CANCELLED) continue;  // its result is dropped
        r.state = DONE;
        r.t_done = tn;
        r.tallies = t[i];
        r.status = stat[i];
        s->st.completed += 1;
    }
    s->st.bytes_in_use -= L.bytes;
    s->st.running -= (int32_t)L.ids.size();
    L = Launch();
}

// Starts the requests `ids` on slot k (called without the lock).
void start(bz_server *s, int k, Launch &L, std::vector<const bz_mixture *> &mixes, std::vector<bz_swarm_config> &cfgs,
           bool alone, std::vector<bz_status> *fail)
{
    if (s->opts.simulate > 0) {
        L.polls_left = s->opts.simulate;
        return;
    }
    bz_status st = BZ_OK;
    if (alone) {
        st = bz_run_swarm(s->ctx, mixes[0], &cfgs[0], (void *)s->streams[k], &L.swarm);
    } else {
        bz_batch_opts o;
        memset(&o, 0, sizeof o);
        o.use_graph = 0;  // each group launches once
        st = bz_create_batch(s->ctx, (int32_t)cfgs.size(), mixes.data(), cfgs.data(), &o, &L.batch);
        if (st == BZ_OK) st = bz_launch_batch(L.batch, (void *)s->streams[k]);
    }
    if (st != BZ_OK) fail->assign(cfgs.size(), st);
}

// Polls slot k's launch without blocking (called without the lock); true
// when it has ended, with its tallies and statuses.
bool poll(bz_server *s, Launch &L, std::vector<bz_tallies> *t, std::vector<bz_status> *stat)
{
    const size_t n = L.ids.size();
    t->assign(n, bz_tallies());
    stat->assign(n, BZ_OK);
    if (s->opts.simulate > 0) {
        if (--L.polls_left > 0) return false;
        return true;  // filled by the caller from the configurations
    }
    if (L.swarm) {
        bz_status q = bz_query_tallies(L.swarm, &(*t)[0]);
        if (q == BZ_ENOTREADY) return false;
        (*stat)[0] = q;
        bz_destroy_swarm(L.swarm);
        L.swarm = nullptr;
        return true;
    }
    if (L.batch) {
        bz_status q = bz_batch_query(L.batch);
        if (q == BZ_ENOTREADY) return false;
        if (q == BZ_OK) {
            bz_batch_read_tallies(L.batch, t->data());
            for (size_t i = 0; i < n; ++i) {
                const int32_t f = (*t)[i].error_flags;
                (*stat)[i] = (f & BZ_ERR_STAGE_TIMEOUT) ? BZ_ETIMEOUT : (f & BZ_ERR_TRIAL) ? BZ_ETRIAL : BZ_OK;
            }
        } else {
            stat->assign(n, q);
        }
        bz_destroy_batch(L.batch);
        L.batch = nullptr;
        return true;
    }
    return true;  // the launch failed to start: its statuses are set already
}

// How deep admission looks past the head of the queue for requests of the
// head's class.
constexpr size_t kLookahead = 4096;

void work(bz_server *s)
{
    if (s->ctx && s->opts.simulate <= 0) cudaSetDevice(bz::ctx_device(s->ctx));
    std::unique_lock<std::mutex> lock(s->mu);
    const int S = (int)s->streams.size() > 0 ? (int)s->streams.size() : s->opts.n_slots;
    while (true) {
        bool progressed = false;
        // admission: the queue's head first, in arrival order
        for (int k = 0; k < S && !s->queue.empty() && !s->paused; ++k) {
            if (!s->slot[k].ids.empty()) continue;
            const Req &head = s->reqs[s->queue.front()];
            if (s->st.bytes_in_use + head.bytes > s->opts.memory_budget_bytes) break;
            Launch L;
            L.bytes = 0.0;
            L.batch = nullptr;
            L.swarm = nullptr;
            L.polls_left = 0;
            std::vector<const bz_mixture *> mixes;
            std::vector<bz_swarm_config> cfgs;
            bool alone = false;
            const double tn = now_s(s);
            // The head first; then, in arrival order, queued requests of the
            // head's step-kernel class from further down the queue (at most
            // kLookahead entries deep), so that a request of another class in
            // between -- an avalanche, which runs alone -- does not cut the
            // launch short.  The head is always admitted first, so no request
            // waits behind a later one of its own class; one of another class
            // waits at most for this launch to be formed.
            size_t scanned = 0;
            for (auto it = s->queue.begin();
                 it != s->queue.end() && (int)L.ids.size() < s->opts.max_group && scanned < kLookahead; ++scanned) {
                Req &r = s->reqs[*it];
                if (!L.ids.empty() && (r.alone || r.key != s->reqs[L.ids[0]].key)) {
                    ++it;
                    continue;
                }
                if (s->st.bytes_in_use + L.bytes + r.bytes > s->opts.memory_budget_bytes) break;
                it = s->queue.erase(it);
                r.state = RUNNING;
                r.t_admit = tn;
                r.launch = s->st.launches;
                L.ids.push_back(r.id);
                L.bytes += r.bytes;
                mixes.push_back(r.mix);
                cfgs.push_back(r.cfg);
                if (r.alone) {
                    alone = true;
                    break;
                }
            }
            for (uint64_t id : L.ids) s->reqs[id].group_size = (int32_t)L.ids.size();
            s->st.launches += 1;
            s->st.bytes_in_use += L.bytes;
            s->st.peak_bytes_in_use = std::max(s->st.peak_bytes_in_use, s->st.bytes_in_use);
            s->st.running += (int32_t)L.ids.size();
            s->st.max_running = std::max(s->st.max_running, s->st.running);
            s->st.queued = (int32_t)s->queue.size();
            s->slot[k] = L;
            // launch outside the lock; the slot is marked busy already
            Launch local = L;
            lock.unlock();
            std::vector<bz_status> fail;
            start(s, k, local, mixes, cfgs, alone, &fail);
            lock.lock();
            s->slot[k].batch = local.batch;
            s->slot[k].swarm = local.swarm;
            s->slot[k].polls_left = local.polls_left;
            if (!fail.empty()) {
                std::vector<bz_tallies> t(fail.size(), bz_tallies());
                for (auto &x : t) memset(&x, 0, sizeof x);
                finish(s, s->slot[k], t, fail);
            }
            progressed = true;
        }
        // completions
        for (int k = 0; k < S; ++k) {
            if (s->slot[k].ids.empty()) continue;
            Launch local = s->slot[k];
            lock.unlock();
            std::vector<bz_tallies> t;
            std::vector<bz_status> stat;
            const bool ended = poll(s, local, &t, &stat);
            lock.lock();
            s->slot[k].polls_left = local.polls_left;
            if (!ended) continue;
            if (s->opts.simulate > 0) {
                for (size_t i = 0; i < local.ids.size(); ++i) {
                    memset(&t[i], 0, sizeof t[i]);
                    auto it = s->reqs.find(local.ids[i]);
                    if (it == s->reqs.end()) continue;
                    t[i].n_particles = it->second.cfg.n_electrons;
                    t[i].n_real = it->second.cfg.n_electrons * (uint64_t)it->second.cfg.real_collisions;
                }
            }
            s->slot[k].batch = nullptr;
            s->slot[k].swarm = nullptr;
            finish(s, s->slot[k], t, stat);
            progressed = true;
        }
        s->st.queued = (int32_t)s->queue.size();
        if (s->stop && s->st.running == 0) break;
        if (!progressed) {
            if (s->st.running == 0 && (s->queue.empty() || s->paused) && !s->stop)
                s->cv.wait(lock);  // idle: until a submission or the stop
            else
                s->cv.wait_for(lock, std::chrono::microseconds(20));
        }
    }
}

bz_status fail_msg(bz_status st, const char *msg)
{
    bz::set_last_error(msg);
    return st;
}

}  // namespace

extern "C" {

bz_status bz_server_create(bz_ctx *ctx, const bz_server_opts *opts, bz_server **out)
{
    if (!out) return fail_msg(BZ_EINVAL, "null output");
    *out = nullptr;
    bz_server_opts o;
    memset(&o, 0, sizeof o);
    if (opts) o = *opts;
    if (!(o.memory_budget_bytes > 0.0)) o.memory_budget_bytes = 60e9;
    if (o.n_slots <= 0) o.n_slots = 3;
    if (o.max_group <= 0) o.max_group = 512;
    if (o.max_group > 65535) return fail_msg(BZ_EINVAL, "max_group is at most 65535 (a batch's limit)");
    if (o.n_slots > 64) return fail_msg(BZ_EINVAL, "n_slots is at most 64");
    if (o.simulate < 0) return fail_msg(BZ_EINVAL, "simulate must be >= 0");
    if (o.simulate == 0 && !ctx) return fail_msg(BZ_EINVAL, "a server on the GPU needs a context");
    bz_server *s = new (std::nothrow) bz_server();
    if (!s) return fail_msg(BZ_ENOMEM, "host allocation");
    s->ctx = ctx;
    s->opts = o;
    memset(&s->st, 0, sizeof s->st);
    s->t0 = std::chrono::steady_clock::now();
    if (o.simulate == 0) {
        cudaError_t e = cudaSetDevice(bz::ctx_device(ctx));
        for (int k = 0; k < o.n_slots && e == cudaSuccess; ++k) {
            cudaStream_t st = nullptr;
            e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
            if (e == cudaSuccess) s->streams.push_back(st);
        }
        if (e != cudaSuccess) {
            for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
            delete s;
            bz::set_last_error(std::string("server streams: ") + cudaGetErrorString(e));
            return BZ_ECUDA;
        }
    }
    s->slot.assign(o.n_slots, Launch());
    s->worker = std::thread(work, s);
    *out = s;
    return BZ_OK;
}

bz_status bz_submit(bz_server *s, const bz_mixture *mix, const bz_swarm_config *cfg, uint64_t *request_id)
{
    if (!s || !cfg || !request_id) return fail_msg(BZ_EINVAL, "null argument");
    if (s->opts.simulate == 0 && !mix) return fail_msg(BZ_EINVAL, "null mixture");
    bz_status st = bz::check_config(cfg);
    if (st != BZ_OK) return st;
    Req r;
    memset(&r.tallies, 0, sizeof r.tallies);
    r.mix = mix;
    r.cfg = *cfg;
    r.bytes = request_bytes(*cfg);
    if (r.bytes > s->opts.memory_budget_bytes)
        return fail_msg(BZ_EBUDGET, "the request alone needs more device memory than the admission budget");
    r.key = kernel_key(mix, *cfg, s->opts.simulate > 0);
    r.alone = cfg->spawn != 0;
    r.state = QUEUED;
    r.t_admit = r.t_done = 0.0;
    r.launch = 0;
    r.group_size = 0;
    r.status = BZ_OK;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        r.id = s->next_id++;
        r.t_submit = now_s(s);
        s->reqs[r.id] = r;
        s->queue.push_back(r.id);
        s->st.submitted += 1;
        s->st.queued = (int32_t)s->queue.size();
        *request_id = r.id;
    }
    s->cv.notify_one();
    return BZ_OK;
}

bz_status bz_poll(bz_server *s, uint64_t request_id, bz_tallies *out, bz_request_info *info)
{
    if (!s) return fail_msg(BZ_EINVAL, "null server");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end()) return fail_msg(BZ_EINVAL, "unknown request (never submitted, or already delivered)");
    Req &r = it->second;
    if (r.state == CANCELLED) {
        s->reqs.erase(it);
        return BZ_ECANCEL;
    }
    if (r.state != DONE) return BZ_ENOTREADY;
    if (out) *out = r.tallies;
    if (info) {
        info->t_submit = r.t_submit;
        info->t_admit = r.t_admit;
        info->t_done = r.t_done;
        info->launch = r.launch;
        info->group_size = r.group_size;
        info->status = r.status;
    }
    const bz_status st = r.status;
    s->reqs.erase(it);
    if (st != BZ_OK) bz::set_last_error("the request's launch reported an error (see bz_request_info.status)");
    return st;
}

bz_status bz_cancel(bz_server *s, uint64_t request_id)
{
    if (!s) return fail_msg(BZ_EINVAL, "null server");
    std::lock_guard<std::mutex> lock(s->mu);
    auto it = s->reqs.find(request_id);
    if (it == s->reqs.end()) return fail_msg(BZ_EINVAL, "unknown request (never submitted, or already delivered)");
    Req &r = it->second;
    if (r.state == CANCELLED) return BZ_OK;
    if (r.state == QUEUED) {
        s->queue.erase(std::find(s->queue.begin(), s->queue.end(), request_id));
        s->st.queued = (int32_t)s->queue.size();
    }
    // a running request's launch goes on with the rest of its group; its
    // result is dropped, and its memory released, when the launch ends
    r.state = CANCELLED;
    s->st.cancelled += 1;
    return BZ_OK;
}

bz_status bz_server_pause(bz_server *s, int32_t paused)
{
    if (!s) return fail_msg(BZ_EINVAL, "null server");
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->paused = paused != 0;
    }
    s->cv.notify_one();
    return BZ_OK;
}

bz_status bz_server_get_stats(bz_server *s, bz_server_stats *out)
{
    if (!s || !out) return fail_msg(BZ_EINVAL, "null argument");
    std::lock_guard<std::mutex> lock(s->mu);
    *out = s->st;
    return BZ_OK;
}

void bz_server_destroy(bz_server *s)
{
    if (!s) return;
    {
        std::lock_guard<std::mutex> lock(s->mu);
        s->stop = true;
        // queued requests never start
        for (uint64_t id : s->queue) s->reqs[id].state = CANCELLED;
        s->queue.clear();
    }
    s->cv.notify_all();
    if (s->worker.joinable()) s->worker.join();
    for (cudaStream_t st : s->streams) cudaStreamDestroy(st);
    delete s;
}

}  // extern "C"
