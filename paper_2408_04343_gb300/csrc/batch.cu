// Batched and served forms: many independent systems advanced together.
//
// A batch owns a worker thread that runs continuous batching in rounds:
//  1. admission -- queued systems are admitted first come first served while
//     the device memory of the systems the batch holds stays within the
//     budget; a system created with SNP_FLAG_DEFER_UPLOAD is uploaded only
//     here, so requests wait on the host until memory frees up (a destroyed
//     system returns its memory to the batch);
//  2. one round -- every admitted system advances by up to `round` steps.
//     Systems small enough for one CTA (the CTA-resident engine, emissions in
//     shared memory) share ONE persistent launch: each CTA takes the next
//     system, largest first, from a device work counter and runs all of that
//     system's steps of the round, with per-system offsets in a table of
//     system descriptors.  Larger systems run on the grid-wide engines on
//     their own streams at the same time, so their work overlaps;
//  3. retirement -- systems that used up their steps or reached a fixed
//     point leave; a ticket completes when all its systems have.
// Requests that arrive while a round runs join at the next round, so the
// device stays busy and new work does not wait for old work to drain.
// Results depend only on each system's seed and state, never on what it
// shared a round with (the Philox key is per system).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <set>
#include <string>
#include <thread>
#include <vector>

#include "kernels.h"
#include "snp_internal.h"
#include "system.h"

namespace snp {

struct Item {
    int64_t ticket = 0;
    snp_system* sys = nullptr;
    int64_t remaining = 0;
    int64_t done = 0;
    bool finished = false;
};

struct Ticket {
    std::vector<std::unique_ptr<Item>> items;
    int64_t outstanding = 0;
    int status = SNP_OK;
    std::string error;
    bool complete() const { return outstanding == 0; }
};

constexpr int64_t kRoundSteps = 64;          // steps per round and system

// Online autotuner of the resident launch.  A candidate is a CTA size
// (256, 512 or 1,024 threads) and whether the round's largest systems --
// those holding at least one CTA's share of the round's work -- get a
// launch of their own: one 1,024-thread CTA each with up to 64 registers,
// beside the persistent 32-register launch for the rest.  Launches are
// grouped by (bits per emission, log2 of the largest system); for each group
// every candidate is tried on one real round (the work is not wasted:
// results do not depend on the candidate), then the fastest by measured
// synaptic updates per second is used.  With SNP_AUTOTUNE_CACHE naming a
// file, choices are read at batch creation and written back at destroy.
struct Autotune {
    static constexpr int kN = 6;
    static constexpr int kThreads[3] = {256, 512, 1024};
    static int threads_of(int c) { return kThreads[c % 3]; }
    static bool split_of(int c) { return c >= 3; }
    struct Stat {
        double work[kN] = {0, 0, 0, 0, 0, 0};
        double secs[kN] = {0, 0, 0, 0, 0, 0};
    };
    std::map<std::pair<int, int>, Stat> stats;
    int pick(const std::pair<int, int>& key) {
        Stat& st = stats[key];
        for (int c = 0; c < kN; ++c)
            if (st.secs[c] == 0.0) return c;
        int best = 0;
        for (int c = 1; c < kN; ++c)
            if (st.work[c] / st.secs[c] > st.work[best] / st.secs[best]) best = c;
        return best;
    }
    void record(const std::pair<int, int>& key, int c, double work, double secs) {
        Stat& st = stats[key];
        st.work[c] += work;
        st.secs[c] += secs > 1e-9 ? secs : 1e-9;
    }
    void load(const char* path) {
        FILE* f = path ? fopen(path, "r") : nullptr;
        if (!f) return;
        int eb, lq, c;
        double w, t;
        while (fscanf(f, "%d %d %d %lf %lf", &eb, &lq, &c, &w, &t) == 5)
            if (c >= 0 && c < kN) record({eb, lq}, c, w, t);
        fclose(f);
    }
    void save(const char* path) const {
        FILE* f = path ? fopen(path, "w") : nullptr;
        if (!f) return;
        for (const auto& kv : stats)
            for (int c = 0; c < kN; ++c)
                if (kv.second.secs[c] > 0.0)
                    fprintf(f, "%d %d %d %.6g %.6g\n", kv.first.first, kv.first.second, c, kv.second.work[c],
                            kv.second.secs[c]);
        fclose(f);
    }
};
constexpr int Autotune::kThreads[3];
constexpr int kBatchResidentMaxQ = 65536;    // larger systems run grid-wide

}  // namespace snp

struct snp_batch {
    snp_options opt{};
    size_t budget = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<snp::Item*> pending;
    std::vector<snp::Item*> active;
    std::map<int64_t, snp::Ticket> tickets;
    std::set<snp_system*> owned;   // systems this batch uploaded (memory accounting)
    size_t resident_bytes = 0;
    size_t peak_bytes = 0;
    int64_t rounds = 0, admitted = 0, finished = 0;
    int64_t next_id = 1;
    bool stop = false;
    bool admitting = false;        // the uploader is uploading a system outside the lock
    size_t reserved = 0;           // device bytes of the system being uploaded (within the budget)
    std::deque<snp::Item*> ready;  // uploaded, waiting for the next round
    std::thread worker;
    std::thread uploader;
    // device tables of the resident launch, grown on demand
    snp::DevSys* d_sys = nullptr;
    long long* d_nsteps = nullptr;
    unsigned long long* d_res = nullptr;  // 3 words per system
    unsigned int* d_work = nullptr;
    size_t cap = 0;
    int sms = 0;
    int threads = 0;
    int64_t round = snp::kRoundSteps;
    snp::Autotune tune;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    cudaStream_t stream2 = nullptr;        // the largest systems' launch
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // where the worker's time goes (seconds, host clock unless noted)
    double t_admit = 0;        // uploading admitted systems
    double t_launch = 0;       // queueing the grid-wide systems' steps of a round
    double t_resident = 0;     // the resident launches of a round, tables to results
    double t_resident_dev = 0; // the resident launches on the device (CUDA events)
    double t_large_tail = 0;   // waiting for grid-wide systems after the resident launches
    double t_idle = 0;         // no admissible system and nothing running
    double t_round = 0;        // whole rounds
};

namespace snp {

static int grow_tables(snp_batch* b, size_t n) {
    if (n <= b->cap) return SNP_OK;
    size_t cap = std::max<size_t>(n, 2 * b->cap);
    cudaFree(b->d_sys);
    cudaFree(b->d_nsteps);
    cudaFree(b->d_res);
    b->d_sys = nullptr;
    b->d_nsteps = nullptr;
    b->d_res = nullptr;
    if (cudaMalloc(&b->d_sys, cap * sizeof(DevSys)) != cudaSuccess ||
        cudaMalloc(&b->d_nsteps, cap * sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&b->d_res, cap * 3 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        b->cap = 0;
        return fail(SNP_ERR_OOM, "batch table allocation failed");
    }
    b->cap = cap;
    return SNP_OK;
}

// CTAs of `threads` threads and `smem` bytes that fit on one SM.
static int ctas_per_sm(int threads, size_t smem) {
    int dev = 0, smem_sm = 0, thr_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    const int by_thr = thr_sm / threads;
    const int by_smem = (int)((size_t)smem_sm / (smem + 1024));
    return std::max(1, std::min(by_thr, by_smem));
}

// One persistent launch over systems that share kernel template parameters;
// steps[i] each; exec_out receives the executed steps.
static int run_resident_group(snp_batch* b, std::vector<snp_system*>& sys, std::vector<int64_t>& steps,
                              std::vector<int64_t>& exec_out, double& dev_seconds) {
    const size_t n = sys.size();
    exec_out.assign(n, 0);
    if (n == 0) return SNP_OK;
    int rc = grow_tables(b, n);
    if (rc) return rc;
    std::vector<size_t> order(n);
    for (size_t i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t c) {
        return (double)(sys[a]->nsyn + sys[a]->q) * steps[a] > (double)(sys[c]->nsyn + sys[c]->q) * steps[c];
    });
    std::vector<DevSys> tab(n);
    std::vector<long long> ns(n);
    int max_q = 0, max_p = 0;
    for (size_t r = 0; r < n; ++r) {
        tab[r] = sys[order[r]]->dev;
        ns[r] = steps[order[r]];
        max_q = std::max(max_q, sys[order[r]]->q);
        max_p = std::max(max_p, sys[order[r]]->max_p);
    }
    ResidentPlan plan;
    plan.e_bits = resident_e_bits(max_p);
    int lq = 0;
    while ((1 << lq) < max_q) ++lq;
    const std::pair<int, int> key{plan.e_bits, lq};
    const int cand = b->threads > 0 ? -1 : b->tune.pick(key);
    plan.threads = cand < 0 ? b->threads : Autotune::threads_of(cand);
    const bool split = cand >= 0 && Autotune::split_of(cand);
    const bool compact = sys[0]->compact;
    const int sel = sys[0]->opt.select;
    std::vector<double> wk(n);
    double work = 0.0;
    for (size_t r = 0; r < n; ++r) {
        wk[r] = (double)(sys[order[r]]->nsyn + sys[order[r]]->q) * ns[r];
        work += wk[r];
    }
    // the largest systems (largest first in the table): each holds at least
    // one CTA's share of the round's work
    size_t nbig = 0;
    if (split) {
        plan.smem = resident_smem_bytes(max_q, plan.e_bits);
        const double share = work / (double)(b->sms * ctas_per_sm(plan.threads, plan.smem));
        while (nbig < n && nbig < (size_t)b->sms && wk[nbig] >= share) ++nbig;
    }
    int max_q_rest = 0;
    for (size_t r = nbig; r < n; ++r) max_q_rest = std::max(max_q_rest, sys[order[r]]->q);
    plan.max_q = max_q_rest;
    plan.smem = resident_smem_bytes(max_q_rest, plan.e_bits);
    plan.ctas = b->sms * ctas_per_sm(plan.threads, plan.smem);
    if (cudaMemcpyAsync(b->d_sys, tab.data(), n * sizeof(DevSys), cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaMemcpyAsync(b->d_nsteps, ns.data(), n * sizeof(long long), cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaMemsetAsync(b->d_work, 0, 2 * sizeof(unsigned int), b->stream) != cudaSuccess)
        return fail(SNP_ERR_CUDA, "batch table upload");
    cudaEventRecord(b->ev0, b->stream);
    if (nbig) {
        ResidentPlan pb = plan;
        pb.big = true;
        pb.threads = 1024;
        pb.max_q = max_q;
        pb.smem = resident_smem_bytes(max_q, plan.e_bits);
        pb.ctas = (int)nbig;
        if (cudaEventRecord(b->ev_fork, b->stream) != cudaSuccess ||
            cudaStreamWaitEvent(b->stream2, b->ev_fork, 0) != cudaSuccess ||
            launch_resident(b->d_sys, b->d_nsteps, (int)nbig, b->d_work + 1, pb, compact, sel, b->stream2) !=
                cudaSuccess ||
            cudaEventRecord(b->ev_join, b->stream2) != cudaSuccess)
            return fail(SNP_ERR_CUDA, std::string("resident launch: ") + cudaGetErrorString(cudaGetLastError()));
    }
    if (n > nbig && launch_resident(b->d_sys + nbig, b->d_nsteps + nbig, (int)(n - nbig), b->d_work, plan, compact,
                                    sel, b->stream) != cudaSuccess)
        return fail(SNP_ERR_CUDA, std::string("resident launch: ") + cudaGetErrorString(cudaGetLastError()));
    if (nbig && cudaStreamWaitEvent(b->stream, b->ev_join, 0) != cudaSuccess)
        return fail(SNP_ERR_CUDA, "batch stream join");
    cudaEventRecord(b->ev1, b->stream);
    std::vector<unsigned long long> ex(n * 3);
    if (launch_gather_results(b->d_sys, (int)n, b->d_res, b->stream) != cudaSuccess ||
        cudaMemcpyAsync(ex.data(), b->d_res, n * 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, b->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return fail(SNP_ERR_CUDA, std::string("batch sync: ") + cudaGetErrorString(cudaGetLastError()));
    {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, b->ev0, b->ev1) == cudaSuccess) {
            dev_seconds += ms * 1e-3;
            if (cand >= 0) b->tune.record(key, cand, work, ms * 1e-3);
        }
    }
    bool overflow = false, bounds = false;
    for (size_t r = 0; r < n; ++r) {
        exec_out[order[r]] = (int64_t)ex[3 * r + 1];
        sys[order[r]]->host_step = ex[3 * r + 0];
        overflow |= (ex[3 * r + 2] & 1ull) != 0ull;
        bounds |= (ex[3 * r + 2] & 2ull) != 0ull;
    }
    if (bounds) return fail(SNP_ERR_INVALID, "bounds check: an index out of range in a batched system");
    if (overflow) return fail(SNP_ERR_OVERFLOW, "a spike count left the int32 range in a batched system");
    return SNP_OK;
}

static bool batch_resident(const snp_system* s) {
    return s->opt.form == SNP_FORM_OPT && s->opt.prop == SNP_PROP_PULL && s->opt.engine != SNP_ENGINE_LAUNCH &&
           s->opt.engine != SNP_ENGINE_TILED && s->q <= kBatchResidentMaxQ && resident_fits(s, nullptr);
}

static double now_s() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

// Where one round's time went (added to the batch's counters under its lock).
struct RoundTimes {
    double launch = 0, resident = 0, resident_dev = 0, large_tail = 0, round = 0;
};

// Runs one round over `items`; on return each item's done/remaining/finished is updated.
static int run_round(snp_batch* b, std::vector<Item*>& items, RoundTimes& tm) {
    const double t0 = now_s();
    std::map<std::pair<int, int>, std::vector<Item*>> groups;
    std::vector<Item*> large;
    for (Item* it : items) {
        if (batch_resident(it->sys))
            groups[{it->sys->compact ? 1 : 0, it->sys->opt.select}].push_back(it);
        else
            large.push_back(it);
    }
    int rc = SNP_OK;
    // grid-wide systems first (asynchronous on their own streams)
    std::vector<int64_t> large_n(large.size());
    for (size_t i = 0; i < large.size() && !rc; ++i) {
        large_n[i] = std::min(large[i]->remaining, b->round);
        rc = run_steps_graphed(large[i]->sys, large_n[i]);
    }
    const double t1 = now_s();
    for (auto& g : groups) {
        if (rc) break;
        std::vector<snp_system*> sys;
        std::vector<int64_t> steps, ex;
        for (Item* it : g.second) {
            sys.push_back(it->sys);
            steps.push_back(std::min(it->remaining, b->round));
        }
        rc = run_resident_group(b, sys, steps, ex, tm.resident_dev);
        if (!rc) {
            for (size_t r = 0; r < g.second.size(); ++r) {
                Item* it = g.second[r];
                it->done += ex[r];
                it->remaining -= steps[r];
                if (ex[r] < steps[r] || it->remaining <= 0) it->finished = true;
            }
        }
    }
    const double t2 = now_s();
    for (size_t i = 0; i < large.size(); ++i) {
        int64_t ex = 0;
        const int r2 = read_flags(large[i]->sys, &ex);
        if (!rc) rc = r2;
        large[i]->done += ex;
        large[i]->remaining -= large_n[i];
        if (ex < large_n[i] || large[i]->remaining <= 0) large[i]->finished = true;
    }
    const double t3 = now_s();
    tm.launch = t1 - t0;
    tm.resident = t2 - t1;
    tm.large_tail = t3 - t2;
    tm.round = t3 - t0;
    return rc;
}

static void finish_item(snp_batch* b, Item* it, int rc, const std::string& err) {
    // b->mu held
    Ticket& t = b->tickets[it->ticket];
    it->finished = true;
    if (rc && !t.status) {
        t.status = rc;
        t.error = err;
    }
    it->sys->busy.store(0);
    t.outstanding -= 1;
    b->finished += 1;
}

// b->mu held.  The budget is a hard bound on the device memory of the systems
// this batch uploaded: the first waiting system is admitted only if it fits
// beside them.  Finished systems keep their memory until they are destroyed
// (their state is still read), so once nothing is running, only a destroy
// can make room.
static bool front_fits(const snp_batch* b) {
    if (b->pending.empty()) return false;
    const snp_system* s = b->pending.front()->sys;
    const size_t need = s->materialized ? 0 : s->planned_bytes;
    return !b->budget || b->resident_bytes + b->reserved + need <= b->budget;
}

// b->mu held.  Waiting systems that nothing but a destroy can admit: no
// system runs, waits for a round or is being uploaded, and the first waiting
// one does not fit.
static bool stalled(const snp_batch* b) {
    return !b->admitting && b->active.empty() && b->ready.empty() && !b->pending.empty() && !front_fits(b);
}

// Admission runs on a thread of its own, so uploads overlap the rounds:
// first come first served, the first waiting system is uploaded (its stream
// created, its device memory reserved within the budget, then allocated and
// copied) while the worker steps the systems already admitted; it joins the
// round after the upload.  On destroy the uploader stops once nothing that
// waits fits.
static void uploader_main(snp_batch* b) {
    std::unique_lock<std::mutex> lk(b->mu);
    for (;;) {
        b->cv.wait(lk, [&] { return b->stop || front_fits(b); });
        if (!front_fits(b)) return;  // stopping, and nothing that waits fits
        // systems already on the device need no upload: admit every one that
        // leads the queue at once, so they start in the same round
        bool moved = false;
        while (front_fits(b) && b->pending.front()->sys->materialized && b->pending.front()->sys->stream) {
            Item* it = b->pending.front();
            b->pending.pop_front();
            if (it->remaining <= 0) {
                finish_item(b, it, SNP_OK, "");
            } else {
                b->ready.push_back(it);
                b->admitted += 1;
            }
            moved = true;
        }
        if (moved) {
            b->cv.notify_all();
            continue;
        }
        Item* it = b->pending.front();
        snp_system* s = it->sys;
        b->pending.pop_front();
        const size_t need = s->materialized ? 0 : s->planned_bytes;
        b->reserved += need;
        b->admitting = true;
        lk.unlock();
        const double a0 = now_s();
        int rc = SNP_OK;
        if (!s->stream) {
            // a stream of its own lets grid-wide systems overlap; a blocking
            // stream keeps the legacy default stream's ordering
            cudaStream_t st = nullptr;
            if (cudaStreamCreate(&st) == cudaSuccess) {
                s->stream = st;
                s->own_stream = true;
            } else {
                cudaGetLastError();
            }
        }
        const bool upload = !s->materialized;
        if (upload) rc = materialize(s);
        const std::string err = rc ? last_error() : "";
        const double a1 = now_s();
        lk.lock();
        b->admitting = false;
        b->reserved -= need;
        b->t_admit += a1 - a0;
        if (!rc && upload) {
            b->resident_bytes += s->device_bytes;
            b->peak_bytes = std::max(b->peak_bytes, b->resident_bytes);
            b->owned.insert(s);
            s->owner = b;
        }
        if (rc)
            finish_item(b, it, rc, err);
        else if (it->remaining <= 0)
            finish_item(b, it, SNP_OK, "");
        else {
            b->ready.push_back(it);
            b->admitted += 1;
        }
        b->cv.notify_all();
    }
}

static void worker_main(snp_batch* b) {
    std::unique_lock<std::mutex> lk(b->mu);
    for (;;) {
        // work arrives from the uploader; a waiting system that does not fit
        // wakes the uploader only when a destroy returns memory
        {
            const double w0 = now_s();
            b->cv.wait(lk, [&] {
                return !b->ready.empty() || !b->active.empty() || (b->stop && !b->admitting && !front_fits(b));
            });
            b->t_idle += now_s() - w0;
        }
        if (b->ready.empty() && b->active.empty()) {
            // destroyed: what still waits does not fit; release it unrun
            for (Item* it : b->pending) finish_item(b, it, SNP_ERR_BUSY, "batch destroyed before admission");
            b->pending.clear();
            b->cv.notify_all();
            return;
        }
        while (!b->ready.empty()) {
            b->active.push_back(b->ready.front());
            b->ready.pop_front();
        }
        if (b->active.empty()) continue;
        b->rounds += 1;
        std::vector<Item*> items = b->active;
        lk.unlock();
        RoundTimes tm;
        const int rc = run_round(b, items, tm);
        const std::string err = rc ? last_error() : "";
        lk.lock();
        b->t_launch += tm.launch;
        b->t_resident += tm.resident;
        b->t_resident_dev += tm.resident_dev;
        b->t_large_tail += tm.large_tail;
        b->t_round += tm.round;
        std::vector<Item*> still;
        for (Item* it : b->active) {
            if (rc || it->finished)
                finish_item(b, it, rc, err);
            else
                still.push_back(it);
        }
        b->active.swap(still);
        b->cv.notify_all();
    }
}

// Called by snp_destroy: the system's memory returns to its batch's budget.
void batch_release(snp_system* s) {
    snp_batch* b = s->owner;
    if (!b) return;
    std::lock_guard<std::mutex> lk(b->mu);
    if (b->owned.erase(s)) b->resident_bytes -= std::min(b->resident_bytes, s->device_bytes);
    s->owner = nullptr;
    b->cv.notify_all();
}

}  // namespace snp

using namespace snp;

extern "C" {

int snp_batch_create(const snp_options* opts, size_t mem_budget, snp_batch** out) {
    if (!out) return fail(SNP_ERR_INVALID, "out is NULL");
    *out = nullptr;
    snp_batch* b = new (std::nothrow) snp_batch();
    if (!b) return fail(SNP_ERR_OOM, "host allocation failed");
    if (opts) b->opt = *opts;
    b->budget = mem_budget;
    b->threads = opts ? opts->threads : 0;
    if (b->opt.stream) {
        b->stream = (cudaStream_t)b->opt.stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete b;
            return fail(SNP_ERR_CUDA, "stream create");
        }
        b->own_stream = true;
    }
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaMalloc(&b->d_work, 2 * sizeof(unsigned int)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&b->stream2, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(b->d_work);
        if (b->own_stream) cudaStreamDestroy(b->stream);
        delete b;
        return fail(SNP_ERR_OOM, "device allocation failed");
    }
    cudaEventCreate(&b->ev0);
    cudaEventCreate(&b->ev1);
    cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming);
    cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming);
    b->tune.load(getenv("SNP_AUTOTUNE_CACHE"));
    b->worker = std::thread(worker_main, b);
    b->uploader = std::thread(uploader_main, b);
    *out = b;
    return SNP_OK;
}

int snp_batch_destroy(snp_batch* b) {
    if (!b) return SNP_OK;
    {
        std::lock_guard<std::mutex> lk(b->mu);
        b->stop = true;
    }
    b->cv.notify_all();
    if (b->uploader.joinable()) b->uploader.join();
    if (b->worker.joinable()) b->worker.join();
    cudaStreamSynchronize(b->stream);
    {
        std::lock_guard<std::mutex> lk(b->mu);
        for (snp_system* s : b->owned) s->owner = nullptr;
        b->owned.clear();
    }
    b->tune.save(getenv("SNP_AUTOTUNE_CACHE"));
    cudaStreamSynchronize(b->stream2);
    cudaEventDestroy(b->ev0);
    cudaEventDestroy(b->ev1);
    cudaEventDestroy(b->ev_fork);
    cudaEventDestroy(b->ev_join);
    cudaStreamDestroy(b->stream2);
    cudaFree(b->d_sys);
    cudaFree(b->d_nsteps);
    cudaFree(b->d_res);
    cudaFree(b->d_work);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return SNP_OK;
}

int snp_batch_submit(snp_batch* b, snp_system* const* sys, const int64_t* steps, int32_t count, int64_t* ticket) {
    if (!b || !sys || !steps || count < 0) return fail(SNP_ERR_INVALID, "bad batch arguments");
    for (int32_t i = 0; i < count; ++i) {
        if (!sys[i]) return fail(SNP_ERR_INVALID, "NULL system in batch");
        if (steps[i] < 0) return fail(SNP_ERR_INVALID, "negative step count in batch");
        for (int32_t j = 0; j < i; ++j)
            if (sys[j] == sys[i]) return fail(SNP_ERR_INVALID, "system listed twice in one ticket");
        const size_t need = sys[i]->materialized ? sys[i]->device_bytes : sys[i]->planned_bytes;
        if (b->budget && need > b->budget) return fail(SNP_ERR_OOM, "a system is larger than the batch memory budget");
    }
    for (int32_t i = 0; i < count; ++i) {
        int expected = 0;
        if (!sys[i]->busy.compare_exchange_strong(expected, 1)) {
            for (int32_t j = 0; j < i; ++j) sys[j]->busy.store(0);
            return fail(SNP_ERR_BUSY, "system already owned by an unfinished batch");
        }
    }
    std::lock_guard<std::mutex> lk(b->mu);
    const int64_t id = b->next_id++;
    Ticket& t = b->tickets[id];
    t.outstanding = count;
    for (int32_t i = 0; i < count; ++i) {
        t.items.emplace_back(new Item());
        Item* it = t.items.back().get();
        it->ticket = id;
        it->sys = sys[i];
        it->remaining = steps[i];
        b->pending.push_back(it);
    }
    if (ticket) *ticket = id;
    b->cv.notify_all();
    return SNP_OK;
}

int snp_batch_poll(snp_batch* b, int64_t ticket, int* done) {
    if (!b || !done) return fail(SNP_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(b->mu);
    auto it = b->tickets.find(ticket);
    if (it == b->tickets.end()) return fail(SNP_ERR_INVALID, "unknown ticket");
    *done = it->second.complete();
    return SNP_OK;
}

int snp_batch_wait(snp_batch* b, int64_t ticket) {
    if (!b) return fail(SNP_ERR_INVALID, "NULL batch");
    std::unique_lock<std::mutex> lk(b->mu);
    auto it = b->tickets.find(ticket);
    if (it == b->tickets.end()) return fail(SNP_ERR_INVALID, "unknown ticket");
    b->cv.wait(lk, [&] { return it->second.complete() || stalled(b); });
    if (!it->second.complete())
        return fail(SNP_ERR_BUSY, "ticket " + std::to_string(ticket) +
                                      " waits for memory that only destroying finished systems can free");
    if (it->second.status) return fail(it->second.status, it->second.error);
    return SNP_OK;
}

int snp_batch_steps_done(snp_batch* b, int64_t ticket, int32_t index, int64_t* steps_done) {
    if (!b || !steps_done) return fail(SNP_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(b->mu);
    auto it = b->tickets.find(ticket);
    if (it == b->tickets.end()) return fail(SNP_ERR_INVALID, "unknown ticket");
    if (!it->second.complete()) return fail(SNP_ERR_BUSY, "ticket not finished");
    if (index < 0 || (size_t)index >= it->second.items.size()) return fail(SNP_ERR_INVALID, "bad index");
    *steps_done = it->second.items[index]->done;
    return SNP_OK;
}

int snp_batch_get_info(snp_batch* b, snp_batch_info* info) {
    if (!b || !info) return fail(SNP_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(b->mu);
    info->budget_bytes = b->budget;
    info->resident_bytes = b->resident_bytes;
    info->peak_resident_bytes = b->peak_bytes;
    info->rounds = b->rounds;
    info->admitted = b->admitted;
    info->finished = b->finished;
    info->waiting = (int64_t)b->pending.size();
    info->running = (int64_t)b->active.size();
    info->admit_seconds = b->t_admit;
    info->launch_seconds = b->t_launch;
    info->resident_seconds = b->t_resident;
    info->resident_device_seconds = b->t_resident_dev;
    info->large_tail_seconds = b->t_large_tail;
    info->idle_seconds = b->t_idle;
    info->round_seconds = b->t_round;
    return SNP_OK;
}

}  // extern "C"
