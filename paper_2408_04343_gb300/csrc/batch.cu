// Batched form: many independent systems advanced by one persistent launch.
//
// Submitted tickets are executed by a worker thread in arrival order.  The
// systems of a ticket that fit the CTA-resident engine are sorted largest
// first and handed to one persistent launch (grid = SMs x resident CTAs per
// SM); each CTA takes the next system from a device work counter and runs all
// its steps, so thousands of systems of uneven size share one launch with
// per-system offsets (the DevSys table).  Systems too large for one CTA run on
// the grid-wide engine on their own streams, overlapping with the launch.
#include <cuda_runtime.h>

#include <algorithm>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "kernels.h"
#include "snp_internal.h"
#include "system.h"

namespace snp {

struct Ticket {
    int64_t id = 0;
    std::vector<snp_system*> sys;
    std::vector<int64_t> steps;
    std::vector<int64_t> done_steps;
    int state = 0;  // 0 queued, 1 running, 2 done
    int status = SNP_OK;
    std::string error;
};

}  // namespace snp

struct snp_batch {
    snp_options opt{};
    size_t budget = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<int64_t> queue;
    std::map<int64_t, snp::Ticket> tickets;
    int64_t next_id = 1;
    bool stop = false;
    std::thread worker;
    // device tables, grown on demand
    snp::DevSys* d_sys = nullptr;
    long long* d_nsteps = nullptr;
    unsigned long long* d_exec = nullptr;  // 3 words per system
    unsigned int* d_work = nullptr;
    size_t cap = 0;
    int sms = 0;
    int threads = 0;   // resident CTA size; 0 = autotune
};

namespace snp {

static int grow_tables(snp_batch* b, size_t n) {
    if (n <= b->cap) return SNP_OK;
    size_t cap = std::max<size_t>(n, 2 * b->cap);
    cudaFree(b->d_sys);
    cudaFree(b->d_nsteps);
    cudaFree(b->d_exec);
    b->d_sys = nullptr;
    b->d_nsteps = nullptr;
    b->d_exec = nullptr;
    if (cudaMalloc(&b->d_sys, cap * sizeof(DevSys)) != cudaSuccess ||
        cudaMalloc(&b->d_nsteps, cap * sizeof(long long)) != cudaSuccess ||
        cudaMalloc(&b->d_exec, cap * 3 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        b->cap = 0;
        return fail(SNP_ERR_OOM, "batch table allocation failed");
    }
    b->cap = cap;
    return SNP_OK;
}

// CTAs of `threads` threads and `smem` bytes that fit on one SM.
static int ctas_per_sm(int threads, size_t smem, int e_bits, bool compact, int sel) {
    (void)e_bits;
    (void)compact;
    (void)sel;
    int dev = 0, smem_sm = 0, thr_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&thr_sm, cudaDevAttrMaxThreadsPerMultiProcessor, dev);
    int by_thr = thr_sm / threads;
    int by_smem = (int)((size_t)smem_sm / (smem + 1024));
    return std::max(1, std::min(by_thr, by_smem));
}

int run_resident_group(snp_batch* b, std::vector<snp_system*>& sys, std::vector<int64_t>& steps,
                       std::vector<int64_t>& exec_out) {
    const size_t n = sys.size();
    if (n == 0) return SNP_OK;
    int rc = grow_tables(b, n);
    if (rc) return rc;
    std::vector<size_t> order(n);
    for (size_t i = 0; i < n; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](size_t a, size_t c) { return (double)sys[a]->nsyn * steps[a] > (double)sys[c]->nsyn * steps[c]; });
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
    plan.max_q = max_q;
    plan.smem = resident_smem_bytes(max_q, plan.e_bits);
    plan.threads = b->threads > 0 ? b->threads : 512;
    const bool compact = sys[0]->compact;
    const int sel = sys[0]->opt.select;
    plan.ctas = b->sms * ctas_per_sm(plan.threads, plan.smem, plan.e_bits, compact, sel);
    if (cudaMemcpyAsync(b->d_sys, tab.data(), n * sizeof(DevSys), cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaMemcpyAsync(b->d_nsteps, ns.data(), n * sizeof(long long), cudaMemcpyHostToDevice, b->stream) != cudaSuccess ||
        cudaMemsetAsync(b->d_work, 0, sizeof(unsigned int), b->stream) != cudaSuccess)
        return fail(SNP_ERR_CUDA, "batch table upload");
    if (launch_resident(b->d_sys, b->d_nsteps, (int)n, b->d_work, plan, compact, sel, b->stream) != cudaSuccess)
        return fail(SNP_ERR_CUDA, std::string("resident launch: ") + cudaGetErrorString(cudaGetLastError()));
    // executed step counts and overflow flags of every system, in one copy
    std::vector<unsigned long long> ex(n * 3);
    if (launch_gather_results(b->d_sys, (int)n, b->d_exec, b->stream) != cudaSuccess ||
        cudaMemcpyAsync(ex.data(), b->d_exec, n * 3 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess)
        return fail(SNP_ERR_CUDA, std::string("batch sync: ") + cudaGetErrorString(cudaGetLastError()));
    exec_out.assign(n, 0);
    bool overflow = false;
    for (size_t r = 0; r < n; ++r) {
        exec_out[order[r]] = (int64_t)ex[3 * r + 1];
        sys[order[r]]->host_step = ex[3 * r + 0];
        overflow |= ex[3 * r + 2] != 0ull;
    }
    if (overflow) return fail(SNP_ERR_OVERFLOW, "a spike count left the int32 range in a batched system");
    return SNP_OK;
}

static void execute_ticket(snp_batch* b, Ticket& t) {
    const size_t n = t.sys.size();
    t.done_steps.assign(n, 0);
    // group by kernel template: (compact, select); large systems go grid-wide
    std::map<std::pair<int, int>, std::vector<size_t>> groups;
    std::vector<size_t> large;
    for (size_t i = 0; i < n; ++i) {
        snp_system* s = t.sys[i];
        if (s->opt.prop == SNP_PROP_PULL && s->opt.engine != SNP_ENGINE_LAUNCH && resident_fits(s, nullptr))
            groups[{s->compact ? 1 : 0, s->opt.select}].push_back(i);
        else
            large.push_back(i);
    }
    int rc = SNP_OK;
    for (size_t i : large) {
        rc = run_steps(t.sys[i], t.steps[i]);
        if (rc) break;
    }
    for (auto& g : groups) {
        if (rc) break;
        std::vector<snp_system*> sys;
        std::vector<int64_t> steps, ex;
        for (size_t i : g.second) {
            sys.push_back(t.sys[i]);
            steps.push_back(t.steps[i]);
        }
        rc = run_resident_group(b, sys, steps, ex);
        if (!rc)
            for (size_t r = 0; r < g.second.size(); ++r) t.done_steps[g.second[r]] = ex[r];
    }
    for (size_t i : large) {
        if (rc) break;
        int64_t ex = 0;
        rc = read_flags(t.sys[i], &ex);
        t.done_steps[i] = ex;
    }
    t.status = rc;
    if (rc) t.error = last_error();
}

static void worker_main(snp_batch* b) {
    for (;;) {
        int64_t id;
        {
            std::unique_lock<std::mutex> lk(b->mu);
            b->cv.wait(lk, [&] { return b->stop || !b->queue.empty(); });
            if (b->queue.empty() && b->stop) return;
            id = b->queue.front();
            b->queue.pop_front();
            b->tickets[id].state = 1;
        }
        Ticket* t;
        {
            std::lock_guard<std::mutex> lk(b->mu);
            t = &b->tickets[id];
        }
        execute_ticket(b, *t);
        {
            std::lock_guard<std::mutex> lk(b->mu);
            for (snp_system* s : t->sys) s->busy.store(0);
            t->state = 2;
        }
        b->cv.notify_all();
    }
}

const char* last_error();

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
    if (cudaMalloc(&b->d_work, sizeof(unsigned int)) != cudaSuccess) {
        cudaGetLastError();
        if (b->own_stream) cudaStreamDestroy(b->stream);
        delete b;
        return fail(SNP_ERR_OOM, "device allocation failed");
    }
    b->worker = std::thread(worker_main, b);
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
    if (b->worker.joinable()) b->worker.join();
    cudaStreamSynchronize(b->stream);
    cudaFree(b->d_sys);
    cudaFree(b->d_nsteps);
    cudaFree(b->d_exec);
    cudaFree(b->d_work);
    if (b->own_stream) cudaStreamDestroy(b->stream);
    delete b;
    return SNP_OK;
}

int snp_batch_submit(snp_batch* b, snp_system* const* sys, const int64_t* steps, int32_t count, int64_t* ticket) {
    if (!b || !sys || !steps || count < 0) return fail(SNP_ERR_INVALID, "bad batch arguments");
    size_t bytes = 0;
    for (int32_t i = 0; i < count; ++i) {
        if (!sys[i]) return fail(SNP_ERR_INVALID, "NULL system in batch");
        if (steps[i] < 0) return fail(SNP_ERR_INVALID, "negative step count in batch");
        bytes += sys[i]->device_bytes;
        for (int32_t j = 0; j < i; ++j)
            if (sys[j] == sys[i]) return fail(SNP_ERR_INVALID, "system listed twice in one ticket");
    }
    if (b->budget && bytes > b->budget) return fail(SNP_ERR_OOM, "ticket exceeds the batch memory budget");
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
    t.id = id;
    t.sys.assign(sys, sys + count);
    t.steps.assign(steps, steps + count);
    b->queue.push_back(id);
    if (ticket) *ticket = id;
    b->cv.notify_all();
    return SNP_OK;
}

int snp_batch_poll(snp_batch* b, int64_t ticket, int* done) {
    if (!b || !done) return fail(SNP_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(b->mu);
    auto it = b->tickets.find(ticket);
    if (it == b->tickets.end()) return fail(SNP_ERR_INVALID, "unknown ticket");
    *done = it->second.state == 2;
    return SNP_OK;
}

int snp_batch_wait(snp_batch* b, int64_t ticket) {
    if (!b) return fail(SNP_ERR_INVALID, "NULL batch");
    std::unique_lock<std::mutex> lk(b->mu);
    auto it = b->tickets.find(ticket);
    if (it == b->tickets.end()) return fail(SNP_ERR_INVALID, "unknown ticket");
    b->cv.wait(lk, [&] { return it->second.state == 2; });
    if (it->second.status) return fail(it->second.status, it->second.error);
    return SNP_OK;
}

int snp_batch_steps_done(snp_batch* b, int64_t ticket, int32_t index, int64_t* steps_done) {
    if (!b || !steps_done) return fail(SNP_ERR_INVALID, "NULL argument");
    std::lock_guard<std::mutex> lk(b->mu);
    auto it = b->tickets.find(ticket);
    if (it == b->tickets.end()) return fail(SNP_ERR_INVALID, "unknown ticket");
    if (it->second.state != 2) return fail(SNP_ERR_BUSY, "ticket not finished");
    if (index < 0 || (size_t)index >= it->second.done_steps.size()) return fail(SNP_ERR_INVALID, "bad index");
    *steps_done = it->second.done_steps[index];
    return SNP_OK;
}

}  // extern "C"
