// C-ABI of libsnp: system life cycle, stepping, state access.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <atomic>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "kernels.h"
#include "snp_internal.h"
#include "system.h"

namespace snp {

const char* last_error();

// ---- device memory -----------------------------------------------------

void* sys_alloc(snp_system* s, size_t bytes) {
    if (bytes == 0) bytes = 16;
    bytes = (bytes + 255) & ~(size_t)255;
    void* p = nullptr;
    if (s->alloc.alloc) {
        p = s->alloc.alloc(s->alloc.ctx, bytes, (void*)s->stream);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
    }
    if (p) {
        s->allocs.push_back({p, bytes});
        s->device_bytes += bytes;
    }
    return p;
}

static void sys_free_all(snp_system* s) {
    for (auto& a : s->allocs) {
        if (s->alloc.release)
            s->alloc.release(s->alloc.ctx, a.first, a.second, (void*)s->stream);
        else
            cudaFree(a.first);
    }
    s->allocs.clear();
    s->device_bytes = 0;
}

// Short-lived device buffers of one call (staging of host arrays): from the
// caller's allocator when the system has one, else stream-ordered cudaMalloc.
static void* stage_alloc(snp_system* s, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (s->alloc.alloc) return s->alloc.alloc(s->alloc.ctx, bytes, (void*)s->stream);
    void* p = nullptr;
    if (cudaMallocAsync(&p, bytes, s->stream) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

static void stage_free(snp_system* s, void* p, size_t bytes) {
    if (!p) return;
    bytes = (bytes + 255) & ~(size_t)255;
    if (s->alloc.release)
        s->alloc.release(s->alloc.ctx, p, bytes, (void*)s->stream);
    else
        cudaFreeAsync(p, s->stream);
}

static int cuda_fail(const char* what) {
    cudaError_t e = cudaGetLastError();
    return fail(SNP_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

// ---- one allocation per system ---------------------------------------------
// Every device buffer of a system is carved from one allocation: the host
// image is turned into a list of pieces (destination pointer field, source or
// fill byte, size), the sizes are summed at 256-byte alignment, one block is
// allocated, and each piece is copied or filled into its place.

size_t plan_bytes(const std::vector<Piece>& plan) {
    size_t t = 0;
    for (const Piece& p : plan) t += (p.bytes + 255) & ~(size_t)255;
    return t;
}

void build_plan(snp_system* s, std::vector<Piece>& plan) {
    HostImage& im = *s->img;
    HostPack& hp = im.hp;
    DevSys& d = s->dev;
    const size_t q = (size_t)hp.q;
    const int32_t nslices = (hp.q + kSlice - 1) / kSlice;
    auto vec = [&](void* field, const auto& v) {
        plan.push_back({reinterpret_cast<void**>(field), v.data(), v.size() * sizeof(v[0]), -1});
    };
    auto fill = [&](void* field, size_t bytes, int byte) {
        plan.push_back({reinterpret_cast<void**>(field), nullptr, bytes, byte});
    };
    d.q = hp.q;
    d.nslices = nslices;
    vec(&d.slice_ptr, hp.slice_ptr);
    if (s->has_in_lists) vec(&d.in_idx, hp.in_idx);
    if (s->opt.form == SNP_FORM_OPT && s->opt.prop == SNP_PROP_PUSH) {
        vec(&d.out_ptr, hp.out_ptr);
        vec(&d.out_idx, hp.out_idx);
    }
    vec(&d.rule_off, hp.rule_off);
    vec(&d.rules, hp.rules);
    d.rec = nullptr;
    if ((s->opt.form == SNP_FORM_OPT || s->unions) && !hp.rec.empty()) vec(&d.rec, hp.rec);
    vec(&d.orig, hp.perm);
    vec(&s->d_rule_base, hp.rule_base);
    vec(&d.C, hp.C0);
    fill(&d.st, q * 4, 0);
    for (int b = 0; b < 2; ++b) {
        if (s->opt.form == SNP_FORM_OPT) fill(&d.E[b], (q + 1) * 4, 0);
        fill(&d.S[b], q * 4, 0xff);  // -1: no rule selected yet
    }
    fill(&d.flags, kNumFlags * 4, 0);
    fill(&d.step, kNumStepWords * 8, 0);
    fill(&s->scratch, q * 4, 0);
    fill(&s->d_nsteps, 8, 0);
    fill(&s->d_work, 4, 0);
    fill(&s->d_self, sizeof(DevSys), 0);
    if (s->opt.form != SNP_FORM_OPT) {
        EllSys& e = s->ell;
        e.m = hp.m;
        if (!im.ep.in_ptr.empty()) {
            vec(&e.in_ptr, im.ep.in_ptr);
            vec(&e.in_ent, im.ep.in_ent);
        }
        if (!im.ep.out_ptr.empty()) {
            vec(&e.out_ptr, im.ep.out_ptr);
            vec(&e.out_ent, im.ep.out_ent);
        }
        if (s->opt.form == SNP_FORM_DENSE) {
            vec(&e.dense, im.dense);
            fill(&e.inflow, q * 4, 0);
        }
        for (int b = 0; b < 2; ++b) fill(&e.Em[b], (size_t)hp.m + 1, 0);
    }
    if (s->has_tiled) {
        TiledSys& tl = s->tiled;
        const TiledPack& tp = im.tp;
        tl.P = tp.P;
        tl.part_words = tp.part_words;
        tl.e_bits = tp.e_bits;
        tl.G = tp.G;
        tl.acc_words = tp.acc_words;
        tl.rin_words = tp.rin_words;
        tl.acc8 = tp.acc8;
        tl.rin_esm = tp.rin_esm;
        tl.src_bits = tp.src_bits;
        tl.pairs = tp.pairs;
        tl.rle = tp.rle;
        tl.tstart = nullptr;
        if (tp.rle) vec(&tl.tstart, tp.tstart);
        tl.ent_words = (int64_t)tp.ent.size();
        vec(&tl.sub, tp.sub);
        vec(&tl.ent, tp.ent);
        vec(&tl.cta_lo, tp.cta_lo);
        tl.inflow = nullptr;  // the fused step sums the partitions' in-flows in distributed shared memory
        if (tp.P > kTiledMaxCluster) fill(&tl.inflow, (size_t)tp.P * nslices * kSlice * 4, 0);
        for (int b = 0; b < 2; ++b) fill(&tl.Eg[b], (size_t)tp.P * tp.part_words * 4, 0);
    }
}

int materialize(snp_system* s) {
    if (s->materialized) return SNP_OK;
    if (!s->img) return fail(SNP_ERR_INVALID, "system has no host image");
    std::vector<Piece> plan;
    build_plan(s, plan);
    const size_t total = plan_bytes(plan);
    char* base = (char*)sys_alloc(s, total);
    if (!base) return fail(SNP_ERR_OOM, "device allocation of " + std::to_string(total) + " bytes failed");
    size_t off = 0;
    for (const Piece& p : plan) {
        *p.dst = base + off;
        cudaError_t e = cudaSuccess;
        if (p.src && p.bytes)
            e = cudaMemcpyAsync(base + off, p.src, p.bytes, cudaMemcpyHostToDevice, s->stream);
        else if (p.fill >= 0 && p.bytes)
            e = cudaMemsetAsync(base + off, p.fill, p.bytes, s->stream);
        if (e != cudaSuccess) return cuda_fail("upload");
        off += (p.bytes + 255) & ~(size_t)255;
    }
    DevSys& d = s->dev;
    d.rules_per_neuron = s->uniform_rules;
    d.identity = s->identity ? 1 : 0;
    d.seed = s->opt.seed;
    philox_round_keys(d.seed, d.philox_rk);
    d.select = s->opt.select;
    d.max_p = s->max_p;
    if (cudaMemcpyAsync(s->d_self, &d, sizeof(DevSys), cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
        return cuda_fail("descriptor upload");
    if (cudaStreamSynchronize(s->stream) != cudaSuccess) return cuda_fail("upload sync");
    s->img.reset();
    s->materialized = true;
    return SNP_OK;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ---- chunk graphs of the grid-wide engines ------------------------------

// One pull launch of the system's grid-wide engine (L2-gather or tiled).
static cudaError_t launch_pull_any(snp_system* s, int kind, int32_t t, cudaStream_t st) {
    if (effective_engine(s) == SNP_ENGINE_TILED)
        return launch_tiled(s->dev, s->tiled, kind, t, st, s->compact, s->opt.select, s->tiled_smem,
                            s->tiled_threads);
    return launch_pull(s->dev, kind, t, st, s->compact, s->opt.select);
}

static int build_chunk_graph(snp_system* s) {
    if (s->chunk_exec) return SNP_OK;
    if (!s->cap_stream && cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
        return cuda_fail("stream create");
    cudaGraph_t g = nullptr;
    if (cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return cuda_fail("begin capture");
    const bool compact = s->compact;
    const int sel = s->opt.select;
    for (int t = 0; t < kChunk; ++t) {
        if (s->opt.prop == SNP_PROP_PUSH)
            launch_push_step(s->dev, t, s->cap_stream, compact, sel);
        else
            launch_pull_any(s, kPullFused, t, s->cap_stream);
    }
    launch_advance(s->dev, kChunk, s->cap_stream);
    if (cudaStreamEndCapture(s->cap_stream, &g) != cudaSuccess) return cuda_fail("end capture");
    cudaError_t e = cudaGraphInstantiate(&s->chunk_exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        s->chunk_exec = nullptr;
        return cuda_fail("graph instantiate");
    }
    return SNP_OK;
}

static int step_launch_engine(snp_system* s, int64_t n) {
    const bool compact = s->compact;
    const int sel = s->opt.select;
    cudaStream_t st = s->stream;
    if (launch_begin(s->dev, st) != cudaSuccess) return cuda_fail("begin");
    if (s->opt.prop == SNP_PROP_PUSH) {
        int64_t left = n;
        if (left >= kChunk) {
            int rc = build_chunk_graph(s);
            if (rc) return rc;
        }
        while (left >= kChunk) {
            if (cudaGraphLaunch(s->chunk_exec, st) != cudaSuccess) return cuda_fail("graph launch");
            left -= kChunk;
        }
        for (int64_t t = 0; t < left; ++t)
            if (launch_push_step(s->dev, (int32_t)t, st, compact, sel) != cudaSuccess) return cuda_fail("push step");
        if (launch_finish(s->dev, (int32_t)left, st) != cudaSuccess) return cuda_fail("finish");
        return SNP_OK;
    }
    if (launch_pull_any(s, kPullSelectOnly, 0, st) != cudaSuccess) return cuda_fail("select");
    int64_t rem = n - 1;
    if (rem >= kChunk) {
        int rc = build_chunk_graph(s);
        if (rc) return rc;
    }
    while (rem >= kChunk) {
        if (cudaGraphLaunch(s->chunk_exec, st) != cudaSuccess) return cuda_fail("graph launch");
        rem -= kChunk;
    }
    for (int64_t t = 0; t < rem; ++t)
        if (launch_pull_any(s, kPullFused, (int32_t)t, st) != cudaSuccess) return cuda_fail("step");
    if (launch_pull_any(s, kPullGatherOnly, (int32_t)rem, st) != cudaSuccess) return cuda_fail("gather");
    if (launch_finish(s->dev, (int32_t)(rem + 1), st) != cudaSuccess) return cuda_fail("finish");
    return SNP_OK;
}

bool resident_fits(const snp_system* s, ResidentPlan* plan) {
    if (!s->has_in_lists) return false;
    const int eb = resident_e_bits(s->max_p);
    const size_t smem = resident_smem_bytes(s->q, eb);
    if ((long long)smem + 1024 > (long long)resident_max_smem()) return false;
    if (plan) {
        plan->e_bits = eb;
        plan->max_q = s->q;
        plan->smem = smem;
        plan->threads = s->opt.threads > 0 ? s->opt.threads : 1024;
        plan->ctas = 1;
        plan->big = plan->threads == 1024;  // one CTA per system: the 64-register instance
    }
    return true;
}

static int step_resident(snp_system* s, int64_t n) {
    ResidentPlan plan;
    if (!resident_fits(s, &plan))
        return fail(SNP_ERR_UNSUPPORTED, "system too large for the resident engine (shared memory)");
    if (cudaMemcpyAsync(s->d_nsteps, &n, sizeof(long long), cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
        return cuda_fail("nsteps upload");
    if (cudaMemsetAsync(s->d_work, 0, sizeof(unsigned int), s->stream) != cudaSuccess) return cuda_fail("work reset");
    if (launch_resident(s->d_self, s->d_nsteps, 1, s->d_work, plan, s->compact, s->opt.select, s->stream) != cudaSuccess)
        return cuda_fail("resident launch");
    return SNP_OK;
}

int effective_engine(const snp_system* s) {
    if (s->opt.form != SNP_FORM_OPT) return SNP_ENGINE_LAUNCH;
    if (s->opt.prop == SNP_PROP_PUSH) return SNP_ENGINE_LAUNCH;
    if (s->opt.engine == SNP_ENGINE_RESIDENT) return SNP_ENGINE_RESIDENT;
    if (s->opt.engine == SNP_ENGINE_LAUNCH) return SNP_ENGINE_LAUNCH;
    if (s->opt.engine == SNP_ENGINE_TILED) return SNP_ENGINE_TILED;
    if (s->q <= kAutoResidentMaxQ && s->m <= kAutoResidentMaxRules && resident_fits(s, nullptr))
        return SNP_ENGINE_RESIDENT;
    return s->has_tiled ? SNP_ENGINE_TILED : SNP_ENGINE_LAUNCH;
}

// Which layouts a system needs, from its options and size (before packing).
static void plan_layouts(const snp_options& o, int32_t q, int64_t m, bool* want_tiled, bool* want_in_lists) {
    if (o.form != SNP_FORM_OPT) {
        *want_tiled = *want_in_lists = false;
        return;
    }
    *want_tiled = o.prop == SNP_PROP_PULL &&
                  (o.engine == SNP_ENGINE_TILED ||
                   (o.engine == SNP_ENGINE_AUTO && (q > kAutoResidentMaxQ || m > kAutoResidentMaxRules)));
    // sliced ELL in-lists: the L2-gather and resident engines and the batch
    *want_in_lists = o.engine != SNP_ENGINE_TILED;
}

// ELL form (pull or push) and dense form: plain launches per step.
static int step_ell_forms(snp_system* s, int64_t n) {
    const bool compact = s->compact;
    const int sel = s->opt.select;
    cudaStream_t st = s->stream;
    const EllSys& e = s->ell;
    if (launch_begin(s->dev, st) != cudaSuccess) return cuda_fail("begin");
    if (s->opt.form == SNP_FORM_ELL && s->opt.prop == SNP_PROP_PULL) {
        if (launch_ell_pull(s->dev, e, kPullSelectOnly, 0, st, compact, sel) != cudaSuccess) return cuda_fail("select");
        for (int64_t t = 0; t + 1 < n; ++t)
            if (launch_ell_pull(s->dev, e, kPullFused, (int32_t)t, st, compact, sel) != cudaSuccess)
                return cuda_fail("ell step");
        if (launch_ell_pull(s->dev, e, kPullGatherOnly, (int32_t)(n - 1), st, compact, sel) != cudaSuccess)
            return cuda_fail("ell gather");
    } else if (s->opt.form == SNP_FORM_ELL) {
        for (int64_t t = 0; t < n; ++t) {
            if (launch_ell_select(s->dev, e, false, true, (int32_t)t, st, compact, sel) != cudaSuccess ||
                launch_ell_push(s->dev, e, (int32_t)t, st) != cudaSuccess)
                return cuda_fail("ell push step");
        }
    } else {
        if (launch_ell_select(s->dev, e, false, true, 0, st, compact, sel) != cudaSuccess) return cuda_fail("select");
        for (int64_t t = 0; t < n; ++t) {
            if (launch_dense_accum(s->dev, e, (int32_t)t, st) != cudaSuccess ||
                launch_ell_select(s->dev, e, true, t + 1 < n, (int32_t)(t + 1), st, compact, sel) != cudaSuccess)
                return cuda_fail("dense step");
        }
    }
    if (launch_finish(s->dev, (int32_t)n, st) != cudaSuccess) return cuda_fail("finish");
    return SNP_OK;
}

int read_flags(snp_system* s, int64_t* exec) {
    uint32_t fl[kNumFlags];
    unsigned long long steps[kNumStepWords];
    if (cudaMemcpyAsync(fl, s->dev.flags, sizeof(fl), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaMemcpyAsync(steps, s->dev.step, sizeof(steps), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return cuda_fail("flag read");
    if (exec) *exec = (int64_t)steps[kStepExec];
    s->host_step = steps[kStepBase];
    if (fl[kFlagOverflow]) {
        const uint32_t zero = 0;
        cudaMemcpyAsync(s->dev.flags + kFlagOverflow, &zero, sizeof(zero), cudaMemcpyHostToDevice, s->stream);
        cudaStreamSynchronize(s->stream);
        return fail(SNP_ERR_OVERFLOW, "a spike count left the int32 range");
    }
    if (fl[kFlagBounds]) {
        char msg[96];
        snprintf(msg, sizeof(msg), "bounds check: an index out of range (sites 0x%x)", fl[kFlagBounds]);
        const uint32_t zero = 0;
        cudaMemcpyAsync(s->dev.flags + kFlagBounds, &zero, sizeof(zero), cudaMemcpyHostToDevice, s->stream);
        cudaStreamSynchronize(s->stream);
        return fail(SNP_ERR_INVALID, msg);
    }
    if (fl[kFlagTimeout]) return fail(SNP_ERR_TIMEOUT, "a bounded device wait gave up");
    if (fl[kFlagChoice]) {
        const uint32_t zero = 0;
        cudaMemcpyAsync(s->dev.flags + kFlagChoice, &zero, sizeof(zero), cudaMemcpyHostToDevice, s->stream);
        cudaStreamSynchronize(s->stream);
        return fail(SNP_ERR_INVALID, "a forced choice index was out of range for its neuron");
    }
    return SNP_OK;
}

int run_steps(snp_system* s, int64_t n) {
    if (n <= 0) return SNP_OK;
    if (s->opt.form != SNP_FORM_OPT) return step_ell_forms(s, n);
    const int eng = effective_engine(s);
    if ((eng == SNP_ENGINE_LAUNCH || eng == SNP_ENGINE_RESIDENT) && s->opt.prop == SNP_PROP_PULL && !s->has_in_lists)
        return fail(SNP_ERR_UNSUPPORTED, "system was created for the tiled engine only");
    return eng == SNP_ENGINE_RESIDENT ? step_resident(s, n) : step_launch_engine(s, n);
}

// The launches of a pull call of n steps on a grid-wide engine, as
// step_launch_engine issues them but without its chunk graph (so without
// the base step's advances, which only bound the step index of the chunk
// graph's launches): begin, the first select, n - 1 fused steps, the last
// gather, finish.  Every parameter is a constant of the call, so the
// sequence can be captured once and replayed.
static cudaError_t enqueue_pull_call(snp_system* s, int64_t n, cudaStream_t st) {
    cudaError_t e = launch_begin(s->dev, st);
    if (e == cudaSuccess) e = launch_pull_any(s, kPullSelectOnly, 0, st);
    for (int64_t t = 0; t < n - 1 && e == cudaSuccess; ++t) e = launch_pull_any(s, kPullFused, (int32_t)t, st);
    if (e == cudaSuccess) e = launch_pull_any(s, kPullGatherOnly, (int32_t)(n - 1), st);
    if (e == cudaSuccess) e = launch_finish(s->dev, (int32_t)n, st);
    return e;
}

int run_steps_graphed(snp_system* s, int64_t n) {
    const int eng = s->opt.form == SNP_FORM_OPT ? effective_engine(s) : SNP_ENGINE_LAUNCH;
    if (n < 2 || n > kMaxGraphedCall || s->opt.form != SNP_FORM_OPT || s->opt.prop != SNP_PROP_PULL ||
        eng == SNP_ENGINE_RESIDENT || (eng == SNP_ENGINE_LAUNCH && !s->has_in_lists))
        return run_steps(s, n);
    if (!s->call_exec || s->call_n != n) {
        if (s->call_exec) cudaGraphExecDestroy(s->call_exec);
        s->call_exec = nullptr;
        if (!s->cap_stream && cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking) != cudaSuccess)
            return cuda_fail("stream create");
        cudaGraph_t g = nullptr;
        if (cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
            return cuda_fail("begin capture");
        const cudaError_t le = enqueue_pull_call(s, n, s->cap_stream);
        if (cudaStreamEndCapture(s->cap_stream, &g) != cudaSuccess || le != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return cuda_fail("call capture");
        }
        const cudaError_t e = cudaGraphInstantiate(&s->call_exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            s->call_exec = nullptr;
            return cuda_fail("graph instantiate");
        }
        s->call_n = n;
    }
    if (cudaGraphLaunch(s->call_exec, s->stream) != cudaSuccess) return cuda_fail("graph launch");
    return SNP_OK;
}

}  // namespace snp

using namespace snp;

extern "C" {

const char* snp_strerror(int st) {
    switch (st) {
        case SNP_OK: return "ok";
        case SNP_ERR_INVALID: return "invalid argument or malformed system";
        case SNP_ERR_OOM: return "out of memory";
        case SNP_ERR_CUDA: return "CUDA runtime error";
        case SNP_ERR_TIMEOUT: return "bounded device wait timed out";
        case SNP_ERR_OVERFLOW: return "spike count overflowed int32";
        case SNP_ERR_BUSY: return "system is owned by an unfinished batch";
        case SNP_ERR_UNSUPPORTED: return "unsupported option combination";
        default: return "unknown status";
    }
}

const char* snp_last_error(void) { return snp::last_error(); }

int snp_create(const snp_desc* desc, const snp_options* opts, snp_system** out) {
    if (!out) return fail(SNP_ERR_INVALID, "out is NULL");
    *out = nullptr;
    int st = validate_desc(desc);
    if (st) return st;
    snp_options o;
    std::memset(&o, 0, sizeof(o));
    if (opts) o = *opts;
    if (o.form != SNP_FORM_OPT && o.form != SNP_FORM_ELL && o.form != SNP_FORM_DENSE)
        return fail(SNP_ERR_INVALID, "bad form");
    if (o.prop != SNP_PROP_PULL && o.prop != SNP_PROP_PUSH) return fail(SNP_ERR_INVALID, "bad prop");
    if (o.select != SNP_SELECT_FIRST && o.select != SNP_SELECT_PHILOX) return fail(SNP_ERR_INVALID, "bad select");
    if (o.engine < SNP_ENGINE_AUTO || o.engine > SNP_ENGINE_TILED) return fail(SNP_ERR_INVALID, "bad engine");
    if (o.prop == SNP_PROP_PUSH && (o.engine == SNP_ENGINE_RESIDENT || o.engine == SNP_ENGINE_TILED))
        return fail(SNP_ERR_UNSUPPORTED, "the resident and tiled engines are pull-only");
    if (o.form != SNP_FORM_OPT && o.engine != SNP_ENGINE_AUTO && o.engine != SNP_ENGINE_LAUNCH)
        return fail(SNP_ERR_UNSUPPORTED, "the ELL and dense forms run on the launch engine");
    if (o.form == SNP_FORM_DENSE && o.prop != SNP_PROP_PULL)
        return fail(SNP_ERR_UNSUPPORTED, "the dense form walks matrix columns (pull) only");

    snp_system* s = new (std::nothrow) snp_system();
    if (!s) return fail(SNP_ERR_OOM, "host allocation failed");
    s->opt = o;
    s->stream = (cudaStream_t)o.stream;
    if (o.alloc) s->alloc = *o.alloc;
    s->img.reset(new (std::nothrow) HostImage());
    if (!s->img) {
        delete s;
        return fail(SNP_ERR_OOM, "host allocation failed");
    }
    HostImage& im = *s->img;
    HostPack& hp = im.hp;
    bool want_tiled = false, want_in = false;
    plan_layouts(o, desc->q, desc->rule_offsets[desc->q], &want_tiled, &want_in);
    int dev = 0, sms = 0, optin = 0;
    if (want_tiled) {
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
            delete s;
            return cuda_fail("device query");
        }
    }
    // The tiled layout needs no in-degree order; without it slots are the
    // caller's neurons, and the select reads no slot-to-neuron map.  Under
    // AUTO the caller's order is kept as well when the system is too large
    // for one CTA (so no resident in-lists): if no tiled layout fits after
    // all, the system is packed again in the in-degree order that the
    // L2-gather engine's in-lists want.
    const bool auto_large = o.engine == SNP_ENGINE_AUTO && want_tiled &&
                            resident_smem_bytes(desc->q, 2) + 1024 > (size_t)optin;
    int window = (o.form == SNP_FORM_OPT && (o.engine == SNP_ENGINE_TILED || auto_large)) ? 0 : kSortWindow;
    st = pack_system(desc, o.form == SNP_FORM_OPT && o.prop == SNP_PROP_PUSH, false, window, &hp);
    if (!st && o.form == SNP_FORM_ELL) st = pack_ell(desc, hp, o.prop == SNP_PROP_PULL, o.prop == SNP_PROP_PUSH, &im.ep);
    if (!st && o.form == SNP_FORM_DENSE) st = pack_dense(desc, hp, &im.dense);
    if (st) {
        delete s;
        return st;
    }
    // union expressions step through the compiled records when every neuron
    // fits one, else through union records in the general rule table
    s->unions = desc->rule_term_offsets != nullptr;

    if (want_tiled) {
        // the gather sums a partition's in-flow in 32-bit shared accumulators,
        // read back as int32: a target must not be able to receive more than
        // INT32_MAX spikes from one partition in one step (the int64 sums of
        // the other engines carry any in-flow to the overflow check)
        if ((int64_t)hp.max_in * (int64_t)hp.max_p > (int64_t)INT32_MAX)
            st = fail(SNP_ERR_UNSUPPORTED, "in-degree x p can exceed the tiled engine's 32-bit accumulators");
        else {
            // clusters of P CTAs with about the largest shared memory per CTA
            int cpw[kTiledMaxCluster + 1] = {0};
            for (int P = 1; P <= kTiledMaxCluster; ++P) cpw[P] = tiled_clusters_per_wave(P, (size_t)optin - 2048);
            st = pack_tiled(desc, hp, sms, (size_t)optin - 2048, &im.tp, cpw);
        }
        // Under AUTO the tiled engine must pay for itself: every CTA copies a
        // whole emission partition into shared memory each step.  With one
        // wave of CTAs that copy overlaps the entry stream; with several
        // waves (large, low-degree systems with 32-bit accumulators: many
        // partitions) it can move more bytes than the gathers it replaces.
        // Keep it when it is one wave or the copies stay under half the
        // entry stream.
        if (st == SNP_OK && o.engine == SNP_ENGINE_AUTO && im.tp.G > sms &&
            (double)im.tp.G * im.tp.part_words * 4.0 > 0.5 * 4.0 * (double)im.tp.ent.size()) {
            im.tp = TiledPack();
            st = SNP_ERR_UNSUPPORTED;
        }
        if (st == SNP_OK) {
            s->has_tiled = true;
            // the resident engine (batches) still needs in-lists when the system fits one CTA
            if (o.engine == SNP_ENGINE_AUTO)
                want_in = resident_smem_bytes(hp.q, resident_e_bits(hp.max_p)) + 1024 <= (size_t)optin;
        } else if (o.engine == SNP_ENGINE_TILED) {
            delete s;
            return st;
        } else {
            want_in = true;  // AUTO falls back to the L2-gather engine
            if (window != kSortWindow) {
                hp = HostPack();
                window = kSortWindow;
                st = pack_system(desc, false, false, window, &hp);
                if (st) {
                    delete s;
                    return st;
                }
            }
        }
    }
    if (want_in) pack_in_lists(desc, &hp);
    s->has_in_lists = want_in;
    s->q = hp.q;
    s->m = hp.m;
    s->nsyn = hp.nsyn;
    s->max_p = hp.max_p;
    s->max_rules = hp.max_rules;
    s->uniform_rules = hp.uniform_rules;
    s->identity = hp.identity;
    s->compact = hp.compact;
    s->compiled = (s->opt.form == SNP_FORM_OPT || s->unions) && !hp.rec.empty();
    s->in_entries = (int64_t)hp.in_idx.size();
    s->out_entries = (int64_t)hp.out_idx.size();
    if (o.form == SNP_FORM_ELL) {
        s->in_entries = (int64_t)im.ep.in_ent.size() / 2;
        s->out_entries = (int64_t)im.ep.out_ent.size() / 2;
    }
    if (o.form == SNP_FORM_DENSE) s->in_entries = (int64_t)im.dense.size();
    s->rule_words = (int64_t)hp.rules.size();
    s->perm = hp.perm;
    s->rule_offsets.assign(desc->rule_offsets, desc->rule_offsets + (size_t)desc->q + 1);
    if (s->has_tiled) {
        s->tiled_smem = tiled_smem_bytes(im.tp);
        s->tiled_entries = (int64_t)im.tp.ent.size();
        s->tiled_threads = kTiledThreads;  // fixed: the entry layout is dealt to this many threads
        s->tiled_P = im.tp.P;
        s->tiled_G = im.tp.G;
        s->tiled_layout = im.tp.rle ? 2 : (im.tp.pairs ? 1 : 0);
        s->tiled_acc_bits = im.tp.acc8 ? 8 : 32;
    }
    {
        std::vector<Piece> plan;
        build_plan(s, plan);
        s->planned_bytes = plan_bytes(plan);
    }
    if (!(o.flags & SNP_FLAG_DEFER_UPLOAD)) {
        st = materialize(s);
        if (st) {
            sys_free_all(s);
            delete s;
            return st;
        }
    }
    *out = s;
    return SNP_OK;
}

int snp_destroy(snp_system* s) {
    if (!s) return SNP_OK;
    if (s->busy.load()) return fail(SNP_ERR_BUSY, "system is owned by an unfinished batch");
    if (s->stream) cudaStreamSynchronize(s->stream);
    else cudaDeviceSynchronize();
    if (s->chunk_exec) cudaGraphExecDestroy(s->chunk_exec);
    if (s->call_exec) cudaGraphExecDestroy(s->call_exec);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    batch_release(s);
    sys_free_all(s);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
    return SNP_OK;
}

// The system's descriptor with `forced` set (or cleared), also in its device
// copy (read by the CTA-resident engine).
static int set_forced(snp_system* s, const int32_t* forced) {
    s->dev.forced = forced;
    if (s->d_self &&
        cudaMemcpyAsync(s->d_self, &s->dev, sizeof(DevSys), cudaMemcpyHostToDevice, s->stream) != cudaSuccess)
        return cuda_fail("descriptor upload");
    return SNP_OK;
}

int snp_step(snp_system* s, int64_t n, int64_t* steps_done) {
    if (!s) return fail(SNP_ERR_INVALID, "system is NULL");
    if (s->busy.load()) return fail(SNP_ERR_BUSY, "system is owned by an unfinished batch");
    if (int rc_ = materialize(s)) return rc_;
    if (n < 0) return fail(SNP_ERR_INVALID, "n < 0");
    if (steps_done) *steps_done = 0;
    if (n == 0) return SNP_OK;
    if (s->choices_pending) {
        // the first step alone, with the forced choices, then the rest
        s->choices_pending = false;
        int rc = set_forced(s, s->d_forced);
        if (!rc) rc = run_steps(s, 1);
        const int rc2 = set_forced(s, nullptr);
        if (rc) return rc;
        if (rc2) return rc2;
        int64_t first = 0;
        if ((rc = read_flags(s, &first))) return rc;
        if (steps_done) *steps_done = first;
        if (n == 1 || first == 0) return SNP_OK;
        if ((rc = run_steps(s, n - 1))) return rc;
        int64_t rest = 0;
        if ((rc = read_flags(s, &rest))) return rc;
        if (steps_done) *steps_done += rest;
        return SNP_OK;
    }
    int rc = run_steps(s, n);
    if (rc) return rc;
    if (steps_done) return read_flags(s, steps_done);
    return SNP_OK;
}

// The message for the first invalid neuron a state check found; its three
// values are read back from the caller's arrays (host or device).
static int state_error(const snp_system* s, int32_t i, const int32_t* C, const int32_t* D, const int32_t* P,
                       const std::string& where = std::string()) {
    (void)s;
    int32_t c = 0, d = 0, p = 0;
    if (cudaMemcpy(&c, C + i, 4, cudaMemcpyDefault) != cudaSuccess ||
        cudaMemcpy(&d, D + i, 4, cudaMemcpyDefault) != cudaSuccess ||
        cudaMemcpy(&p, P + i, 4, cudaMemcpyDefault) != cudaSuccess)
        return cuda_fail("state read-back");
    const std::string at = " at neuron " + std::to_string(i);
    if (c < 0) return fail(SNP_ERR_INVALID, where + "negative spike count" + at);
    if (d < 0 || d > kMaxDelay) return fail(SNP_ERR_INVALID, where + "D out of range" + at);
    if (p == -1) return fail(SNP_ERR_INVALID, where + "D > 0 without a pending rule" + at);
    return fail(SNP_ERR_INVALID, where + "pending rule does not belong to neuron " + std::to_string(i));
}

int snp_branch_step(snp_system* s, int32_t nb, const int32_t* C, const int32_t* D, const int32_t* P,
                    const int32_t* choices, int32_t* C_out, int32_t* D_out, int32_t* P_out, int32_t* executed,
                    int32_t* bad, int32_t* counts) {
    if (!s) return fail(SNP_ERR_INVALID, "system is NULL");
    if (nb < 0) return fail(SNP_ERR_INVALID, "nb < 0");
    if (nb == 0) return SNP_OK;
    if (!C || !D || !P || !choices || !C_out || !D_out || !P_out || !executed || !bad)
        return fail(SNP_ERR_INVALID, "NULL argument");
    if (s->busy.load()) return fail(SNP_ERR_BUSY, "system is owned by an unfinished batch");
    if (int rc_ = materialize(s)) return rc_;
    if (s->opt.form != SNP_FORM_OPT || !s->has_in_lists || s->q > kBranchMaxQ)
        return fail(SNP_ERR_UNSUPPORTED, "branch steps need the optimized form with in-lists and q <= 8192");
    const size_t n = (size_t)nb * (size_t)s->q;
    cudaStream_t st = s->stream;
    // Host buffers are staged on the device in one block from the system's
    // allocator, together with the word the input check reports into.
    struct Buf {
        const void* user;
        void* dev;
        size_t bytes;
        bool in, host;
    };
    Buf bufs[10] = {{C, nullptr, n * 4, true, false},      {D, nullptr, n * 4, true, false},
                    {P, nullptr, n * 4, true, false},      {choices, nullptr, n * 4, true, false},
                    {C_out, nullptr, n * 4, false, false}, {D_out, nullptr, n * 4, false, false},
                    {P_out, nullptr, n * 4, false, false}, {executed, nullptr, (size_t)nb * 4, false, false},
                    {bad, nullptr, (size_t)nb * 4, false, false}, {counts, nullptr, n * 4, false, false}};
    size_t stage = 256;  // the first 256 bytes hold the check's word
    for (Buf& b : bufs) {
        if (!b.user) continue;  // counts is optional
        b.host = !is_device_ptr(b.user);
        if (b.host) stage += (b.bytes + 255) & ~(size_t)255;
    }
    char* block = (char*)stage_alloc(s, stage);
    if (!block) return fail(SNP_ERR_OOM, "staging buffer for snp_branch_step");
    unsigned long long* d_first_bad = (unsigned long long*)block;
    size_t off = 256;
    int rc = SNP_OK;
    for (Buf& b : bufs) {
        if (!b.user) continue;
        if (!b.host) {
            b.dev = const_cast<void*>(b.user);
            continue;
        }
        b.dev = block + off;
        off += (b.bytes + 255) & ~(size_t)255;
        if (b.in && cudaMemcpyAsync(b.dev, b.user, b.bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            rc = cuda_fail("staging copy");
            break;
        }
    }
    // The input check runs, and is read back, before the step kernel is
    // launched: a configuration out of range never reaches k_branch_step.
    unsigned long long first_bad = ~0ull;
    if (!rc && (cudaMemsetAsync(d_first_bad, 0xff, sizeof(unsigned long long), st) != cudaSuccess ||
                launch_branch_check(s->dev, s->d_rule_base, nb, (const int32_t*)bufs[0].dev,
                                    (const int32_t*)bufs[1].dev, (const int32_t*)bufs[2].dev, d_first_bad,
                                    st) != cudaSuccess ||
                cudaMemcpyAsync(&first_bad, d_first_bad, sizeof(first_bad), cudaMemcpyDeviceToHost, st) !=
                    cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess))
        rc = cuda_fail("branch input check");
    if (!rc && first_bad != ~0ull) {
        const unsigned long long b = first_bad / (unsigned long long)s->q;
        const int32_t i = (int32_t)(first_bad % (unsigned long long)s->q);
        rc = state_error(s, i, C + b * (unsigned long long)s->q, D + b * (unsigned long long)s->q,
                         P + b * (unsigned long long)s->q, "configuration " + std::to_string(b) + ": ");
    }
    if (!rc && launch_branch_step(s->dev, s->d_rule_base, resident_e_bits(s->max_p), s->compact, nb,
                                  (const int32_t*)bufs[0].dev, (const int32_t*)bufs[1].dev, (const int32_t*)bufs[2].dev,
                                  (const int32_t*)bufs[3].dev, (int32_t*)bufs[4].dev, (int32_t*)bufs[5].dev,
                                  (int32_t*)bufs[6].dev, (int32_t*)bufs[7].dev, (int32_t*)bufs[8].dev,
                                  (int32_t*)bufs[9].dev, st) != cudaSuccess)
        rc = cuda_fail("branch step");
    for (Buf& b : bufs) {
        if (!b.host || !b.dev || b.in || rc) continue;
        if (cudaMemcpyAsync(const_cast<void*>(b.user), b.dev, b.bytes, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            rc = cuda_fail("staging copy");
    }
    uint32_t over = 0;
    const bool synced = cudaMemcpyAsync(&over, s->dev.flags + kFlagOverflow, 4, cudaMemcpyDeviceToHost, st) ==
                            cudaSuccess &&
                        cudaStreamSynchronize(st) == cudaSuccess;
    stage_free(s, block, stage);
    if (!synced) return rc ? rc : cuda_fail("branch step");
    if (rc) return rc;
    if (over) {
        const uint32_t zero = 0;
        cudaMemcpyAsync(s->dev.flags + kFlagOverflow, &zero, 4, cudaMemcpyHostToDevice, st);
        cudaStreamSynchronize(st);
        return fail(SNP_ERR_OVERFLOW, "a spike count left the int32 range");
    }
    return SNP_OK;
}

int snp_set_choices(snp_system* s, const int32_t* idx, int64_t len) {
    if (!s || !idx) return fail(SNP_ERR_INVALID, "NULL argument");
    if (s->busy.load()) return fail(SNP_ERR_BUSY, "system is owned by an unfinished batch");
    if (int rc_ = materialize(s)) return rc_;
    if (len < s->q) return fail(SNP_ERR_INVALID, "choices shorter than q");
    std::vector<int32_t> host((size_t)s->q), slots((size_t)s->q);
    if (is_device_ptr(idx)) {
        if (cudaMemcpyAsync(host.data(), idx, sizeof(int32_t) * (size_t)s->q, cudaMemcpyDeviceToHost, s->stream) !=
                cudaSuccess ||
            cudaStreamSynchronize(s->stream) != cudaSuccess)
            return cuda_fail("choices copy");
    } else {
        std::memcpy(host.data(), idx, sizeof(int32_t) * (size_t)s->q);
    }
    for (int32_t slot = 0; slot < s->q; ++slot) slots[slot] = host[(size_t)s->perm[slot]];
    if (!s->d_forced) {
        s->d_forced = (int32_t*)sys_alloc(s, sizeof(int32_t) * (size_t)std::max(1, s->q));
        if (!s->d_forced) return fail(SNP_ERR_OOM, "device allocation for forced choices failed");
    }
    if (cudaMemcpyAsync(s->d_forced, slots.data(), sizeof(int32_t) * (size_t)s->q, cudaMemcpyHostToDevice,
                        s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return cuda_fail("choices upload");
    s->choices_pending = true;
    return SNP_OK;
}

static int export_vec(const snp_system* sc, int what, int32_t* out, int64_t len) {
    snp_system* s = const_cast<snp_system*>(sc);
    if (!s || !out) return fail(SNP_ERR_INVALID, "NULL argument");
    if (s->busy.load()) return fail(SNP_ERR_BUSY, "system is owned by an unfinished batch");
    if (int rc_ = materialize(s)) return rc_;
    if (len < s->q) return fail(SNP_ERR_INVALID, "output shorter than q");
    const bool dev = is_device_ptr(out);
    int32_t* dst = dev ? out : s->scratch;
    if (launch_export(s->dev, s->d_rule_base, what, dst, -1, s->stream, s->compact) != cudaSuccess)
        return cuda_fail("export");
    if (!dev) {
        if (cudaMemcpyAsync(out, s->scratch, sizeof(int32_t) * (size_t)s->q, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
            cudaStreamSynchronize(s->stream) != cudaSuccess)
            return cuda_fail("export copy");
    }
    return SNP_OK;
}

int snp_get_config(const snp_system* s, int32_t* out, int64_t len) { return export_vec(s, kExportConfig, out, len); }
int snp_count_choices(const snp_system* s, int32_t* out, int64_t len) {
    return export_vec(s, kExportChoices, out, len);
}
int snp_get_spiking(const snp_system* s, int32_t* out, int64_t len) { return export_vec(s, kExportSpiking, out, len); }
int snp_get_status(const snp_system* s, int32_t* out, int64_t len) { return export_vec(s, kExportStatus, out, len); }
int snp_get_pending(const snp_system* s, int32_t* out, int64_t len) { return export_vec(s, kExportPending, out, len); }

int snp_get_state(const snp_system* s, int32_t* C, int32_t* D, int32_t* P, int64_t len, uint64_t* step) {
    if (!s) return fail(SNP_ERR_INVALID, "system is NULL");
    if (int rc_ = materialize(const_cast<snp_system*>(s))) return rc_;
    int rc;
    if (C && (rc = snp_get_config(s, C, len))) return rc;
    if (D && (rc = snp_get_status(s, D, len))) return rc;
    if (P && (rc = snp_get_pending(s, P, len))) return rc;
    if (step) {
        unsigned long long v = 0;
        if (cudaMemcpyAsync(&v, s->dev.step + kStepBase, sizeof(v), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
            cudaStreamSynchronize(s->stream) != cudaSuccess)
            return cuda_fail("step read");
        *step = v;
    }
    return SNP_OK;
}

// Imports (C, D, P) on the device: the three arrays are copied (from host or
// device memory) into buffers whose contents set_state discards anyway (the
// spiking vectors and the export scratch), checked by one launch, and only
// if every neuron passes written in slot order by a second.
int snp_set_state(snp_system* s, const int32_t* C, const int32_t* D, const int32_t* P, int64_t len, uint64_t step) {
    if (!s || !C || !D || !P) return fail(SNP_ERR_INVALID, "NULL argument");
    if (s->busy.load()) return fail(SNP_ERR_BUSY, "system is owned by an unfinished batch");
    if (int rc_ = materialize(s)) return rc_;
    if (len < s->q) return fail(SNP_ERR_INVALID, "state shorter than q");
    cudaStream_t st = s->stream;
    const size_t bytes = sizeof(int32_t) * (size_t)s->q;
    int32_t* sc = s->scratch;
    int32_t* sd = s->dev.S[0];
    int32_t* sp = s->dev.S[1];
    uint32_t bad = 0xffffffffu;
    if (cudaMemcpyAsync(sc, C, bytes, cudaMemcpyDefault, st) != cudaSuccess ||
        cudaMemcpyAsync(sd, D, bytes, cudaMemcpyDefault, st) != cudaSuccess ||
        cudaMemcpyAsync(sp, P, bytes, cudaMemcpyDefault, st) != cudaSuccess ||
        cudaMemsetAsync(s->dev.flags + kFlagImport, 0xff, sizeof(uint32_t), st) != cudaSuccess ||
        launch_import(s->dev, s->d_rule_base, sc, sd, sp, false, st) != cudaSuccess ||
        cudaMemcpyAsync(&bad, s->dev.flags + kFlagImport, sizeof(bad), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return cuda_fail("state upload");
    if (bad == 0xffffffffu && launch_import(s->dev, s->d_rule_base, sc, sd, sp, true, st) != cudaSuccess)
        return cuda_fail("state import");
    // the spiking vectors held the staged D and P: all -1 again either way
    if (cudaMemsetAsync(s->dev.S[0], 0xff, bytes, st) != cudaSuccess ||
        cudaMemsetAsync(s->dev.S[1], 0xff, bytes, st) != cudaSuccess)
        return cuda_fail("state upload");
    if (bad != 0xffffffffu) {
        if (cudaStreamSynchronize(st) != cudaSuccess) return cuda_fail("state upload");
        return state_error(s, (int32_t)bad, C, D, P);
    }
    unsigned long long steps[kNumStepWords] = {step, step, 0ull, 0ull};
    uint32_t fz[kNumFlags] = {0};
    if (cudaMemcpyAsync(s->dev.step, steps, sizeof(steps), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(s->dev.flags, fz, sizeof(fz), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return cuda_fail("state upload");
    return SNP_OK;
}

int snp_check_bounded_wait(int32_t polls) {
    if (polls < 1 || polls > 1000000) return fail(SNP_ERR_INVALID, "polls must be in 1..1000000");
    cudaStream_t st = nullptr;
    uint32_t* d_out = nullptr;
    uint32_t h_out = 0;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) return cuda_fail("stream");
    int rc = SNP_OK;
    if (cudaMalloc(&d_out, sizeof(uint32_t)) != cudaSuccess || cudaMemsetAsync(d_out, 0, 4, st) != cudaSuccess ||
        launch_wait_check(polls, d_out, st) != cudaSuccess ||
        cudaMemcpyAsync(&h_out, d_out, 4, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        rc = cuda_fail("bounded wait check");
    else if (h_out == 2u)
        rc = fail(SNP_ERR_TIMEOUT, "the bounded wait gave up after " + std::to_string(polls) + " polls");
    else if (h_out != 1u)
        rc = fail(SNP_ERR_CUDA, "the wait check did not report");
    if (d_out) cudaFree(d_out);
    cudaStreamDestroy(st);
    return rc;
}

int snp_get_info(const snp_system* s, snp_info* info) {
    if (!s || !info) return fail(SNP_ERR_INVALID, "NULL argument");
    std::memset(info, 0, sizeof(*info));
    info->q = s->q;
    info->form = s->opt.form;
    info->prop = s->opt.prop;
    info->select = s->opt.select;
    info->engine = effective_engine(s);
    info->m = s->m;
    info->num_syn = s->nsyn;
    info->in_entries = info->engine == SNP_ENGINE_TILED ? s->tiled_entries : s->in_entries;
    info->out_entries = s->out_entries;
    info->rule_words = s->rule_words;
    info->device_bytes = (int64_t)(s->materialized ? s->device_bytes : s->planned_bytes);
    info->max_rules = s->max_rules;
    info->max_p = s->max_p;
    info->compact_rules = s->compact ? 1 : 0;
    info->e_bits = info->engine == SNP_ENGINE_TILED ? s->tiled.e_bits : resident_e_bits(s->max_p);
    info->step = s->host_step;
    info->compiled_rules = s->compiled ? 1 : 0;
    if (s->has_tiled) {
        info->tiled_partitions = s->tiled_P;
        info->tiled_ctas = s->tiled_G;
        info->tiled_layout = s->tiled_layout;
        info->tiled_acc_bits = s->tiled_acc_bits;
        info->tiled_smem_bytes = (int64_t)s->tiled_smem;
    }
    return SNP_OK;
}

}  // extern "C"
