// Neuron-sharded step: one system split by neuron range, each range (shard)
// on its own device, one exchange of emissions per step.
//
// A system too large for one device is partitioned by neuron range.  Every
// step of the definition has one point where a neuron needs data of other
// neurons: the in-flow of phase 2 (Sec. 2: the spikes a neuron receives are
// the emissions of its in-neighbours).  Phase 1 (the choice of a rule,
// consumption, the delay status) and the delay update only read the
// neuron's own state.  So a shard runs phase 1 for its neurons, writing
// their emissions into its slice of a full-length emission vector; the
// caller exchanges the slices between shards (an allgather of the vector,
// 2 bytes per neuron); the shard then runs phase 2 for its neurons from the
// whole vector.  The fixed-point test is the OR over shards of "a neuron of
// mine is pending or chose a rule", which the caller reduces with the same
// exchange.  A shard's in-lists hold global source ids, so no data but the
// emissions crosses devices, and remote data is only ever read after it has
// been copied into the shard's own vector.
//
// Kernels: one thread per neuron of the shard (select: the library's select
// of a slot with the global neuron id as the Philox counter word; gather:
// the neuron's CSR in-list against the emission vector, 64-bit sums).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "device_common.cuh"
#include "snp_internal.h"

struct snp_shard {
    int32_t q = 0, lo = 0, hi = 0, n = 0;
    snp_options opt{};
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    snp::DevSys dev{};          // the shard's neurons as a system of n slots (orig = global ids)
    uint16_t* E = nullptr;      // [q + 1] emissions of the step being run, caller's or own
    int32_t* in_off = nullptr;  // [n + 1] CSR in-lists of the shard's neurons
    int32_t* in_src = nullptr;  // global source ids
    void* block = nullptr;      // one device allocation for everything the shard owns
    bool compact = true;
    std::vector<int64_t> rule_offsets;  // the system's N_Pi (global rule ids on export)
    int s_last = -1;            // parity of the spiking vector of the last executed step, -1 none
    unsigned long long k_sel = 0;
    bool selected = false;      // phase 1 of step k_sel ran, phase 2 not yet
};

namespace snp {

constexpr int kShardFlagActive = 0, kShardFlagOverflow = 1;

template <bool COMPACT, int SEL>
__global__ void __launch_bounds__(256) k_shard_select(DevSys s, uint16_t* E, int32_t lo, unsigned long long k) {
    const int32_t i = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    bool act = false;
    if (i < s.q) {
        const SelOut o = select_slot<COMPACT, SEL>(s, i, s.C[i], s.st[i], k);
        s.C[i] = o.c_after;
        s.st[i] = o.st;
        SNP_PICK(s.S, k)[i] = o.s;
        E[lo + i] = (uint16_t)o.emit;  // p <= 65535
        act = o.active;
    }
    if (__syncthreads_or(act) && threadIdx.x == 0) atomicOr(s.flags + kShardFlagActive, 1u);
}

__global__ void __launch_bounds__(256) k_shard_gather(DevSys s, const uint16_t* __restrict__ E,
                                                      const int32_t* __restrict__ in_off,
                                                      const int32_t* __restrict__ in_src) {
    const int32_t i = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    if (i >= s.q) return;
    if ((s.st[i] >> kPendShift) != 0u) return;  // closed this step: receives nothing
    long long sum = 0;
    for (int32_t e = in_off[i]; e < in_off[i + 1]; ++e) sum += E[in_src[e]];
    long long c = (long long)s.C[i] + sum;
    if (c > 2147483647ll) {
        atomicOr(s.flags + kShardFlagOverflow, 1u);
        c = 2147483647ll;
    }
    s.C[i] = (int32_t)c;
}

static int shard_cuda_fail(const char* what) {
    const cudaError_t e = cudaGetLastError();
    return fail(SNP_ERR_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

}  // namespace snp

using namespace snp;

extern "C" {

int snp_shard_create(const snp_desc* d, int32_t lo, int32_t hi, const snp_options* opts, uint16_t* E,
                     snp_shard** out) {
    if (!out) return fail(SNP_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (int st = validate_desc(d)) return st;
    if (lo < 0 || hi > d->q || lo >= hi) return fail(SNP_ERR_INVALID, "need 0 <= lo < hi <= q");
    snp_options o{};
    if (opts) o = *opts;
    if (o.select != SNP_SELECT_FIRST && o.select != SNP_SELECT_PHILOX) return fail(SNP_ERR_INVALID, "bad select");
    const int32_t n = hi - lo;
    const int64_t r0 = d->rule_offsets[lo], r1 = d->rule_offsets[hi];
    // the shard's neurons and rules as a system of their own (no synapses):
    // the packer lays out their rule table and compiled records
    std::vector<int64_t> ro((size_t)n + 1), so((size_t)n + 1, 0), to;
    for (int32_t i = 0; i <= n; ++i) ro[(size_t)i] = d->rule_offsets[lo + i] - r0;
    snp_desc sub{};
    sub.q = n;
    sub.init_spikes = d->init_spikes + lo;
    sub.rule_offsets = ro.data();
    sub.rule_k = d->rule_k ? d->rule_k + r0 : nullptr;
    sub.rule_j = d->rule_j ? d->rule_j + r0 : nullptr;
    sub.rule_c = d->rule_c + r0;
    sub.rule_p = d->rule_p + r0;
    sub.rule_d = d->rule_d + r0;
    sub.num_syn = 0;
    sub.syn_offsets = so.data();
    sub.syn_targets = nullptr;
    if (d->rule_term_offsets) {
        const int64_t t0 = d->rule_term_offsets[r0];
        to.resize((size_t)(r1 - r0) + 1);
        for (int64_t r = 0; r <= r1 - r0; ++r) to[(size_t)r] = d->rule_term_offsets[r0 + r] - t0;
        sub.rule_term_offsets = to.data();
        sub.term_k = d->term_k + t0;
        sub.term_j = d->term_j + t0;
    }
    HostPack hp;
    if (int st = pack_system(&sub, false, false, 0, &hp)) return st;
    // in-lists of the shard's neurons, sources as global ids
    std::vector<int32_t> in_off((size_t)n + 1, 0);
    for (int64_t e = 0; e < d->num_syn; ++e) {
        const int32_t t = d->syn_targets[e];
        if (t >= lo && t < hi) in_off[(size_t)(t - lo) + 1]++;
    }
    for (int32_t i = 0; i < n; ++i) {
        if ((int64_t)in_off[(size_t)i + 1] + in_off[(size_t)i] > INT32_MAX)
            return fail(SNP_ERR_UNSUPPORTED, "shard has more than 2^31 in-edges");
        in_off[(size_t)i + 1] += in_off[(size_t)i];
    }
    std::vector<int32_t> in_src((size_t)std::max(1, in_off[(size_t)n])), fill(in_off.begin(), in_off.end() - 1);
    for (int32_t i = 0; i < d->q; ++i)
        for (int64_t e = d->syn_offsets[i]; e < d->syn_offsets[i + 1]; ++e) {
            const int32_t t = d->syn_targets[e];
            if (t >= lo && t < hi) in_src[(size_t)fill[(size_t)(t - lo)]++] = i;
        }
    std::vector<int32_t> orig((size_t)n);
    for (int32_t i = 0; i < n; ++i) orig[(size_t)i] = lo + i;

    snp_shard* s = new (std::nothrow) snp_shard();
    if (!s) return fail(SNP_ERR_OOM, "host allocation failed");
    s->q = d->q;
    s->lo = lo;
    s->hi = hi;
    s->n = n;
    s->opt = o;
    s->compact = hp.compact;
    s->rule_offsets.assign(d->rule_offsets, d->rule_offsets + (size_t)d->q + 1);
    if (o.stream) {
        s->stream = (cudaStream_t)o.stream;
    } else if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) == cudaSuccess) {
        s->own_stream = true;
    } else {
        delete s;
        return shard_cuda_fail("stream create");
    }
    // one allocation: every piece 256-byte aligned
    const bool compiled = !hp.rec.empty();
    struct P {
        void** dst;
        const void* src;
        size_t bytes;
        int fill;
    };
    DevSys& dv = s->dev;
    std::vector<P> plan = {{(void**)&dv.rule_off, hp.rule_off.data(), hp.rule_off.size() * 4, -1},
                           {(void**)&dv.rules, hp.rules.data(), std::max<size_t>(4, hp.rules.size() * 4), -1},
                           {(void**)&dv.orig, orig.data(), orig.size() * 4, -1},
                           {(void**)&dv.C, hp.C0.data(), hp.C0.size() * 4, -1},
                           {(void**)&dv.st, nullptr, (size_t)n * 4, 0},
                           {(void**)&dv.S[0], nullptr, (size_t)n * 4, 0xff},
                           {(void**)&dv.S[1], nullptr, (size_t)n * 4, 0xff},
                           {(void**)&dv.flags, nullptr, 16, 0},
                           {(void**)&s->in_off, in_off.data(), in_off.size() * 4, -1},
                           {(void**)&s->in_src, in_src.data(), in_src.size() * 4, -1}};
    if (compiled) plan.push_back({(void**)&dv.rec, hp.rec.data(), hp.rec.size() * 4, -1});
    if (!E) plan.push_back({(void**)&s->E, nullptr, ((size_t)d->q + 1) * 2, 0});
    size_t total = 0;
    for (const P& p : plan) total += (p.bytes + 255) & ~(size_t)255;
    if (cudaMalloc(&s->block, total) != cudaSuccess) {
        cudaGetLastError();
        if (s->own_stream) cudaStreamDestroy(s->stream);
        delete s;
        return fail(SNP_ERR_OOM, "device allocation of " + std::to_string(total) + " bytes failed");
    }
    size_t off = 0;
    int rc = SNP_OK;
    for (const P& p : plan) {
        *p.dst = (char*)s->block + off;
        cudaError_t e = p.src ? cudaMemcpyAsync(*p.dst, p.src, p.bytes, cudaMemcpyHostToDevice, s->stream)
                              : cudaMemsetAsync(*p.dst, p.fill, p.bytes, s->stream);
        if (e != cudaSuccess) rc = shard_cuda_fail("shard upload");
        off += (p.bytes + 255) & ~(size_t)255;
    }
    if (E) s->E = E;
    dv.q = n;
    dv.nslices = (n + kSlice - 1) / kSlice;
    if (!compiled) dv.rec = nullptr;
    dv.seed = o.seed;
    philox_round_keys(dv.seed, dv.philox_rk);
    dv.select = o.select;
    dv.max_p = hp.max_p;
    dv.forced = nullptr;
    dv.rules_per_neuron = hp.uniform_rules;
    dv.identity = 0;  // orig[slot] = lo + slot: the global neuron id keys Philox
    if (!rc && cudaStreamSynchronize(s->stream) != cudaSuccess) rc = shard_cuda_fail("shard upload");
    if (rc) {
        cudaFree(s->block);
        if (s->own_stream) cudaStreamDestroy(s->stream);
        delete s;
        return rc;
    }
    *out = s;
    return SNP_OK;
}

int snp_shard_destroy(snp_shard* s) {
    if (!s) return SNP_OK;
    cudaStreamSynchronize(s->stream);
    cudaFree(s->block);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    delete s;
    return SNP_OK;
}

int snp_shard_emissions(snp_shard* s, uint16_t** out) {
    if (!s || !out) return fail(SNP_ERR_INVALID, "NULL argument");
    *out = s->E;
    return SNP_OK;
}

int snp_shard_select(snp_shard* s, uint64_t k, int32_t* active) {
    if (!s || !active) return fail(SNP_ERR_INVALID, "NULL argument");
    *active = 0;
    uint32_t fl[2] = {0u, 0u};
    const unsigned grid = (unsigned)((s->n + 255) / 256);
    if (cudaMemsetAsync(s->dev.flags + kShardFlagActive, 0, 4, s->stream) != cudaSuccess)
        return shard_cuda_fail("shard select");
    if (s->compact) {
        if (s->opt.select == SNP_SELECT_FIRST)
            k_shard_select<true, SNP_SELECT_FIRST><<<grid, 256, 0, s->stream>>>(s->dev, s->E, s->lo, k);
        else
            k_shard_select<true, SNP_SELECT_PHILOX><<<grid, 256, 0, s->stream>>>(s->dev, s->E, s->lo, k);
    } else {
        if (s->opt.select == SNP_SELECT_FIRST)
            k_shard_select<false, SNP_SELECT_FIRST><<<grid, 256, 0, s->stream>>>(s->dev, s->E, s->lo, k);
        else
            k_shard_select<false, SNP_SELECT_PHILOX><<<grid, 256, 0, s->stream>>>(s->dev, s->E, s->lo, k);
    }
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(fl, s->dev.flags, sizeof(fl), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return shard_cuda_fail("shard select");
    s->k_sel = k;
    s->selected = true;
    *active = fl[kShardFlagActive] ? 1 : 0;
    if (fl[kShardFlagOverflow]) return fail(SNP_ERR_OVERFLOW, "a spike count left the int32 range");
    return SNP_OK;
}

int snp_shard_gather(snp_shard* s) {
    if (!s) return fail(SNP_ERR_INVALID, "NULL shard");
    if (!s->selected) return fail(SNP_ERR_INVALID, "snp_shard_gather before snp_shard_select");
    const unsigned grid = (unsigned)((s->n + 255) / 256);
    k_shard_gather<<<grid, 256, 0, s->stream>>>(s->dev, s->E, s->in_off, s->in_src);
    if (cudaGetLastError() != cudaSuccess) return shard_cuda_fail("shard gather");
    s->s_last = (int)(s->k_sel & 1ull);
    s->selected = false;
    return SNP_OK;
}

int snp_shard_get_state(const snp_shard* s, int32_t* C, int32_t* D, int32_t* P, int32_t* S, int64_t len) {
    if (!s || !C || !D || !P || !S) return fail(SNP_ERR_INVALID, "NULL argument");
    if (len < s->n) return fail(SNP_ERR_INVALID, "arrays shorter than the shard");
    const size_t n = (size_t)s->n;
    std::vector<int32_t> c(n), sv(n, -1);
    std::vector<uint32_t> st(n);
    uint32_t fl[2] = {0u, 0u};
    if (cudaMemcpyAsync(c.data(), s->dev.C, n * 4, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaMemcpyAsync(st.data(), s->dev.st, n * 4, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        (s->s_last >= 0 &&
         cudaMemcpyAsync(sv.data(), s->dev.S[s->s_last], n * 4, cudaMemcpyDeviceToHost, s->stream) != cudaSuccess) ||
        cudaMemcpyAsync(fl, s->dev.flags, sizeof(fl), cudaMemcpyDeviceToHost, s->stream) != cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess)
        return shard_cuda_fail("shard state read");
    std::vector<int32_t> d(n), p(n), sg(n);
    for (size_t i = 0; i < n; ++i) {
        const uint32_t pend = st[i] >> kPendShift;
        const int64_t base = s->rule_offsets[(size_t)s->lo + i];
        d[i] = pend ? (int32_t)(st[i] & kDMask) : 0;
        p[i] = pend ? (int32_t)(base + pend - 1) : -1;
        sg[i] = sv[i] >= 0 ? (int32_t)(base + sv[i]) : -1;
    }
    if (cudaMemcpy(C, c.data(), n * 4, cudaMemcpyDefault) != cudaSuccess ||
        cudaMemcpy(D, d.data(), n * 4, cudaMemcpyDefault) != cudaSuccess ||
        cudaMemcpy(P, p.data(), n * 4, cudaMemcpyDefault) != cudaSuccess ||
        cudaMemcpy(S, sg.data(), n * 4, cudaMemcpyDefault) != cudaSuccess)
        return shard_cuda_fail("shard state copy");
    if (fl[kShardFlagOverflow]) return fail(SNP_ERR_OVERFLOW, "a spike count left the int32 range");
    return SNP_OK;
}

}  // extern "C"
