// snp_step_noalloc: the pull step for callers that must not allocate.
//
// Some callers cannot call cudaMalloc: code running inside a host framework
// that owns every byte of device memory (a plugin or custom operator whose
// framework hands out memory only through its own pool), or latency-critical
// loops where an allocation may synchronize the device at an unpredictable
// moment.  This entry point takes the system and its state in the caller's
// device arrays and keeps its own working buffers (the two emission vectors
// and a few flag words) in one file-scope device array of fixed size, so it
// allocates nothing.
//
// The kernels are a variant of the grid-wide pull step (kernels_step.cu):
// one launch per SNP step fuses the gather of step k with the select of step
// k+1, on the caller's neuron order and in-neighbour CSR lists, with the
// state kept as the caller's (C, D, P) arrays.  Every index read from the
// caller's arrays is bounds-checked, and so are the fields of every rule a
// step fires (the ranges snp_create enforces on the host: k, j, c >= 0,
// p and d in [0, 65535], no delay on a forgetting rule) and the number of
// rules of a neuron; a bad one sets an error flag and the call returns
// SNP_ERR_INVALID instead of silently packing an out-of-range value.
#include <cuda_runtime.h>

#include <mutex>

#include "device_common.cuh"
#include "snp_internal.h"

namespace snp {

// ---- the static scratch ----------------------------------------------------
// Layout (32-bit words): [0, 16) flag words, [16, 24) step counters (four
// 64-bit values), then two emission vectors of SNP_NOALLOC_MAX_Q + 1 words.
// Each emission word holds the spikes sent (low 16 bits) and 1 + the local
// index of the rule selected at that step (high 16 bits, 0 = none).
constexpr int kNaFlagWords = 16;
constexpr int kNaStepWords = 8;
constexpr long long kNaEWords = (long long)SNP_NOALLOC_MAX_Q + 1;
constexpr long long kNaWords = kNaFlagWords + kNaStepWords + 2 * kNaEWords;
enum : int { kNaAct0 = 0, kNaHalted = 3, kNaOverflow = 4, kNaInvalid = 5 };
enum : int { kNaBase = 0, kNaStart = 1, kNaExec = 2, kNaHalt = 3 };

static __device__ __align__(256) uint32_t g_noalloc_scratch[kNaWords];

struct NaSys {
    int32_t q;
    long long m;
    const int32_t* rule_off;
    const int32_t* rk;
    const int32_t* rj;
    const int32_t* rc;
    const int32_t* rp;
    const int32_t* rd;
    const int32_t* in_off;
    const int32_t* in_src;
    long long nin;
    int32_t* C;
    int32_t* D;
    int32_t* P;
    int32_t* S;
    uint32_t* scratch;  // device address of g_noalloc_scratch
    uint64_t seed;
};

__device__ __forceinline__ uint32_t* na_flags(const NaSys& s) { return s.scratch; }
__device__ __forceinline__ unsigned long long* na_steps(const NaSys& s) {
    return reinterpret_cast<unsigned long long*>(s.scratch + kNaFlagWords);
}
__device__ __forceinline__ uint32_t* na_e(const NaSys& s, unsigned long long k) {
    return s.scratch + kNaFlagWords + kNaStepWords + (k & 1ull) * kNaEWords;
}

__device__ __forceinline__ RuleF na_rule(const NaSys& s, int32_t r) {
    RuleF f;
    f.k = s.rk[r];
    f.j = s.rj[r];
    f.c = s.rc[r];
    f.p = s.rp[r];
    f.d = s.rd[r];
    return f;
}

// The field ranges snp_create's validation enforces on the host; the status
// word and the emission words below hold p and d in 16 bits.
__device__ __forceinline__ bool na_rule_ok(const RuleF& f) {
    return f.k >= 0 && f.j >= 0 && f.c >= 0 && f.p >= 0 && f.p <= kMaxP && f.d >= 0 && f.d <= kMaxDelay &&
           (f.p != 0 || f.d == 0);
}

// Select phase of neuron j at step k on the caller's state; same rules as
// select_neuron in device_common.cuh, over rule fields held as separate arrays.
// *bad is set when a rule the step fires has a field out of range (the step
// then treats the neuron as idle).
template <int SEL>
__device__ __forceinline__ SelOut na_select(const NaSys& s, int32_t j, int32_t r0, int32_t r1, int32_t n,
                                            uint32_t st, unsigned long long k, bool* bad) {
    SelOut o;
    o.c_after = n;
    o.emit = 0;
    o.s = -1;
    const uint32_t pend = st >> kPendShift;
    if (pend != 0u) {
        o.active = true;
        if ((st & kDMask) == 0u) {
            const RuleF f = na_rule(s, r0 + (int32_t)pend - 1);
            if (!na_rule_ok(f)) {
                *bad = true;
                o.active = false;
            } else {
                o.emit = f.p;
            }
            o.st = 0u;
        } else {
            o.st = st - 1u;
        }
        return o;
    }
    o.st = 0u;
    o.active = false;
    int32_t pick = -1, cnt = 0, first = -1;
    for (int32_t r = r0; r < r1; ++r) {
        if (rule_applies(n, na_rule(s, r))) {
            if (cnt == 0) first = r;
            ++cnt;
            if (SEL == SNP_SELECT_FIRST) break;
        }
    }
    if (cnt == 1 || (SEL == SNP_SELECT_FIRST && cnt > 0)) {
        pick = first;
    } else if (cnt > 1) {
        const uint32_t x = philox_draw(k, (uint32_t)j, s.seed);
        int32_t idx = (int32_t)(((unsigned long long)x * (unsigned long long)cnt) >> 32);
        for (int32_t r = first; r < r1; ++r) {
            if (rule_applies(n, na_rule(s, r))) {
                if (idx == 0) {
                    pick = r;
                    break;
                }
                --idx;
            }
        }
    }
    if (pick >= 0) {
        const RuleF f = na_rule(s, pick);
        if (!na_rule_ok(f)) {
            *bad = true;
            return o;
        }
        o.active = true;
        o.s = pick - r0;
        o.c_after = n - f.c;
        if (f.d == 0)
            o.emit = f.p;
        else
            o.st = ((uint32_t)(o.s + 1) << kPendShift) | (uint32_t)(f.d - 1);
    }
    return o;
}

template <bool GATHER, bool SELECT, int SEL>
__global__ void __launch_bounds__(256) k_na_step(NaSys s, int32_t t) {
    uint32_t* fl = na_flags(s);
    unsigned long long* steps = na_steps(s);
    const unsigned long long kg = steps[kNaBase] + (unsigned long long)t;
    const unsigned long long ks = GATHER ? kg + 1ull : kg;
    if (GATHER) {
        if (ld_volatile(fl + kNaHalted)) return;
        if (ld_volatile(fl + kNaAct0 + (int)(kg % 3ull)) == 0u) {
            if (threadIdx.x == 0) {
                steps[kNaHalt] = kg;
                __threadfence();
                atomicExch(fl + kNaHalted, 1u);
            }
            return;
        }
        if (SELECT && blockIdx.x == 0 && threadIdx.x == 0) fl[kNaAct0 + (int)((kg + 2ull) % 3ull)] = 0u;
    }
    const int32_t j = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    bool active = false;
    if (j < s.q) {
        int32_t r0 = s.rule_off[j], r1 = s.rule_off[j + 1];
        int32_t c = s.C[j];
        bool ok = r0 >= 0 && r0 <= r1 && (long long)r1 <= s.m && r1 - r0 <= kMaxRulesPerNeuron && c >= 0;
        const int32_t P = s.P[j], D = s.D[j];
        uint32_t st = 0u;
        if (P != -1) {
            ok = ok && P >= r0 && P < r1 && D >= 0 && D <= (int32_t)kDMask;
            st = ((uint32_t)(P - r0 + 1) << kPendShift) | ((uint32_t)D & kDMask);
        } else {
            ok = ok && D == 0;  // a neuron can only be closed by a pending rule
        }
        if (!ok) {
            atomicOr(fl + kNaInvalid, 1u);
            r0 = r1 = 0;
            st = 0u;
        }
        if (GATHER) {
            const uint32_t* Ek = na_e(s, kg);
            const int32_t a = s.in_off[j], b = s.in_off[j + 1];
            long long sum = 0;
            if (a < 0 || a > b || (long long)b > s.nin) {
                atomicOr(fl + kNaInvalid, 1u);
            } else {
                for (int32_t e = a; e < b; ++e) {
                    const int32_t src = s.in_src[e];
                    if (src < 0 || src >= s.q) {
                        atomicOr(fl + kNaInvalid, 1u);
                        continue;
                    }
                    sum += (long long)(Ek[src] & 0xffffu);
                }
            }
            if ((st >> kPendShift) == 0u) {
                long long nc = (long long)c + sum;
                if (nc > 2147483647ll) {
                    atomicOr(fl + kNaOverflow, 1u);
                    nc = 2147483647ll;
                }
                c = (int32_t)nc;
            }
            // step kg is executed: publish its spiking vector
            const uint32_t sel = Ek[j] >> 16;
            s.S[j] = sel ? r0 + (int32_t)sel - 1 : -1;
        }
        if (SELECT) {
            bool bad = false;
            const SelOut o = na_select<SEL>(s, j, r0, r1, c, st, ks, &bad);
            if (bad) atomicOr(fl + kNaInvalid, 1u);
            c = o.c_after;
            active = o.active;
            na_e(s, ks)[j] = ((uint32_t)o.emit & 0xffffu) | ((uint32_t)(o.s + 1) << 16);
            const uint32_t pend = o.st >> kPendShift;
            s.P[j] = pend ? r0 + (int32_t)pend - 1 : -1;
            s.D[j] = pend ? (int32_t)(o.st & kDMask) : 0;
        }
        s.C[j] = c;
    }
    if (SELECT) {
        if (__syncthreads_or(active) && threadIdx.x == 0) {
            uint32_t* a = fl + kNaAct0 + (int)(ks % 3ull);
            if (ld_volatile(a) == 0u) atomicExch(a, 1u);
        }
    }
}

__global__ void k_na_begin(NaSys s, unsigned long long k0) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        uint32_t* fl = na_flags(s);
        for (int i = 0; i < kNaFlagWords; ++i) fl[i] = 0u;
        unsigned long long* st = na_steps(s);
        st[kNaBase] = k0;
        st[kNaStart] = k0;
        st[kNaExec] = 0ull;
        st[kNaHalt] = 0ull;
    }
}

__global__ void k_na_finish(NaSys s, int32_t tail) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        unsigned long long* st = na_steps(s);
        if (ld_volatile(na_flags(s) + kNaHalted))
            st[kNaBase] = st[kNaHalt];
        else
            st[kNaBase] += (unsigned long long)tail;
        st[kNaExec] = st[kNaBase] - st[kNaStart];
    }
}

template <bool G, bool S>
static void na_launch(const NaSys& s, int32_t t, int sel, cudaStream_t st) {
    const unsigned grid = (unsigned)((s.q + 255) / 256);
    if (sel == SNP_SELECT_FIRST)
        k_na_step<G, S, SNP_SELECT_FIRST><<<grid, 256, 0, st>>>(s, t);
    else
        k_na_step<G, S, SNP_SELECT_PHILOX><<<grid, 256, 0, st>>>(s, t);
}

// Device address of the scratch array, looked up once per device.  The
// cached address belongs to the device's primary context: cudaDeviceReset
// makes it stale, which the library cannot detect (documented in snp.h).
static std::mutex g_na_mu;
static uint32_t* g_na_ptr[64] = {nullptr};

static int na_scratch(uint32_t** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return fail(SNP_ERR_CUDA, "no current CUDA device");
    }
    std::lock_guard<std::mutex> lk(g_na_mu);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return fail(SNP_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
        }
        g_na_ptr[dev] = (uint32_t*)p;
    }
    *out = g_na_ptr[dev];
    return SNP_OK;
}

}  // namespace snp

using namespace snp;

extern "C" int snp_step_noalloc(const snp_device_system* d, int32_t select, uint64_t seed, uint64_t step, int64_t n,
                                void* stream, int64_t* steps_done) {
    if (steps_done) *steps_done = 0;
    if (!d) return fail(SNP_ERR_INVALID, "system is NULL");
    if (d->q < 1 || d->q > SNP_NOALLOC_MAX_Q)
        return fail(SNP_ERR_INVALID, "q must be in [1, SNP_NOALLOC_MAX_Q] (262,144) for snp_step_noalloc");
    if (d->m < 0 || d->m > INT32_MAX - 1 || d->num_in < 0 || d->num_in > INT32_MAX)
        return fail(SNP_ERR_INVALID, "m or num_in out of range");
    if (!d->rule_offsets || (d->m > 0 && (!d->rule_k || !d->rule_j || !d->rule_c || !d->rule_p || !d->rule_d)) ||
        !d->in_offsets || (d->num_in > 0 && !d->in_sources) || !d->C || !d->D || !d->P || !d->S)
        return fail(SNP_ERR_INVALID, "NULL array");
    if (select != SNP_SELECT_FIRST && select != SNP_SELECT_PHILOX) return fail(SNP_ERR_INVALID, "bad select");
    if (n < 0 || n > INT32_MAX) return fail(SNP_ERR_INVALID, "n must be in [0, 2^31 - 1]");
    if (n == 0) return SNP_OK;
    uint32_t* scratch = nullptr;
    int rc = na_scratch(&scratch);
    if (rc) return rc;
    NaSys s;
    s.q = d->q;
    s.m = d->m;
    s.rule_off = d->rule_offsets;
    s.rk = d->rule_k;
    s.rj = d->rule_j;
    s.rc = d->rule_c;
    s.rp = d->rule_p;
    s.rd = d->rule_d;
    s.in_off = d->in_offsets;
    s.in_src = d->in_sources;
    s.nin = d->num_in;
    s.C = d->C;
    s.D = d->D;
    s.P = d->P;
    s.S = d->S;
    s.scratch = scratch;
    s.seed = seed;
    cudaStream_t st = (cudaStream_t)stream;
    k_na_begin<<<1, 32, 0, st>>>(s, (unsigned long long)step);
    na_launch<false, true>(s, 0, select, st);
    for (int64_t t = 0; t + 1 < n; ++t) na_launch<true, true>(s, (int32_t)t, select, st);
    na_launch<true, false>(s, (int32_t)(n - 1), select, st);
    k_na_finish<<<1, 32, 0, st>>>(s, (int32_t)n);
    if (cudaGetLastError() != cudaSuccess) return fail(SNP_ERR_CUDA, "snp_step_noalloc launch failed");
    if (!steps_done) return SNP_OK;
    uint32_t fl[kNaFlagWords];
    unsigned long long sw[4];
    if (cudaMemcpyAsync(fl, scratch, sizeof(fl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(sw, scratch + kNaFlagWords, sizeof(sw), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaError_t e = cudaGetLastError();
        return fail(SNP_ERR_CUDA, std::string("snp_step_noalloc: ") + cudaGetErrorString(e));
    }
    *steps_done = (int64_t)sw[kNaExec];
    if (fl[kNaInvalid]) return fail(SNP_ERR_INVALID, "an index or a fired rule's field in the device arrays was out of range");
    if (fl[kNaOverflow]) return fail(SNP_ERR_OVERFLOW, "a spike count left the int32 range");
    return SNP_OK;
}
