// Grid-wide step kernels: one launch covers one step of one system.
//
// Pull form (SNP_FORM_OPT, SNP_PROP_PULL).  Each warp owns a slice of 32
// slots; lane l owns slot 32*slice + l.  One launch fuses the end of step k
// with the start of step k+1 (the paper's STEP of k, UPDATE_DELAYS, then
// SV_CALC of k+1, Alg. 1 and Sec. 5):
//   gather : C_{k+1}[j] = C'_k[j] + [j open] * sum_{i in in(j)} E_k[i]
//   select : per neuron, complete / count down / pick a rule for step k+1,
//            consume, and write E_{k+1}, S_{k+1} and the status word.
// E is double-buffered by step parity, so one launch per step needs no
// grid-wide barrier; the kernel boundary is the barrier between the paper's
// "choose the spiking vector" and "update the configuration" phases.
//
// Push form (SNP_PROP_PUSH) follows Alg. 5's direction: a select launch, then
// every emitter adds p into each open target with atomics aggregated across
// the warp (lanes that hit the same target add once), the out-list's columns
// dealt to warps in equal runs so hub sources do not serialise a warp.
//
// Fixed point: a select pass raises a per-step activity word when any neuron
// is pending or selected.  A gather launch that finds its step's word clear
// marks the system halted; later launches of the call return at once.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "kernels.h"
#include "push_balanced.cuh"

namespace snp {

template <bool GATHER, bool SELECT, bool COMPACT, int SEL>
__global__ void __launch_bounds__(256) k_step_pull(DevSys s, int32_t t) {
    uint32_t* fl = s.flags;
    const unsigned long long base = s.step[kStepBase];
    const unsigned long long kg = base + (unsigned long long)t;
    const unsigned long long ks = GATHER ? kg + 1ull : kg;
    if (GATHER) {
        if (step_blocked(fl, s.step, kg)) return;
        if (SELECT && blockIdx.x == 0 && threadIdx.x == 0) fl[kFlagAct0 + (int)((kg + 2ull) % 3ull)] = 0u;
    }
    const int lane = threadIdx.x & 31;
    const int32_t slice = (int32_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int32_t slot = slice * kSlice + lane;
    bool active = false;
    if (slice < s.nslices) {
        const bool valid = slot < s.q;
        int32_t c = 0;
        uint32_t st = 0u;
        if (valid) {
            c = s.C[slot];
            st = s.st[slot];
        }
        if (GATHER) {
            const int32_t* __restrict__ E = SNP_PICK(s.E, kg);
            const int32_t b = __ldg(s.slice_ptr + slice);
            const int32_t w = __ldg(s.slice_ptr + slice + 1) - b;
            const int32_t* __restrict__ p = s.in_idx + (size_t)b * kSlice + lane;
            long long sum = 0;
            int32_t col = 0;
            for (; col + 4 <= w; col += 4) {
                const int32_t i0 = __ldg(p + (col + 0) * kSlice);
                const int32_t i1 = __ldg(p + (col + 1) * kSlice);
                const int32_t i2 = __ldg(p + (col + 2) * kSlice);
                const int32_t i3 = __ldg(p + (col + 3) * kSlice);
                sum += (long long)E[SNP_IDX(fl, 0, i0, s.q + 1)] + E[SNP_IDX(fl, 0, i1, s.q + 1)] +
                       E[SNP_IDX(fl, 0, i2, s.q + 1)] + E[SNP_IDX(fl, 0, i3, s.q + 1)];
            }
            for (; col < w; ++col) sum += E[SNP_IDX(fl, 0, __ldg(p + col * kSlice), s.q + 1)];
            if (valid && (st >> kPendShift) == 0u) {
                long long nc = (long long)c + sum;
                if (nc > 2147483647ll) {
                    atomicOr(fl + kFlagOverflow, 1u);
                    nc = 2147483647ll;
                }
                c = (int32_t)nc;
            }
        }
        if (SELECT && valid) {
            const SelOut o = select_slot<COMPACT, SEL>(s, slot, c, st, ks);
            c = o.c_after;
            active = o.active;
            SNP_PICK(s.E, ks)[slot] = o.emit;
            SNP_PICK(s.S, ks)[slot] = o.s;
            if (o.st != st) s.st[slot] = o.st;
        }
        if (valid) s.C[slot] = c;
    }
    if (SELECT) raise_step_activity(fl, ks, active);
}

// Push propagation of step kg = base + t: select already ran for kg.  The
// optimized form's out-lists (Sy_Pi as sliced ELL by source, pad -1); each
// warp takes an equal run of their columns (push_balanced.cuh).
struct PushOptSrc {
    using Ent = int32_t;
    const int32_t* E;
    int32_t q;
    __device__ __forceinline__ Ent pad() const { return -1; }
    __device__ __forceinline__ int32_t value(int32_t slice, int lane) const {
        const int32_t slot = slice * kSlice + lane;
        return slot < q ? E[slot] : 0;
    }
    __device__ __forceinline__ int32_t target(Ent e) const { return e; }
    __device__ __forceinline__ int32_t amount(Ent, int32_t v) const { return v; }
};

constexpr int kPushBlocksPerSm = 8;

__global__ void __launch_bounds__(256, kPushBlocksPerSm) k_push_scatter(DevSys s, int32_t t) {
    uint32_t* fl = s.flags;
    const unsigned long long kg = s.step[kStepBase] + (unsigned long long)t;
    if (step_blocked(fl, s.step, kg)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) fl[kFlagAct0 + (int)((kg + 1ull) % 3ull)] = 0u;
    PushOptSrc src;
    src.E = SNP_PICK(s.E, kg);
    src.q = s.q;
    push_scatter_balanced<8>(src, s.out_ptr, s.nslices, s.out_idx, s.C, s.st, fl, s.q);
}

// Select-only launch for the push form: step kg = base + t.
template <bool COMPACT, int SEL>
__global__ void __launch_bounds__(256) k_select_push(DevSys s, int32_t t) {
    uint32_t* fl = s.flags;
    const unsigned long long ks = s.step[kStepBase] + (unsigned long long)t;
    if (call_halted(fl)) return;
    const int lane = threadIdx.x & 31;
    const int32_t slice = (int32_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int32_t slot = slice * kSlice + lane;
    bool active = false;
    if (slice < s.nslices && slot < s.q) {
        const SelOut o = select_slot<COMPACT, SEL>(s, slot, s.C[slot], s.st[slot], ks);
        active = o.active;
        s.C[slot] = o.c_after;
        SNP_PICK(s.E, ks)[slot] = o.emit;
        SNP_PICK(s.S, ks)[slot] = o.s;
        s.st[slot] = o.st;
    }
    raise_step_activity(fl, ks, active);
}

// Call bookkeeping: remember where the call started and clear its flags.
__global__ void k_begin(DevSys s) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        uint32_t* fl = s.flags;
        fl[kFlagAct0 + 0] = 0u;
        fl[kFlagAct0 + 1] = 0u;
        fl[kFlagAct0 + 2] = 0u;
        fl[kFlagHalted] = 0u;
        s.step[kStepHalt] = 0ull;
        s.step[kStepCallStart] = s.step[kStepBase];
    }
}

// Advances the base step after `count` launched steps unless the call halted.
__global__ void k_advance(DevSys s, int32_t count) {
    if (threadIdx.x == 0 && blockIdx.x == 0 && !ld_volatile(s.flags + kFlagHalted))
        s.step[kStepBase] += (unsigned long long)count;
}

// Ends a call: settles the base step at the halt point if the call halted
// and records the executed step count of the call.
__global__ void k_finish(DevSys s, int32_t tail) {
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        uint32_t* fl = s.flags;
        if (ld_volatile(fl + kFlagHalted))
            s.step[kStepBase] = s.step[kStepHalt];
        else
            s.step[kStepBase] += (unsigned long long)tail;
        s.step[kStepExec] = s.step[kStepBase] - s.step[kStepCallStart];
    }
}

// ---- host launchers -------------------------------------------------------

static inline dim3 grid_for(const DevSys& s, int threads) {
    const long long warps = s.nslices;
    const long long wpb = threads / 32;
    return dim3((unsigned)((warps + wpb - 1) / wpb));
}

template <bool G, bool S>
static cudaError_t launch_pull_t(const DevSys& s, int32_t t, cudaStream_t st, bool compact, int sel) {
    const dim3 grid = grid_for(s, 256);
    if (compact) {
        if (sel == SNP_SELECT_FIRST)
            k_step_pull<G, S, true, SNP_SELECT_FIRST><<<grid, 256, 0, st>>>(s, t);
        else
            k_step_pull<G, S, true, SNP_SELECT_PHILOX><<<grid, 256, 0, st>>>(s, t);
    } else {
        if (sel == SNP_SELECT_FIRST)
            k_step_pull<G, S, false, SNP_SELECT_FIRST><<<grid, 256, 0, st>>>(s, t);
        else
            k_step_pull<G, S, false, SNP_SELECT_PHILOX><<<grid, 256, 0, st>>>(s, t);
    }
    return cudaGetLastError();
}

cudaError_t launch_pull(const DevSys& s, int kind, int32_t t, cudaStream_t st, bool compact, int sel) {
    switch (kind) {
        case kPullSelectOnly: return launch_pull_t<false, true>(s, t, st, compact, sel);
        case kPullFused: return launch_pull_t<true, true>(s, t, st, compact, sel);
        case kPullGatherOnly: return launch_pull_t<true, false>(s, t, st, compact, sel);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_push_step(const DevSys& s, int32_t t, cudaStream_t st, bool compact, int sel) {
    const dim3 grid = grid_for(s, 256);
    if (compact) {
        if (sel == SNP_SELECT_FIRST)
            k_select_push<true, SNP_SELECT_FIRST><<<grid, 256, 0, st>>>(s, t);
        else
            k_select_push<true, SNP_SELECT_PHILOX><<<grid, 256, 0, st>>>(s, t);
    } else {
        if (sel == SNP_SELECT_FIRST)
            k_select_push<false, SNP_SELECT_FIRST><<<grid, 256, 0, st>>>(s, t);
        else
            k_select_push<false, SNP_SELECT_PHILOX><<<grid, 256, 0, st>>>(s, t);
    }
    k_push_scatter<<<push_blocks(kPushBlocksPerSm, s.nslices), 256, 0, st>>>(s, t);
    return cudaGetLastError();
}

cudaError_t launch_begin(const DevSys& s, cudaStream_t st) {
    k_begin<<<1, 32, 0, st>>>(s);
    return cudaGetLastError();
}
cudaError_t launch_advance(const DevSys& s, int32_t count, cudaStream_t st) {
    k_advance<<<1, 32, 0, st>>>(s, count);
    return cudaGetLastError();
}
cudaError_t launch_finish(const DevSys& s, int32_t tail, cudaStream_t st) {
    k_finish<<<1, 32, 0, st>>>(s, tail);
    return cudaGetLastError();
}

// ---- state export / import ------------------------------------------------

__global__ void k_export(const DevSys s, const int32_t* __restrict__ rule_base, int what, int32_t* out,
                         int parity, int compact) {
    const int32_t slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= s.q) return;
    const int32_t nid = s.orig[slot];
    int32_t v = 0;
    const uint32_t st = s.st[slot];
    switch (what) {
        case kExportConfig: v = s.C[slot]; break;
        case kExportStatus: v = (st >> kPendShift) ? (int32_t)(st & kDMask) : 0; break;
        case kExportPending: v = (st >> kPendShift) ? rule_base[slot] + (int32_t)(st >> kPendShift) - 1 : -1; break;
        case kExportSpiking: {
            // S of the last executed step k-1 (parity < 0: read k on the device)
            const unsigned long long k = s.step[kStepBase];
            const int par = parity >= 0 ? parity : (int)((k + 1ull) & 1ull);
            const int32_t x = (parity < 0 && k == 0ull) ? -1 : SNP_PICK(s.S, par)[slot];
            v = x >= 0 ? rule_base[slot] + x : -1;
            break;
        }
        case kExportChoices: v = compact ? choices_of<true>(s, slot) : choices_of<false>(s, slot); break;
    }
    out[nid] = v;
}

// State import: the caller's C, D, P (neuron order, on the device) checked
// neuron by neuron with the ranges snp_set_state documents, then written in
// slot order (spikes, and the status word: 1 + local pending rule above D).
template <bool COMMIT>
__global__ void k_import(DevSys s, const int32_t* __restrict__ rule_base, const int32_t* __restrict__ C,
                         const int32_t* __restrict__ D, const int32_t* __restrict__ P) {
    const int32_t slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= s.q) return;
    const uint32_t i = neuron_id(s, slot);
    const int32_t c = C[i], d = D[i], p = P[i];
    const int32_t r0 = rule_base[slot];
    if (!COMMIT) {
        bool ok = c >= 0 && d >= 0 && d <= kMaxDelay;
        if (p == -1)
            ok = ok && d == 0;
        else
            ok = ok && p >= r0 && p - r0 < rule_hi(s, slot) - rule_lo(s, slot);
        if (!ok) atomicMin(s.flags + kFlagImport, i);
        return;
    }
    s.C[slot] = c;
    s.st[slot] = p == -1 ? 0u : ((uint32_t)(p - r0 + 1) << kPendShift) | (uint32_t)d;
}

cudaError_t launch_import(const DevSys& s, const int32_t* rule_base, const int32_t* C, const int32_t* D,
                          const int32_t* P, bool commit, cudaStream_t st) {
    if (s.q == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((s.q + 255) / 256);
    if (commit)
        k_import<true><<<grid, 256, 0, st>>>(s, rule_base, C, D, P);
    else
        k_import<false><<<grid, 256, 0, st>>>(s, rule_base, C, D, P);
    return cudaGetLastError();
}

cudaError_t launch_export(const DevSys& s, const int32_t* rule_base, int what, int32_t* out, int parity,
                          cudaStream_t st, bool compact) {
    if (s.q == 0) return cudaSuccess;
    k_export<<<(s.q + 255) / 256, 256, 0, st>>>(s, rule_base, what, out, parity, compact ? 1 : 0);
    return cudaGetLastError();
}

}  // namespace snp
