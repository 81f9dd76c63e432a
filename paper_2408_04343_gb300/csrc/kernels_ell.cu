// The ELL form and the uncompressed ("Sparse") form of the transition matrix.
//
// Both forms keep the paper's per-rule view: the spiking vector has one entry
// per rule (Sec. 2: S_k of length m), and spikes travel as (rule, value)
// pairs.  Em_k[r] = 1 when rule r emits at step k (it fired with d = 0, or
// its delay ran out), stored as bytes, double-buffered by step parity.
//
//  * ELL pull: each target neuron sums Em_k[r] * p over the (rule, p) pairs
//    of its in-ELL column (the transpose of M^s_Pi's +p rows, Sec. 4);
//  * ELL push: each emitting rule walks its column of M^s_Pi and adds p into
//    every open target with warp-aggregated atomics (Alg. 4's direction),
//    the columns dealt to warps in equal runs (push_balanced.cuh);
//  * dense: each neuron walks its column of M_Pi over all m rules and adds
//    Em_k[r] * M[r, j] (Alg. 3's direction); the (row block x neuron tile)
//    partial sums meet in an in-flow vector, and the select launch applies it.
// Consumption (-c) is applied when a rule is selected (the pair in row 0 of
// M^s_Pi is not walked): with delays a rule consumes at t and emits at t+d.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "kernels.h"
#include "push_balanced.cuh"

namespace snp {

// Select for step ks on one slot, writing the per-rule emission bytes.
template <bool COMPACT, int SEL>
__device__ __forceinline__ bool ell_select_slot(const DevSys& s, const EllSys& e, int32_t slot, int32_t& c,
                                                unsigned long long ks) {
    const uint32_t st = s.st[slot];
    const int32_t r0 = rule_lo(s, slot), r1 = rule_hi(s, slot);
    const SelOut o = select_slot<COMPACT, SEL>(s, slot, c, st, ks);
    int32_t emitting = -1;  // local index of the rule that emits at ks
    if ((st >> kPendShift) != 0u && (st & kDMask) == 0u) emitting = (int32_t)(st >> kPendShift) - 1;
    else if (o.s >= 0 && o.emit > 0) emitting = o.s;
    uint8_t* Em = SNP_PICK(e.Em, ks);
    for (int32_t r = r0; r < r1; ++r) Em[r] = (r - r0) == emitting ? 1 : 0;
    c = o.c_after;
    SNP_PICK(s.S, ks)[slot] = o.s;
    s.st[slot] = o.st;
    return o.active;
}

// ELL pull: gather of step kg (+ select of kg+1), like k_step_pull.
template <bool GATHER, bool SELECT, bool COMPACT, int SEL>
__global__ void __launch_bounds__(256) k_ell_pull(DevSys s, EllSys e, int32_t t) {
    uint32_t* fl = s.flags;
    const unsigned long long kg = s.step[kStepBase] + (unsigned long long)t;
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
        int32_t c = valid ? s.C[slot] : 0;
        if (GATHER) {
            const uint8_t* __restrict__ Em = SNP_PICK(e.Em, kg);
            const int32_t b = __ldg(e.in_ptr + slice);
            const int32_t w = __ldg(e.in_ptr + slice + 1) - b;
            const int2* __restrict__ p = e.in_ent + (size_t)b * kSlice + lane;
            long long sum = 0;
            int32_t col = 0;
            for (; col + 4 <= w; col += 4) {
                const int2 a0 = __ldg(p + (col + 0) * kSlice), a1 = __ldg(p + (col + 1) * kSlice);
                const int2 a2 = __ldg(p + (col + 2) * kSlice), a3 = __ldg(p + (col + 3) * kSlice);
                sum += (Em[SNP_IDX(fl, 4, a0.x, e.m + 1)] ? a0.y : 0) + (Em[SNP_IDX(fl, 4, a1.x, e.m + 1)] ? a1.y : 0) +
                       (Em[SNP_IDX(fl, 4, a2.x, e.m + 1)] ? a2.y : 0) + (Em[SNP_IDX(fl, 4, a3.x, e.m + 1)] ? a3.y : 0);
            }
            for (; col < w; ++col) {
                const int2 a = __ldg(p + col * kSlice);
                sum += Em[SNP_IDX(fl, 4, a.x, e.m + 1)] ? a.y : 0;
            }
            if (valid && (s.st[slot] >> kPendShift) == 0u) {
                long long nc = (long long)c + sum;
                if (nc > 2147483647ll) {
                    atomicOr(fl + kFlagOverflow, 1u);
                    nc = 2147483647ll;
                }
                c = (int32_t)nc;
            }
        }
        if (SELECT && valid) active = ell_select_slot<COMPACT, SEL>(s, e, slot, c, ks);
        if (valid) s.C[slot] = c;
    }
    if (SELECT) raise_step_activity(fl, ks, active);
}

// Select launch of step ks = base + t for the push and dense variants.  With
// INFLOW it first finishes step ks - 1 by adding the in-flow accumulated by
// the dense launch (to open neurons) and clears it; with !SELECT it only
// finishes.
template <bool INFLOW, bool SELECT, bool COMPACT, int SEL>
__global__ void __launch_bounds__(256) k_ell_select(DevSys s, EllSys e, int32_t t) {
    uint32_t* fl = s.flags;
    const unsigned long long ks = s.step[kStepBase] + (unsigned long long)t;
    if (call_halted(fl)) return;
    const int32_t slot = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x);
    bool active = false;
    if (slot < s.q) {
        int32_t c = s.C[slot];
        if (INFLOW) {
            const int32_t in = e.inflow[slot];
            e.inflow[slot] = 0;
            if ((s.st[slot] >> kPendShift) == 0u) {
                long long nc = (long long)c + in;
                if (nc > 2147483647ll) {
                    atomicOr(fl + kFlagOverflow, 1u);
                    nc = 2147483647ll;
                }
                c = (int32_t)nc;
            }
        }
        if (SELECT) active = ell_select_slot<COMPACT, SEL>(s, e, slot, c, ks);
        s.C[slot] = c;
    }
    if (SELECT) raise_step_activity(fl, ks, active);
}

// ELL push of step kg = base + t: per-rule columns of (target, p) pairs in
// slices of 32 consecutive rules; each warp takes an equal run of their
// columns (push_balanced.cuh).
struct PushEllSrc {
    using Ent = int2;
    const uint8_t* Em;
    int64_t m;
    __device__ __forceinline__ Ent pad() const { return make_int2(-1, 0); }
    __device__ __forceinline__ int32_t value(int32_t slice, int lane) const {
        const int64_t r = (int64_t)slice * kSlice + lane;
        return r < m && Em[r] ? 1 : 0;
    }
    __device__ __forceinline__ int32_t target(Ent e) const { return e.x; }
    __device__ __forceinline__ int32_t amount(Ent e, int32_t) const { return e.y; }
};

constexpr int kEllPushBlocksPerSm = 6;

__global__ void __launch_bounds__(256, kEllPushBlocksPerSm) k_ell_push(DevSys s, EllSys e, int32_t t) {
    uint32_t* fl = s.flags;
    const unsigned long long kg = s.step[kStepBase] + (unsigned long long)t;
    if (step_blocked(fl, s.step, kg)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) fl[kFlagAct0 + (int)((kg + 1ull) % 3ull)] = 0u;
    PushEllSrc src;
    src.Em = SNP_PICK(e.Em, kg);
    src.m = e.m;
    const int32_t nrs = (int32_t)((e.m + kSlice - 1) / kSlice);
    push_scatter_balanced<8>(src, e.out_ptr, nrs, e.out_ent, s.C, s.st, fl, s.q);
}

// Dense accumulation of step kg = base + t: CTA (bx, by) covers neurons
// [bx*256, bx*256+256) and rules [by*rows, (by+1)*rows); every rule row of
// M_Pi is read whether or not the rule emits, as Alg. 3 walks all m rules.
__global__ void __launch_bounds__(256) k_dense_accum(DevSys s, EllSys e, int32_t t, int32_t rows) {
    uint32_t* fl = s.flags;
    const unsigned long long kg = s.step[kStepBase] + (unsigned long long)t;
    if (step_blocked(fl, s.step, kg)) return;
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) fl[kFlagAct0 + (int)((kg + 2ull) % 3ull)] = 0u;
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.y * rows;
    const int64_t r1 = r0 + rows < e.m ? r0 + rows : e.m;
    const uint8_t* __restrict__ Em = SNP_PICK(e.Em, kg);
    if (j >= s.q) return;
    long long sum = 0;
    const int32_t* __restrict__ col = e.dense + j;
    for (int64_t r = r0; r < r1; ++r) sum += (long long)Em[r] * __ldg(col + r * (int64_t)s.q);
    if (sum) {
        const int old = atomicAdd(e.inflow + j, (int)sum);
        if ((long long)old + sum > 2147483647ll) atomicOr(fl + kFlagOverflow, 1u);
    }
}

// ---- launchers ----------------------------------------------------------

template <bool G, bool S>
static cudaError_t ell_pull_t(const DevSys& s, const EllSys& e, int32_t t, cudaStream_t st, bool compact, int sel) {
    const dim3 grid((unsigned)((s.nslices + 7) / 8));
    if (compact) {
        if (sel == SNP_SELECT_FIRST) k_ell_pull<G, S, true, SNP_SELECT_FIRST><<<grid, 256, 0, st>>>(s, e, t);
        else k_ell_pull<G, S, true, SNP_SELECT_PHILOX><<<grid, 256, 0, st>>>(s, e, t);
    } else {
        if (sel == SNP_SELECT_FIRST) k_ell_pull<G, S, false, SNP_SELECT_FIRST><<<grid, 256, 0, st>>>(s, e, t);
        else k_ell_pull<G, S, false, SNP_SELECT_PHILOX><<<grid, 256, 0, st>>>(s, e, t);
    }
    return cudaGetLastError();
}

cudaError_t launch_ell_pull(const DevSys& s, const EllSys& e, int kind, int32_t t, cudaStream_t st, bool compact,
                            int sel) {
    switch (kind) {
        case kPullSelectOnly: return ell_pull_t<false, true>(s, e, t, st, compact, sel);
        case kPullFused: return ell_pull_t<true, true>(s, e, t, st, compact, sel);
        case kPullGatherOnly: return ell_pull_t<true, false>(s, e, t, st, compact, sel);
        default: return cudaErrorInvalidValue;
    }
}

template <bool IN, bool S>
static cudaError_t ell_select_t(const DevSys& s, const EllSys& e, int32_t t, cudaStream_t st, bool compact, int sel) {
    const dim3 grid((unsigned)((s.q + 255) / 256));
    if (compact) {
        if (sel == SNP_SELECT_FIRST) k_ell_select<IN, S, true, SNP_SELECT_FIRST><<<grid, 256, 0, st>>>(s, e, t);
        else k_ell_select<IN, S, true, SNP_SELECT_PHILOX><<<grid, 256, 0, st>>>(s, e, t);
    } else {
        if (sel == SNP_SELECT_FIRST) k_ell_select<IN, S, false, SNP_SELECT_FIRST><<<grid, 256, 0, st>>>(s, e, t);
        else k_ell_select<IN, S, false, SNP_SELECT_PHILOX><<<grid, 256, 0, st>>>(s, e, t);
    }
    return cudaGetLastError();
}

cudaError_t launch_ell_select(const DevSys& s, const EllSys& e, bool inflow, bool select, int32_t t, cudaStream_t st,
                              bool compact, int sel) {
    if (inflow) return select ? ell_select_t<true, true>(s, e, t, st, compact, sel)
                              : ell_select_t<true, false>(s, e, t, st, compact, sel);
    return ell_select_t<false, true>(s, e, t, st, compact, sel);
}

cudaError_t launch_ell_push(const DevSys& s, const EllSys& e, int32_t t, cudaStream_t st) {
    const int64_t nrs = (e.m + kSlice - 1) / kSlice;
    if (nrs == 0) {
        k_ell_push<<<1, 32, 0, st>>>(s, e, t);  // still settles the halt test
        return cudaGetLastError();
    }
    k_ell_push<<<push_blocks(kEllPushBlocksPerSm, nrs), 256, 0, st>>>(s, e, t);
    return cudaGetLastError();
}

cudaError_t launch_dense_accum(const DevSys& s, const EllSys& e, int32_t t, cudaStream_t st) {
    const int32_t rows = 512;
    const unsigned gy = (unsigned)((e.m + rows - 1) / rows);
    const dim3 grid((unsigned)((s.q + 255) / 256), gy > 0 ? gy : 1u);
    k_dense_accum<<<grid, 256, 0, st>>>(s, e, t, rows);
    return cudaGetLastError();
}

}  // namespace snp
