// CTA-resident engine: one CTA owns one whole system and runs all its steps.
//
// Used for the batched form (thousands of independent systems in one
// persistent launch, each CTA taking the next system from a device work
// counter, largest first) and for single systems small enough that their
// emission vector fits in shared memory.
//
// Per step and system the CTA makes one pass over its slices (one warp per
// slice, one lane per neuron) that gathers step k and selects step k+1, the
// same fusion as the grid-wide engine.  The emission vectors E_k and E_{k+1}
// live in shared memory, bit-packed at e_bits per neuron, so the random
// in-neighbour reads of the gather never leave the SM.  __syncthreads_or at
// the end of a pass is both the barrier between steps and the fixed-point
// test (Alg. 1 stop condition).
#include <cuda_runtime.h>

#include <algorithm>

#include "device_common.cuh"
#include "kernels.h"

namespace snp {

// Occupancy of the resident kernel.  The kernel is bound by the latency of
// its global loads (a warp per slice, one dependent chain per slice), so
// resident warps matter most: 2 CTAs of up to 1,024 threads per SM hold it
// to 32 registers (64 warps per SM; a few spilled values stay in L1), where
// the unbounded form used 64 registers and fit 32 warps.  CTAs of 1,024
// threads stay available because a batch's largest systems run one CTA each
// and set its critical path: capping CTAs at 512 threads (40 registers, 48
// warps) matched this on 8,192 systems but lost 40% on 1,024.
constexpr int kResMaxThreads = 1024;
constexpr int kResMinBlocks = 2;

template <int EB>
__device__ __forceinline__ int32_t e_get(const uint32_t* __restrict__ e, int32_t i) {
    if (EB == 32) return (int32_t)e[i];
    constexpr uint32_t mask = (1u << EB) - 1u;
    const uint32_t bit = (uint32_t)i * EB;
    return (int32_t)((e[bit >> 5] >> (bit & 31u)) & mask);
}

// All 32 lanes call this for one slice; lane l contributes slot 32*slice+l.
template <int EB>
__device__ __forceinline__ void e_put_slice(uint32_t* e, int32_t slice, int lane, int32_t v) {
    if (EB == 32) {
        e[slice * 32 + lane] = (uint32_t)v;
        return;
    }
    constexpr int per = 32 / EB;  // neurons per word
    uint32_t w = ((uint32_t)v) << ((lane % per) * EB);
#pragma unroll
    for (int off = 1; off < per; off <<= 1) w |= __shfl_xor_sync(0xffffffffu, w, off);
    if (lane % per == 0) e[slice * EB + lane / per] = w;
}

template <bool COMPACT, int SEL, int EB>
__device__ void run_resident(const DevSys& s, long long n, uint32_t* esm) {
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int words = (int)(((long long)(s.nslices * 32 + 32) * EB + 31) / 32);
    uint32_t* Eb[2] = {esm, esm + words};
    for (int i = threadIdx.x; i < 2 * words; i += blockDim.x) esm[i] = 0u;
    const unsigned long long base = s.step[kStepBase];
    __syncthreads();

    // select pass for step `base`
    bool act = false;
    for (int32_t slice = warp; slice < s.nslices; slice += nwarps) {
        const int32_t slot = slice * kSlice + lane;
        int32_t emit = 0;
        if (slot < s.q) {
            const SelOut o = select_slot<COMPACT, SEL>(s, slot, s.C[slot], s.st[slot], base);
            s.C[slot] = o.c_after;
            s.st[slot] = o.st;
            SNP_PICK(s.S, base)[slot] = o.s;
            emit = o.emit;
            act |= o.active;
        }
        e_put_slice<EB>(SNP_PICK(Eb, base), slice, lane, emit);
    }
    bool any = __syncthreads_or(act);

    long long exec = 0;
    bool halted = false;
    for (long long t = 0; t < n; ++t) {
        if (!any) {
            halted = true;
            break;
        }
        const unsigned long long kg = base + (unsigned long long)t;
        const bool do_sel = (t + 1) < n;
        const uint32_t* __restrict__ Ek = SNP_PICK(Eb, kg);
        uint32_t* En = SNP_PICK(Eb, kg + 1ull);
        act = false;
        for (int32_t slice = warp; slice < s.nslices; slice += nwarps) {
            const int32_t slot = slice * kSlice + lane;
            const bool valid = slot < s.q;
            int32_t c = 0;
            uint32_t st = 0u;
            if (valid) {
                c = s.C[slot];
                st = s.st[slot];
            }
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
                const int32_t lim = s.nslices * 32 + 32;  // the packed vector's entries
                sum += (long long)e_get<EB>(Ek, SNP_IDX(s.flags, 0, i0, lim)) +
                       e_get<EB>(Ek, SNP_IDX(s.flags, 0, i1, lim)) + e_get<EB>(Ek, SNP_IDX(s.flags, 0, i2, lim)) +
                       e_get<EB>(Ek, SNP_IDX(s.flags, 0, i3, lim));
            }
            for (; col < w; ++col)
                sum += e_get<EB>(Ek, SNP_IDX(s.flags, 0, __ldg(p + col * kSlice), s.nslices * 32 + 32));
            if (valid && (st >> kPendShift) == 0u) {
                long long nc = (long long)c + sum;
                if (nc > 2147483647ll) {
                    atomicOr(s.flags + kFlagOverflow, 1u);
                    nc = 2147483647ll;
                }
                c = (int32_t)nc;
            }
            int32_t emit = 0;
            if (do_sel && valid) {
                const SelOut o = select_slot<COMPACT, SEL>(s, slot, c, st, kg + 1ull);
                c = o.c_after;
                s.st[slot] = o.st;
                SNP_PICK(s.S, kg + 1ull)[slot] = o.s;
                emit = o.emit;
                act |= o.active;
            }
            if (valid) s.C[slot] = c;
            if (do_sel) e_put_slice<EB>(En, slice, lane, emit);
        }
        ++exec;
        any = __syncthreads_or(act);
    }
    if (threadIdx.x == 0) {
        s.step[kStepCallStart] = base;
        s.step[kStepBase] = base + (unsigned long long)exec;
        s.step[kStepExec] = (unsigned long long)exec;
        s.step[kStepHalt] = halted ? base + (unsigned long long)exec : 0ull;
        s.flags[kFlagHalted] = halted ? 1u : 0u;
    }
}

// BIG: the instance for a batch's largest systems, one 1,024-thread CTA per
// SM with up to 64 registers (no spills on their long critical path).
template <bool COMPACT, int SEL, int EB, bool BIG>
__global__ void __launch_bounds__(kResMaxThreads, BIG ? 1 : kResMinBlocks)
    k_resident(const DevSys* __restrict__ systems, const long long* __restrict__ nsteps, int nsys,
               unsigned int* work) {
    extern __shared__ uint32_t esm[];
    __shared__ int s_id;
    for (;;) {
        if (threadIdx.x == 0) s_id = (int)atomicAdd(work, 1u);
        __syncthreads();
        const int id = s_id;
        if (id >= nsys) return;
        const DevSys s = systems[id];
        run_resident<COMPACT, SEL, EB>(s, nsteps[id], esm);
        __syncthreads();
    }
}

// Per-system results of a batch launch: base step, executed steps, overflow.
__global__ void k_gather_results(const DevSys* __restrict__ systems, int nsys, unsigned long long* out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= nsys) return;
    const DevSys& s = systems[r];
    out[3 * r + 0] = s.step[kStepBase];
    out[3 * r + 1] = s.step[kStepExec];
    out[3 * r + 2] = (s.flags[kFlagOverflow] ? 1u : 0u) | (s.flags[kFlagBounds] ? 2u : 0u);
}

cudaError_t launch_gather_results(const DevSys* d_systems, int nsys, unsigned long long* d_out, cudaStream_t st) {
    if (nsys <= 0) return cudaSuccess;
    k_gather_results<<<(nsys + 255) / 256, 256, 0, st>>>(d_systems, nsys, d_out);
    return cudaGetLastError();
}

// ---- batched forced steps (computation-tree exploration) -----------------
// One forced step of each of nb configurations of one system, one CTA per
// configuration at a time.  Branch b reads C0/D0/P0 and its choice indices
// at offset b*q in the caller's neuron order (D = steps until the neuron
// reopens, P = global id of its pending rule or -1) and writes C1/D1/P1 and
// executed[b] = 1, or 0 at a fixed point (the configuration is copied), and
// bad[b] = 1 when a choice index was out of range (that neuron took its
// first rule).  Phase 1 selects every neuron (select_forced_idx) into
// shared memory and packs the emissions; phase 2 gathers the in-lists
// against them and finishes the step, as run_resident does.
template <bool COMPACT, int EB>
__global__ void __launch_bounds__(256) k_branch_step(DevSys s, const int32_t* __restrict__ rule_base, int nb,
                                                     const int32_t* __restrict__ C0, const int32_t* __restrict__ D0,
                                                     const int32_t* __restrict__ P0, const int32_t* __restrict__ ch,
                                                     int32_t* C1, int32_t* D1, int32_t* P1, int32_t* executed,
                                                     int32_t* bad, int32_t* counts) {
    extern __shared__ uint32_t sm[];
    __shared__ int s_bad;
    const int words = (int)(((long long)(s.nslices * 32 + 32) * EB + 31) / 32);
    uint32_t* Esm = sm;
    int32_t* csm = reinterpret_cast<int32_t*>(sm + words);  // c after the selection
    uint32_t* ssm = reinterpret_cast<uint32_t*>(csm + s.nslices * 32);  // status after the selection
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    // the words past the last slice stay zero (slot q, the in-lists' pad, emits 0)
    for (int i = s.nslices * EB + threadIdx.x; i < words; i += blockDim.x) Esm[i] = 0u;
    for (int b = blockIdx.x; b < nb; b += gridDim.x) {
        const size_t off = (size_t)b * s.q;
        if (threadIdx.x == 0) s_bad = 0;
        __syncthreads();
        bool act = false, badl = false;
        for (int32_t sl = warp; sl < s.nslices; sl += nw) {
            const int32_t slot = sl * kSlice + lane;
            int32_t emit = 0;
            if (slot < s.q) {
                const int32_t nid = (int32_t)neuron_id(s, slot);
                const int32_t c = C0[off + nid], d = D0[off + nid], p = P0[off + nid];
                const uint32_t st = p >= 0 ? ((uint32_t)(p - rule_base[slot] + 1) << kPendShift) | (uint32_t)d : 0u;
                const SelOut o = select_forced_idx<COMPACT>(s, slot, c, st, ch[off + nid], badl);
                csm[slot] = o.c_after;
                ssm[slot] = o.st;
                emit = o.emit;
                act |= o.active;
            }
            e_put_slice<EB>(Esm, sl, lane, emit);
        }
        if (badl) s_bad = 1;
        const bool any = __syncthreads_or(act);
        for (int32_t sl = warp; sl < s.nslices; sl += nw) {
            const int32_t slot = sl * kSlice + lane;
            long long in = 0;
            if (any) {
                const int32_t b0 = __ldg(s.slice_ptr + sl);
                const int32_t w = __ldg(s.slice_ptr + sl + 1) - b0;
                const int32_t* __restrict__ p = s.in_idx + (size_t)b0 * kSlice + lane;
                for (int32_t col = 0; col < w; ++col)
                    in += e_get<EB>(Esm, SNP_IDX(s.flags, 0, __ldg(p + col * kSlice), s.nslices * 32 + 32));
            }
            if (slot < s.q) {
                const int32_t nid = (int32_t)neuron_id(s, slot);
                if (!any) {  // a fixed point: the configuration does not change
                    C1[off + nid] = C0[off + nid];
                    D1[off + nid] = D0[off + nid];
                    P1[off + nid] = P0[off + nid];
                    if (counts) counts[off + nid] = 0;
                    continue;
                }
                const uint32_t st = ssm[slot];
                long long c = csm[slot];
                if ((st >> kPendShift) == 0u) c += in;
                if (c > 2147483647ll) {
                    atomicOr(s.flags + kFlagOverflow, 1u);
                    c = 2147483647ll;
                }
                const uint32_t pend = st >> kPendShift;
                C1[off + nid] = (int32_t)c;
                D1[off + nid] = pend ? (int32_t)(st & kDMask) : 0;
                P1[off + nid] = pend ? rule_base[slot] + (int32_t)pend - 1 : -1;
                if (counts)  // the choices of the new configuration (its next level)
                    counts[off + nid] =
                        pend ? 0 : count_applicable_slot<COMPACT>(s, slot, (int32_t)c);
            }
        }
        if (threadIdx.x == 0) {
            executed[b] = any ? 1 : 0;
            bad[b] = s_bad;
        }
        __syncthreads();  // the next configuration reuses the shared memory
    }
}

// Input check of snp_branch_step, run before k_branch_step reads anything:
// configuration b's neuron i (caller's order, at b*q + i) must hold C >= 0,
// 0 <= D <= 65535, P = -1 or one of neuron i's rules, and D > 0 only with a
// pending rule -- the rules snp_set_state's import applies.  The smallest
// offending index b*q + i goes to *first_bad (set to ~0 by the caller).
// Every array read here is in range for any values of C, D and P.
__global__ void k_branch_check(DevSys s, const int32_t* __restrict__ rule_base, long long total,
                               const int32_t* __restrict__ C0, const int32_t* __restrict__ D0,
                               const int32_t* __restrict__ P0, unsigned long long* first_bad) {
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
        const long long b = idx / s.q;
        const int32_t slot = (int32_t)(idx - b * s.q);
        const unsigned long long at = (unsigned long long)b * (unsigned long long)s.q + neuron_id(s, slot);
        const int32_t c = C0[at], d = D0[at], p = P0[at];
        const int32_t r0 = rule_base[slot];
        bool ok = c >= 0 && d >= 0 && d <= kMaxDelay;
        if (p == -1)
            ok = ok && d == 0;
        else
            ok = ok && p >= r0 && p - r0 < rule_hi(s, slot) - rule_lo(s, slot);
        if (!ok) atomicMin(first_bad, at);
    }
}

cudaError_t launch_branch_check(const DevSys& s, const int32_t* rule_base, int nb, const int32_t* C0,
                                const int32_t* D0, const int32_t* P0, unsigned long long* first_bad,
                                cudaStream_t st) {
    const long long total = (long long)nb * s.q;
    if (total <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (total + 255) / 256;
    const int grid = (int)std::max(1ll, std::min<long long>(want, (long long)std::max(1, sms) * 8));
    k_branch_check<<<grid, 256, 0, st>>>(s, rule_base, total, C0, D0, P0, first_bad);
    return cudaGetLastError();
}

size_t branch_smem_bytes(int q, int e_bits) {
    const long long nslices = ((long long)q + 31) / 32;
    const long long words = ((nslices * 32 + 32) * e_bits + 31) / 32;
    return (size_t)(words * 4 + nslices * 32 * 8);
}

template <bool C, int EB>
static cudaError_t launch_branch_t(const DevSys& s, const int32_t* rule_base, int nb, const int32_t* C0,
                                   const int32_t* D0, const int32_t* P0, const int32_t* ch, int32_t* C1, int32_t* D1,
                                   int32_t* P1, int32_t* ex, int32_t* bad, int32_t* counts, cudaStream_t st) {
    auto fn = k_branch_step<C, EB>;
    const size_t smem = branch_smem_bytes(s.q, EB);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = std::max(1, std::min(nb, sms * 8));
    fn<<<grid, 256, smem, st>>>(s, rule_base, nb, C0, D0, P0, ch, C1, D1, P1, ex, bad, counts);
    return cudaGetLastError();
}

cudaError_t launch_branch_step(const DevSys& s, const int32_t* rule_base, int e_bits, bool compact, int nb,
                               const int32_t* C0, const int32_t* D0, const int32_t* P0, const int32_t* ch,
                               int32_t* C1, int32_t* D1, int32_t* P1, int32_t* ex, int32_t* bad, int32_t* counts,
                               cudaStream_t st) {
#define SNP_BR(CC, EE) \
    return launch_branch_t<CC, EE>(s, rule_base, nb, C0, D0, P0, ch, C1, D1, P1, ex, bad, counts, st)
    if (compact) {
        if (e_bits == 2) SNP_BR(true, 2);
        if (e_bits == 4) SNP_BR(true, 4);
        if (e_bits == 8) SNP_BR(true, 8);
        SNP_BR(true, 16);
    }
    if (e_bits == 2) SNP_BR(false, 2);
    if (e_bits == 4) SNP_BR(false, 4);
    if (e_bits == 8) SNP_BR(false, 8);
    SNP_BR(false, 16);
#undef SNP_BR
}

int resident_e_bits(int max_p) {
    if (max_p < 4) return 2;
    if (max_p < 16) return 4;
    if (max_p < 256) return 8;
    return 16;
}

size_t resident_smem_bytes(int max_q, int e_bits) {
    const long long nslices = ((long long)max_q + 31) / 32;
    const long long words = ((nslices * 32 + 32) * e_bits + 31) / 32;
    return (size_t)(2 * words * 4);
}

int resident_max_smem() {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    return v;
}

template <bool C, int S, int EB>
static cudaError_t launch_res_t(const DevSys* d_systems, const long long* d_nsteps, int nsys, unsigned int* d_work,
                                const ResidentPlan& plan, cudaStream_t st) {
    if (plan.big) {  // one 1,024-thread CTA per system, 64 registers
        auto fb = k_resident<C, S, EB, true>;
        cudaError_t e = cudaFuncSetAttribute(fb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem);
        if (e != cudaSuccess) return e;
        fb<<<nsys, kResMaxThreads, plan.smem, st>>>(d_systems, d_nsteps, nsys, d_work);
        return cudaGetLastError();
    }
    auto fn = k_resident<C, S, EB, false>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)plan.smem);
    if (e != cudaSuccess) return e;
    const int threads = plan.threads < kResMaxThreads ? plan.threads : kResMaxThreads;
    int ctas = plan.ctas;
    if (ctas > 1) {
        // persistent grid: exactly the CTAs that are resident at once
        // (registers, shared memory and threads all counted)
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, plan.smem) == cudaSuccess &&
            sms > 0 && per_sm > 0)
            ctas = sms * per_sm;
        else
            cudaGetLastError();
    }
    fn<<<ctas, threads, plan.smem, st>>>(d_systems, d_nsteps, nsys, d_work);
    return cudaGetLastError();
}

template <bool C, int S>
static cudaError_t launch_res_eb(const DevSys* d_systems, const long long* d_nsteps, int nsys, unsigned int* d_work,
                                 const ResidentPlan& plan, cudaStream_t st) {
    switch (plan.e_bits) {
        case 2: return launch_res_t<C, S, 2>(d_systems, d_nsteps, nsys, d_work, plan, st);
        case 4: return launch_res_t<C, S, 4>(d_systems, d_nsteps, nsys, d_work, plan, st);
        case 8: return launch_res_t<C, S, 8>(d_systems, d_nsteps, nsys, d_work, plan, st);
        case 16: return launch_res_t<C, S, 16>(d_systems, d_nsteps, nsys, d_work, plan, st);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_resident(const DevSys* d_systems, const long long* d_nsteps, int nsys, unsigned int* d_work,
                            const ResidentPlan& plan, bool compact, int sel, cudaStream_t st) {
    if (compact) {
        if (sel == SNP_SELECT_FIRST) return launch_res_eb<true, SNP_SELECT_FIRST>(d_systems, d_nsteps, nsys, d_work, plan, st);
        return launch_res_eb<true, SNP_SELECT_PHILOX>(d_systems, d_nsteps, nsys, d_work, plan, st);
    }
    if (sel == SNP_SELECT_FIRST) return launch_res_eb<false, SNP_SELECT_FIRST>(d_systems, d_nsteps, nsys, d_work, plan, st);
    return launch_res_eb<false, SNP_SELECT_PHILOX>(d_systems, d_nsteps, nsys, d_work, plan, st);
}

}  // namespace snp
