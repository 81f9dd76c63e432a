// Tiled engine: grid-wide pull step with the emission vector in shared memory.
//
// Random reads of E_k are the cost of the pull step: each in-edge reads one
// neuron's emission, and on this part random 4-byte reads served by L2 or L1
// run near one distinct line per clock per SM, well below what HBM can feed
// the index stream.  Here E_k is bit-packed (2 bits per neuron when every p
// is at most 3) and every CTA copies it into its shared memory, one source
// partition at a time, so the gathers become shared-memory reads.
//
// A step is two launches:
//  * k_tiled_gather -- one CTA per SM, each owning a range of slices.  For
//    every partition h the CTA loads h's packed emissions and streams its
//    group of in-edge words edge-parallel (16-byte vector loads, no
//    per-neuron bookkeeping): each word names a local target slot and a
//    source, whose emission is added to the target's shared-memory
//    accumulator.  The accumulators become the in-flow vector of step k.
//  * k_tiled_select -- full occupancy, one warp per slice: finishes step k
//    (C_{k+1} = C' + [open] * in-flow), selects step k+1 and writes the
//    packed E_{k+1} that the next gather loads.
// Same status word, fixed-point test and activity words as k_step_pull.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "kernels.h"

namespace snp {

__device__ __forceinline__ uint4 ld_stream_v4(const uint4* p) {
    uint4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "l"(p));
    return v;
}

template <int EB>
__device__ __forceinline__ uint32_t pk_get(const uint32_t* __restrict__ e, uint32_t i) {
    constexpr uint32_t mask = (1u << EB) - 1u;
    const uint32_t bit = i * EB;
    return (e[bit >> 5] >> (bit & 31u)) & mask;
}

// All 32 lanes of a warp call this for one slice; lane l supplies slot 32*slice+l.
template <int EB>
__device__ __forceinline__ void pk_put_slice(uint32_t* e, int32_t slice, int lane, uint32_t v) {
    constexpr int per = 32 / EB;
    uint32_t w = v << ((lane % per) * EB);
#pragma unroll
    for (int off = 1; off < per; off <<= 1) w |= __shfl_xor_sync(0xffffffffu, w, off);
    if (lane % per == 0) e[slice * EB + lane / per] = w;
}

template <int EB>
__device__ __forceinline__ void edge(const uint32_t* __restrict__ Esm, int* acc, uint32_t w, uint32_t smask,
                                     int sbits) {
    const uint32_t v = pk_get<EB>(Esm, w & smask);
    if (v) atomicAdd(acc + (w >> sbits), (int)v);
}

// In-flow of step kg = base + t into tl.inflow.
template <int EB>
__global__ void __launch_bounds__(1024, 1) k_tiled_gather(DevSys s, TiledSys tl, int32_t t) {
    extern __shared__ uint32_t smem[];
    uint32_t* Esm = smem;
    int* acc = reinterpret_cast<int*>(smem + tl.part_words);
    uint32_t* fl = s.flags;
    const unsigned long long kg = s.step[kStepBase] + (unsigned long long)t;
    if (step_blocked(fl, s.step, kg)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) fl[kFlagAct0 + (int)((kg + 2ull) % 3ull)] = 0u;
    const int32_t lo = __ldg(tl.cta_lo + blockIdx.x), hi = __ldg(tl.cta_lo + blockIdx.x + 1);
    for (int i = threadIdx.x; i < tl.acc_words; i += blockDim.x) acc[i] = 0;
    const uint32_t* Eprev = SNP_PICK(tl.Eg, kg);
    const uint32_t smask = (tl.src_bits >= 32) ? 0xffffffffu : ((1u << tl.src_bits) - 1u);
    const int sbits = tl.src_bits;
    const uint4* ent = reinterpret_cast<const uint4*>(tl.ent);
    for (int h = 0; h < tl.P; ++h) {
        const uint4* src = reinterpret_cast<const uint4*>(Eprev + (size_t)h * tl.part_words);
        uint4* dst = reinterpret_cast<uint4*>(Esm);
        for (int i = threadIdx.x; i < tl.part_words / 4; i += blockDim.x) dst[i] = __ldcg(src + i);
        __syncthreads();
        const int64_t g = (int64_t)blockIdx.x * tl.P + h;
        const int32_t g0 = __ldg(tl.grp + g) / 4, g1 = __ldg(tl.grp + g + 1) / 4;
        const int32_t stride = blockDim.x;
        int32_t i = g0 + threadIdx.x;
        for (; i + 3 * stride < g1; i += 4 * stride) {
            const uint4 a = ld_stream_v4(ent + i);
            const uint4 b = ld_stream_v4(ent + i + stride);
            const uint4 c = ld_stream_v4(ent + i + 2 * stride);
            const uint4 d = ld_stream_v4(ent + i + 3 * stride);
            edge<EB>(Esm, acc, a.x, smask, sbits); edge<EB>(Esm, acc, a.y, smask, sbits);
            edge<EB>(Esm, acc, a.z, smask, sbits); edge<EB>(Esm, acc, a.w, smask, sbits);
            edge<EB>(Esm, acc, b.x, smask, sbits); edge<EB>(Esm, acc, b.y, smask, sbits);
            edge<EB>(Esm, acc, b.z, smask, sbits); edge<EB>(Esm, acc, b.w, smask, sbits);
            edge<EB>(Esm, acc, c.x, smask, sbits); edge<EB>(Esm, acc, c.y, smask, sbits);
            edge<EB>(Esm, acc, c.z, smask, sbits); edge<EB>(Esm, acc, c.w, smask, sbits);
            edge<EB>(Esm, acc, d.x, smask, sbits); edge<EB>(Esm, acc, d.y, smask, sbits);
            edge<EB>(Esm, acc, d.z, smask, sbits); edge<EB>(Esm, acc, d.w, smask, sbits);
        }
        for (; i < g1; i += stride) {
            const uint4 a = ld_stream_v4(ent + i);
            edge<EB>(Esm, acc, a.x, smask, sbits); edge<EB>(Esm, acc, a.y, smask, sbits);
            edge<EB>(Esm, acc, a.z, smask, sbits); edge<EB>(Esm, acc, a.w, smask, sbits);
        }
        __syncthreads();
    }
    const int32_t slot0 = lo * kSlice;
    const int32_t nloc = (hi - lo) * kSlice;
    for (int i = threadIdx.x; i < nloc; i += blockDim.x) tl.inflow[slot0 + i] = acc[i];
}

// Finishes step kg (GATHER: adds the in-flow to open neurons) and selects
// step ks (SELECT), one warp per slice.
template <bool GATHER, bool SELECT, bool COMPACT, int SEL, int EB>
__global__ void __launch_bounds__(256) k_tiled_select(DevSys s, TiledSys tl, int32_t t) {
    uint32_t* fl = s.flags;
    const unsigned long long kg = s.step[kStepBase] + (unsigned long long)t;
    const unsigned long long ks = GATHER ? kg + 1ull : kg;
    if (call_halted(fl)) return;
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
        if (GATHER && valid && (st >> kPendShift) == 0u) {
            const long long nc = (long long)c + tl.inflow[slot];
            if (nc > 2147483647ll) {
                atomicOr(fl + kFlagOverflow, 1u);
                c = 2147483647;
            } else {
                c = (int32_t)nc;
            }
        }
        uint32_t emit = 0u;
        if (SELECT && valid) {
            const SelOut o = select_neuron<COMPACT, SEL>(
                s.rules, rule_lo(s, slot), rule_hi(s, slot), c, st, ks,
                SEL == SNP_SELECT_PHILOX ? neuron_id(s, slot) : 0u, s.seed);
            c = o.c_after;
            active = o.active;
            emit = (uint32_t)o.emit;
            SNP_PICK(s.S, ks)[slot] = o.s;
            s.st[slot] = o.st;
        }
        if (valid) s.C[slot] = c;
        if (SELECT) pk_put_slice<EB>(SNP_PICK(tl.Eg, ks), slice, lane, emit);
    }
    if (SELECT) raise_step_activity(fl, ks, active);
}

template <int EB>
static cudaError_t launch_gather_eb(const DevSys& s, const TiledSys& tl, int32_t t, cudaStream_t st, size_t smem,
                                    int threads) {
    auto fn = k_tiled_gather<EB>;
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    fn<<<tl.G, threads, smem, st>>>(s, tl, t);
    return cudaGetLastError();
}

template <bool G, bool S, bool C, int SEL, int EB>
static cudaError_t launch_select_t(const DevSys& s, const TiledSys& tl, int32_t t, cudaStream_t st) {
    const dim3 grid((unsigned)((s.nslices + 7) / 8));
    k_tiled_select<G, S, C, SEL, EB><<<grid, 256, 0, st>>>(s, tl, t);
    return cudaGetLastError();
}

template <int EB>
static cudaError_t launch_tiled_eb(const DevSys& s, const TiledSys& tl, int kind, int32_t t, cudaStream_t st,
                                   bool compact, int sel, size_t smem, int threads) {
    cudaError_t e = cudaSuccess;
    if (kind != kPullSelectOnly) e = launch_gather_eb<EB>(s, tl, t, st, smem, threads);
    if (e != cudaSuccess) return e;
#define SNP_TILED_SEL(G, S)                                                                              \
    do {                                                                                                 \
        if (compact)                                                                                     \
            return sel == SNP_SELECT_FIRST ? launch_select_t<G, S, true, SNP_SELECT_FIRST, EB>(s, tl, t, st) \
                                           : launch_select_t<G, S, true, SNP_SELECT_PHILOX, EB>(s, tl, t, st); \
        return sel == SNP_SELECT_FIRST ? launch_select_t<G, S, false, SNP_SELECT_FIRST, EB>(s, tl, t, st)    \
                                       : launch_select_t<G, S, false, SNP_SELECT_PHILOX, EB>(s, tl, t, st);  \
    } while (0)
    switch (kind) {
        case kPullSelectOnly: SNP_TILED_SEL(false, true);
        case kPullFused: SNP_TILED_SEL(true, true);
        case kPullGatherOnly: SNP_TILED_SEL(true, false);
        default: return cudaErrorInvalidValue;
    }
#undef SNP_TILED_SEL
}

cudaError_t launch_tiled(const DevSys& s, const TiledSys& tl, int kind, int32_t t, cudaStream_t st, bool compact,
                         int sel, size_t smem, int threads) {
    switch (tl.e_bits) {
        case 2: return launch_tiled_eb<2>(s, tl, kind, t, st, compact, sel, smem, threads);
        case 4: return launch_tiled_eb<4>(s, tl, kind, t, st, compact, sel, smem, threads);
        case 8: return launch_tiled_eb<8>(s, tl, kind, t, st, compact, sel, smem, threads);
        case 16: return launch_tiled_eb<16>(s, tl, kind, t, st, compact, sel, smem, threads);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace snp
