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
//  * k_tiled_gather -- one CTA per SM.  CTA g*P + h owns slice range g and
//    source partition h: it loads h's packed emissions once and streams the
//    group of in-edge words of its range from h edge-parallel (16-byte vector loads, no
//    per-neuron bookkeeping): each word names a local target slot and a
//    source, whose emission is added to the target's shared-memory
//    accumulator (words are sorted by target, so runs of one target within
//    a load are summed first).  The accumulators become partition h's
//    in-flow vector of step k; the select launch sums the P of them.
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

// Four target-sorted words of one window: the emissions of consecutive words
// with the same target are summed in registers and added to that target
// (window base + dst) with one atomic, without branches: r_i is the running
// sum of the run that ends at word i, flushed when the next word's target
// differs (or at the last word).
template <int EB>
__device__ __forceinline__ void edges4(const uint32_t* __restrict__ Esm, int* acc, const uint4& q, uint32_t base,
                                       uint32_t smask, int sbits) {
    const uint32_t v0 = pk_get<EB>(Esm, q.x & smask), v1 = pk_get<EB>(Esm, q.y & smask);
    const uint32_t v2 = pk_get<EB>(Esm, q.z & smask), v3 = pk_get<EB>(Esm, q.w & smask);
    const uint32_t d0 = q.x >> sbits, d1 = q.y >> sbits, d2 = q.z >> sbits, d3 = q.w >> sbits;
    const bool s1 = d1 == d0, s2 = d2 == d1, s3 = d3 == d2;
    const uint32_t r0 = v0;
    const uint32_t r1 = (s1 ? r0 : 0u) + v1;
    const uint32_t r2 = (s2 ? r1 : 0u) + v2;
    const uint32_t r3 = (s3 ? r2 : 0u) + v3;
    if (!s1 && r0) atomicAdd(acc + base + d0, (int)r0);
    if (!s2 && r1) atomicAdd(acc + base + d1, (int)r1);
    if (!s3 && r2) atomicAdd(acc + base + d2, (int)r2);
    if (r3) atomicAdd(acc + base + d3, (int)r3);
}

// Target window of the 16-byte word group at index i (monotone in i).
__device__ __forceinline__ uint32_t window_of(const int32_t* wb, int32_t i, int& k) {
    while (k + 1 < kTiledMaxSub && i >= wb[k + 1]) ++k;
    return (uint32_t)k;
}

// In-flow of step kg = base + t into tl.inflow (partition h's share).
template <int EB>
__global__ void __launch_bounds__(1024, 1) k_tiled_gather(DevSys s, TiledSys tl, int32_t t) {
    extern __shared__ uint32_t smem[];
    __shared__ int32_t wb[kTiledMaxSub + 1];
    uint32_t* Esm = smem;                                              // part_words + a zero word
    int* acc = reinterpret_cast<int*>(smem + tl.part_words + 4);
    uint32_t* fl = s.flags;
    const unsigned long long kg = s.step[kStepBase] + (unsigned long long)t;
    if (step_blocked(fl, s.step, kg)) return;
    if (blockIdx.x == 0 && threadIdx.x == 0) fl[kFlagAct0 + (int)((kg + 2ull) % 3ull)] = 0u;
    const int range = blockIdx.x / tl.P, h = blockIdx.x % tl.P;
    const int32_t lo = __ldg(tl.cta_lo + range), hi = __ldg(tl.cta_lo + range + 1);
    if (threadIdx.x <= kTiledMaxSub) wb[threadIdx.x] = __ldg(tl.sub + (size_t)blockIdx.x * (kTiledMaxSub + 1) + threadIdx.x) / 4;
    if (threadIdx.x < 4) Esm[tl.part_words + threadIdx.x] = 0u;
    for (int i = threadIdx.x; i < tl.acc_words; i += blockDim.x) acc[i] = 0;
    const uint32_t smask = (1u << tl.src_bits) - 1u;
    const int sbits = tl.src_bits;
    const int db = 32 - sbits;
    const uint4* ent = reinterpret_cast<const uint4*>(tl.ent);
    {
        const uint4* src = reinterpret_cast<const uint4*>(SNP_PICK(tl.Eg, kg) + (size_t)h * tl.part_words);
        uint4* dst = reinterpret_cast<uint4*>(Esm);
        for (int i = threadIdx.x; i < tl.part_words / 4; i += blockDim.x) dst[i] = __ldcg(src + i);
        __syncthreads();
        const int32_t g1 = wb[kTiledMaxSub];
        const int32_t stride = blockDim.x;
        int32_t i = wb[0] + threadIdx.x;
        // eight independent 16-byte loads per thread in flight, then their
        // shared-memory work; the window index only moves forward
        int k = 0;
        for (; i + 7 * stride < g1; i += 8 * stride) {
            uint4 q[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) q[u] = ld_stream_v4(ent + i + u * stride);
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                int ku = k;
                const uint32_t base = window_of(wb, i + u * stride, ku) << db;
                edges4<EB>(Esm, acc, q[u], base, smask, sbits);
            }
            window_of(wb, i + 7 * stride, k);
        }
        for (; i < g1; i += stride) {
            const uint4 a = ld_stream_v4(ent + i);
            edges4<EB>(Esm, acc, a, window_of(wb, i, k) << db, smask, sbits);
        }
        __syncthreads();
    }
    const int32_t slot0 = lo * kSlice;
    const int32_t nloc = (hi - lo) * kSlice;
    int32_t* out = tl.inflow + (size_t)h * s.nslices * kSlice + slot0;
    for (int i = threadIdx.x; i < nloc; i += blockDim.x) out[i] = acc[i];
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
            long long in = 0;
            for (int h = 0; h < tl.P; ++h) in += tl.inflow[(size_t)h * s.nslices * kSlice + slot];
            const long long nc = (long long)c + in;
            if (nc > 2147483647ll) {
                atomicOr(fl + kFlagOverflow, 1u);
                c = 2147483647;
            } else {
                c = (int32_t)nc;
            }
        }
        uint32_t emit = 0u;
        if (SELECT && valid) {
            const SelOut o = select_slot<COMPACT, SEL>(s, slot, c, st, ks);
            c = o.c_after;
            active = o.active;
            emit = (uint32_t)o.emit;
            SNP_PICK(s.S, ks)[slot] = o.s;
            if (o.st != st) s.st[slot] = o.st;  // most neurons stay open: skip the write
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
