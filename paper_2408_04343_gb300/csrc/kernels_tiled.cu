// Tiled engine: grid-wide pull step with the emission vector in shared memory.
//
// Random reads of E_k are the cost of the pull step: each in-edge reads one
// neuron's emission, and on this part random 4-byte reads served by L2 or L1
// run near one distinct line per clock per SM, well below what HBM can feed
// the index stream.  Here E_k is bit-packed (2 bits per neuron when every p
// is at most 3) and every CTA copies it into its shared memory, one source
// partition at a time, so the gathers become shared-memory reads.
//
// One persistent launch per step, one CTA per SM, each CTA owning a range of
// slices (32 neurons, one warp each).  For every partition h the CTA loads
// h's packed emissions, then each warp walks the jagged column-major blocks
// of its slices (one coalesced load per column, no padding) and accumulates
// per-lane sums; with more than one partition the sums wait in shared memory
// for the select pass, which also writes the packed E_{k+1} for the next
// launch.  Same fusion, halt test and status word as k_step_pull.
#include <cuda_runtime.h>

#include "device_common.cuh"
#include "kernels.h"

namespace snp {

__device__ __forceinline__ int32_t ld_stream_i32(const int32_t* p) {
    int32_t v;
    asm volatile("ld.global.nc.L1::no_allocate.s32 %0, [%1];" : "=r"(v) : "l"(p));
    return v;
}

template <int EB>
__device__ __forceinline__ uint32_t pk_get(const uint32_t* __restrict__ e, int32_t i) {
    constexpr uint32_t mask = (EB == 32) ? 0xffffffffu : ((1u << EB) - 1u);
    const uint32_t bit = (uint32_t)i * EB;
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

// Sum of the packed emissions of one lane's in-neighbours in one block.
template <int EB, int U>
__device__ __forceinline__ int32_t block_sum(const TiledSys& tl, const uint32_t* __restrict__ Esm, int64_t blk_id,
                                             int lane) {
    const int32_t base = __ldg(tl.blk + blk_id);
    const int32_t n = (int32_t)__ldg(tl.cnt + blk_id * kSlice + lane);
    const int32_t maxn = __reduce_max_sync(0xffffffffu, (unsigned)n);
    const unsigned lt = (1u << lane) - 1u;
    int32_t pos = base;
    int32_t sum = 0;
    for (int32_t t = 0; t < maxn; t += U) {
        int32_t idx[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const bool v = n > t + u;
            const unsigned a = __ballot_sync(0xffffffffu, v);
            idx[u] = v ? ld_stream_i32(tl.ent + pos + __popc(a & lt)) : -1;
            pos += __popc(a);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (idx[u] >= 0) sum += (int32_t)pk_get<EB>(Esm, idx[u]);
    }
    return sum;
}

template <bool GATHER, bool SELECT, bool COMPACT, int SEL, int EB, bool MULTI>
__global__ void __launch_bounds__(1024, 1) k_tiled(DevSys s, TiledSys tl, int32_t t) {
    constexpr int U = 8;
    extern __shared__ uint32_t smem[];
    uint32_t* Esm = smem;
    int32_t* partial = reinterpret_cast<int32_t*>(smem + tl.part_words);
    uint32_t* fl = s.flags;
    const unsigned long long base = s.step[kStepBase];
    const unsigned long long kg = base + (unsigned long long)t;
    const unsigned long long ks = GATHER ? kg + 1ull : kg;
    if (GATHER) {
        if (ld_volatile(fl + kFlagHalted)) return;
        if (ld_volatile(fl + kFlagAct0 + (int)(kg % 3ull)) == 0u) {
            if (threadIdx.x == 0) {
                s.step[kStepHalt] = kg;
                __threadfence();
                atomicExch(fl + kFlagHalted, 1u);
            }
            return;
        }
        if (SELECT && blockIdx.x == 0 && threadIdx.x == 0) fl[kFlagAct0 + (int)((kg + 2ull) % 3ull)] = 0u;
    }
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int nwarps = blockDim.x >> 5;
    const int32_t lo = __ldg(tl.cta_lo + blockIdx.x), hi = __ldg(tl.cta_lo + blockIdx.x + 1);
    uint32_t* Enext = tl.Eg[ks & 1ull];
    bool active = false;

    // select phase of one slice; `sum` is its gathered in-flow (GATHER only)
    auto finish_slice = [&](int32_t slice, int32_t sum) {
        const int32_t slot = slice * kSlice + lane;
        const bool valid = slot < s.q;
        int32_t c = 0;
        uint32_t st = 0u;
        if (valid) {
            c = s.C[slot];
            st = s.st[slot];
        }
        if (GATHER && valid && (st >> kPendShift) == 0u) {
            const long long nc = (long long)c + sum;
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
                s.rules, __ldg(s.rule_off + slot), __ldg(s.rule_off + slot + 1), c, st, ks,
                SEL == SNP_SELECT_PHILOX ? (uint32_t)__ldg(s.orig + slot) : 0u, s.seed);
            c = o.c_after;
            active |= o.active;
            emit = (uint32_t)o.emit;
            s.S[ks & 1ull][slot] = o.s;
            s.st[slot] = o.st;
        }
        if (valid) s.C[slot] = c;
        if (SELECT) pk_put_slice<EB>(Enext, slice, lane, emit);
    };

    if (GATHER) {
        const uint32_t* Eprev = tl.Eg[kg & 1ull];
        for (int h = 0; h < tl.P; ++h) {
            const uint4* src = reinterpret_cast<const uint4*>(Eprev + (size_t)h * tl.part_words);
            uint4* dst = reinterpret_cast<uint4*>(Esm);
            for (int i = threadIdx.x; i < tl.part_words / 4; i += blockDim.x) dst[i] = __ldcg(src + i);
            __syncthreads();
            for (int32_t slice = lo + warp; slice < hi; slice += nwarps) {
                const int32_t sum = block_sum<EB, U>(tl, Esm, (int64_t)slice * tl.P + h, lane);
                if (MULTI) {
                    int32_t* pp = partial + (slice - lo) * kSlice + lane;
                    *pp = (h == 0) ? sum : *pp + sum;
                } else {
                    finish_slice(slice, sum);
                }
            }
            __syncthreads();
        }
    }
    if (!GATHER || MULTI) {
        for (int32_t slice = lo + warp; slice < hi; slice += nwarps)
            finish_slice(slice, GATHER ? partial[(slice - lo) * kSlice + lane] : 0);
    }
    if (SELECT) {
        if (__syncthreads_or(active) && threadIdx.x == 0) {
            uint32_t* a = fl + kFlagAct0 + (int)(ks % 3ull);
            if (ld_volatile(a) == 0u) atomicExch(a, 1u);
        }
    }
}

template <bool G, bool S, bool C, int SEL, int EB>
static cudaError_t launch_tiled_t(const DevSys& s, const TiledSys& tl, int32_t t, cudaStream_t st, size_t smem,
                                  int threads) {
    cudaError_t e;
    if (tl.P > 1) {
        auto fn = k_tiled<G, S, C, SEL, EB, true>;
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        fn<<<tl.G, threads, smem, st>>>(s, tl, t);
    } else {
        auto fn = k_tiled<G, S, C, SEL, EB, false>;
        e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        fn<<<tl.G, threads, smem, st>>>(s, tl, t);
    }
    return cudaGetLastError();
}

template <bool G, bool S, bool C, int SEL>
static cudaError_t launch_tiled_eb(const DevSys& s, const TiledSys& tl, int32_t t, cudaStream_t st, size_t smem,
                                   int threads) {
    switch (tl.e_bits) {
        case 2: return launch_tiled_t<G, S, C, SEL, 2>(s, tl, t, st, smem, threads);
        case 4: return launch_tiled_t<G, S, C, SEL, 4>(s, tl, t, st, smem, threads);
        case 8: return launch_tiled_t<G, S, C, SEL, 8>(s, tl, t, st, smem, threads);
        case 16: return launch_tiled_t<G, S, C, SEL, 16>(s, tl, t, st, smem, threads);
        default: return cudaErrorInvalidValue;
    }
}

template <bool G, bool S>
static cudaError_t launch_tiled_k(const DevSys& s, const TiledSys& tl, int32_t t, cudaStream_t st, bool compact,
                                  int sel, size_t smem, int threads) {
    if (compact) {
        if (sel == SNP_SELECT_FIRST) return launch_tiled_eb<G, S, true, SNP_SELECT_FIRST>(s, tl, t, st, smem, threads);
        return launch_tiled_eb<G, S, true, SNP_SELECT_PHILOX>(s, tl, t, st, smem, threads);
    }
    if (sel == SNP_SELECT_FIRST) return launch_tiled_eb<G, S, false, SNP_SELECT_FIRST>(s, tl, t, st, smem, threads);
    return launch_tiled_eb<G, S, false, SNP_SELECT_PHILOX>(s, tl, t, st, smem, threads);
}

cudaError_t launch_tiled(const DevSys& s, const TiledSys& tl, int kind, int32_t t, cudaStream_t st, bool compact,
                         int sel, size_t smem, int threads) {
    switch (kind) {
        case kPullSelectOnly: return launch_tiled_k<false, true>(s, tl, t, st, compact, sel, smem, threads);
        case kPullFused: return launch_tiled_k<true, true>(s, tl, t, st, compact, sel, smem, threads);
        case kPullGatherOnly: return launch_tiled_k<true, false>(s, tl, t, st, compact, sel, smem, threads);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace snp
