// Load-balanced push over a sliced-ELL out-list (the direction of Alg. 4 and
// Alg. 5: every emitting source adds its spikes to each open target).
//
// The out-list is column-major in slices of 32 sources: slice s holds
// columns ptr[s] .. ptr[s+1]-1 of the global column space, and entry
// (column c, lane l) is ent[32 c + l], the l-th source's c-th target (or a
// pad).  One warp per slice, as the paper's kernels do with one thread per
// rule or neuron, leaves a slice that holds a hub (thousands of targets) to
// a single warp that walks its whole column serially.  Here each warp takes
// an equal contiguous run of the global column space instead, so the work is
// the same for every warp whatever the degree distribution:
//   * the warp finds the slice holding its first column with a 32-way
//     search over ptr (each lane probes one point, a ballot keeps the last
//     probe at or below the column);
//   * a slice in which no lane emits is skipped without reading its entries;
//   * columns are handled U at a time: U entry loads, then U status loads,
//     then U aggregated atomics in flight together, so a long run is not a
//     chain of dependent memory round trips;
//   * lanes of a warp that hit the same target add once (match + reduce),
//     and an add that leaves the int32 range raises the overflow flag.
#pragma once

#include <cuda_runtime.h>

#include <atomic>

#include "device_common.cuh"

namespace snp {

// Largest i in [0, n) with ptr[i] <= x, for nondecreasing ptr with
// ptr[0] <= x.  Warp-collective; every lane gets the result.
__device__ __forceinline__ int32_t warp_last_le(const int32_t* __restrict__ ptr, int32_t n, int32_t x, int lane) {
    int32_t lo = 0, len = n;  // the answer lies in [lo, lo + len); ptr[lo] <= x
    while (len > 32) {
        const int32_t stride = (len + 31) >> 5;
        const int32_t off = lane * stride;
        const bool le = off < len && __ldg(ptr + lo + off) <= x;
        const unsigned m = __ballot_sync(0xffffffffu, le);  // bit 0 is set: ptr[lo] <= x
        const int32_t nlo = lo + (31 - __clz(m)) * stride;
        len = min(stride, lo + len - nlo);
        lo = nlo;
    }
    const bool le = lane < len && __ldg(ptr + lo + lane) <= x;
    const unsigned m = __ballot_sync(0xffffffffu, le);
    return lo + (31 - __clz(m));
}

// Src describes one out-list form:
//   using Ent            entry type;
//   Ent pad()            the entry read by a lane whose source does not emit;
//   int32_t value(slice, lane)   the lane's source value for this step
//                                (0: the source does not emit);
//   int32_t target(Ent)  target slot, < 0 for a pad;
//   int32_t amount(Ent, value)   spikes the entry delivers.
template <int U, class Src>
__device__ __forceinline__ void push_scatter_balanced(const Src& src, const int32_t* __restrict__ ptr, int32_t nslices,
                                                      const typename Src::Ent* __restrict__ ent, int32_t* C,
                                                      const uint32_t* __restrict__ st, uint32_t* flags, int32_t q) {
    uint32_t* overflow_flag = flags + kFlagOverflow;
    using Ent = typename Src::Ent;
    const int lane = threadIdx.x & 31;
    const long long warp = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long total = __ldg(ptr + nslices);
    const int32_t c0 = (int32_t)(total * warp / nwarps);
    const int32_t c1 = (int32_t)(total * (warp + 1) / nwarps);
    if (c0 >= c1) return;  // warp-uniform
    int32_t slice = warp_last_le(ptr, nslices, c0, lane);
    int32_t end = __ldg(ptr + slice + 1);
    bool ovf = false;
    for (int32_t c = c0;;) {
        const int32_t v = src.value(slice, lane);
        const int32_t stop = min(end, c1);
        if (__any_sync(0xffffffffu, v != 0)) {
            const Ent* __restrict__ p = ent + (size_t)lane;
            int32_t col = c;
            for (; col + U <= stop; col += U) {
                int32_t tg[U], amt[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const Ent e = v != 0 ? __ldg(p + (size_t)(col + u) * kSlice) : src.pad();
                    tg[u] = src.target(e);
                    if (tg[u] >= 0) tg[u] = (int32_t)SNP_IDX(flags, 3, tg[u], q);
                    amt[u] = src.amount(e, v);
                }
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (tg[u] >= 0 && (__ldg(st + tg[u]) >> kPendShift) != 0u) tg[u] = -1;  // closed: lost
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const unsigned grp = __match_any_sync(0xffffffffu, tg[u]);
                    const unsigned add = __reduce_add_sync(grp, tg[u] >= 0 ? (unsigned)amt[u] : 0u);
                    if (tg[u] >= 0 && (__ffs(grp) - 1) == lane) {
                        const int old = atomicAdd(C + tg[u], (int)add);
                        ovf |= (long long)old + (long long)add > 2147483647ll;
                    }
                }
            }
            for (; col < stop; ++col) {
                const Ent e = v != 0 ? __ldg(p + (size_t)col * kSlice) : src.pad();
                int32_t tg = src.target(e);
                if (tg >= 0) tg = (int32_t)SNP_IDX(flags, 3, tg, q);
                if (tg >= 0 && (__ldg(st + tg) >> kPendShift) != 0u) tg = -1;
                const unsigned grp = __match_any_sync(0xffffffffu, tg);
                const unsigned add = __reduce_add_sync(grp, tg >= 0 ? (unsigned)src.amount(e, v) : 0u);
                if (tg >= 0 && (__ffs(grp) - 1) == lane) {
                    const int old = atomicAdd(C + tg, (int)add);
                    ovf |= (long long)old + (long long)add > 2147483647ll;
                }
            }
        }
        c = stop;
        if (c >= c1) break;
        do {  // the next slice holding column c (zero-width slices skipped)
            ++slice;
            end = __ldg(ptr + slice + 1);
        } while (end <= c);
    }
    if (ovf) atomicOr(overflow_flag, 1u);
}

// Blocks of 256 threads for a balanced push launch: `per_sm` blocks on every
// SM (the kernel's __launch_bounds__ minimum, so they are all resident at
// once), and no more than one warp per slice.  The SM count is a plain
// device-attribute query, cached per device (launches may be captured into
// CUDA graphs, so nothing here synchronizes or allocates).
inline unsigned push_blocks(int per_sm, long long nslices) {
    static std::atomic<int> sms_of[64];
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64) {
        sms = sms_of[dev].load(std::memory_order_relaxed);
        if (sms <= 0 && cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0)
            sms_of[dev].store(sms, std::memory_order_relaxed);
    }
    if (sms <= 0) {
        cudaGetLastError();
        sms = 152;
    }
    const long long full = (long long)sms * per_sm;
    const long long by_slices = (nslices * 32 + 255) / 256;
    const long long b = by_slices < full ? by_slices : full;
    return (unsigned)(b > 0 ? b : 1);
}

}  // namespace snp
