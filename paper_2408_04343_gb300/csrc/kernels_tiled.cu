// Tiled engine: grid-wide pull step with the emission vector in shared memory.
//
// Random reads of E_k are the cost of the pull step: each in-edge reads one
// neuron's emission, and on this part random 4-byte reads served by L2 or L1
// run near one distinct line per clock per SM, well below what HBM can feed
// the index stream.  Here E_k is bit-packed (2 bits per neuron when every p
// is at most 3) and every CTA copies it into its shared memory, one source
// partition at a time, so the gathers become shared-memory reads.
//
// A step is one launch, k_tiled_step, when the P partitions of a slice range
// fit one thread-block cluster (P <= kTiledMaxCluster): the gather below,
// then the select of the next step in the same CTAs, the in-flow summed
// across the cluster through distributed shared memory.  Otherwise a step is
// two launches:
//  * k_tiled_gather -- one CTA per SM.  CTA g*P + h owns slice range g and
//    source partition h: it loads h's packed emissions once and streams the
//    group of in-edge words of its range from h edge-parallel (16-byte vector loads, no
//    per-neuron bookkeeping): each word names a local target slot and a
//    source, whose emission is added to the target's shared-memory
//    accumulator (words are sorted by target; one reduction per aligned pair
//    of words in the paired layout, per run of equal targets within a load
//    otherwise).  The accumulators become partition h's
//    in-flow vector of step k; the select launch sums the P of them.
//  * k_tiled_select -- full occupancy, one warp per slice: finishes step k
//    (C_{k+1} = C' + [open] * in-flow), selects step k+1 and writes the
//    packed E_{k+1} that the next gather loads.
// Same status word, fixed-point test and activity words as k_step_pull.
#include <cuda_runtime.h>

#include <type_traits>

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
    if constexpr (EB <= 4) {
#pragma unroll
        for (int g = 0; g < EB; ++g) {
            const uint32_t part = __reduce_or_sync(0xffffffffu, lane / per == g ? w : 0u);
            if (lane == g * per) e[slice * EB + g] = part;
        }
    } else {
#pragma unroll
        for (int off = 1; off < per; off <<= 1) w |= __shfl_xor_sync(0xffffffffu, w, off);
        if (lane % per == 0) e[slice * EB + lane / per] = w;
    }
}

// ---- shared-memory access by 32-bit shared addresses ----------------------
// The gather's reductions are written with 32-bit shared-window addresses
// (no generic 64-bit address arithmetic), and conditional reductions are
// predicated rather than branched around.
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void red_add(uint32_t a, uint32_t v) {
    asm volatile("red.shared.add.u32 [%0], %1;" ::"r"(a), "r"(v));
}
__device__ __forceinline__ void red_add_if(uint32_t a, uint32_t v, bool p) {
    asm volatile(
        "{\n\t.reg .pred q;\n\t"
        "setp.ne.u32 q, %2, 0;\n\t"
        "@q red.shared.add.u32 [%0], %1;\n\t}"
        :
        : "r"(a), "r"(v), "r"((uint32_t)p));
}

// Emission of the source named by the low bits of entry word w (the bits
// above the source field do not disturb it): word src / per of the packed
// vector Esm in shared memory, field src mod per.  `wmask` keeps the
// source's word index.  A plain shared-memory load, so the compiler may
// issue the lookups of a whole batch ahead of the reductions (which touch
// only the accumulators).
template <int EB>
__device__ __forceinline__ uint32_t emission_of(const uint32_t* __restrict__ Esm, uint32_t w, uint32_t wmask) {
    constexpr uint32_t per = 32u / EB;  // emissions per 32-bit word
    const uint32_t word = Esm[(w >> __builtin_ctz(per)) & wmask];
    // rotate by (src mod per) * EB: the shift count is taken mod 32
    return __funnelshift_r(word, word, w * (uint32_t)EB) & ((1u << EB) - 1u);
}

// Run layout, one 16-byte load of a window: four words sorted by target
// (abase = shared address of the window's first accumulator).  The
// emissions of consecutive words with the same target are summed in
// registers, without branches (r_i is the running sum of the run that ends
// at word i), and a run is added when the next word's target differs or at
// the last word.
template <int EB>
__device__ __forceinline__ void edges4(const uint32_t* __restrict__ Esm, uint32_t abase, const uint4& q,
                                       uint32_t wmask, int sbits) {
    const uint32_t v0 = emission_of<EB>(Esm, q.x, wmask), v1 = emission_of<EB>(Esm, q.y, wmask);
    const uint32_t v2 = emission_of<EB>(Esm, q.z, wmask), v3 = emission_of<EB>(Esm, q.w, wmask);
    const uint32_t d0 = q.x >> sbits, d1 = q.y >> sbits, d2 = q.z >> sbits, d3 = q.w >> sbits;
    const bool s1 = d1 == d0, s2 = d2 == d1, s3 = d3 == d2;
    const uint32_t r0 = v0;
    const uint32_t r1 = (s1 ? r0 : 0u) + v1;
    const uint32_t r2 = (s2 ? r1 : 0u) + v2;
    const uint32_t r3 = (s3 ? r2 : 0u) + v3;
    red_add_if(abase + d0 * 4u, r0, !s1);
    red_add_if(abase + d1 * 4u, r1, !s2);
    red_add_if(abase + d2 * 4u, r2, !s3);
    red_add(abase + d3 * 4u, r3);
}

// Paired layout, one 16-byte load (two pairs) of a thread's contiguous run:
// runs of pairs with the same target are summed in `run` and added to the
// accumulator at `cur` (a shared address) only when the target changes, so
// a target costs one reduction however many pairs it has.  The first and
// last target of a thread's run may be shared with the neighbouring thread;
// the reduction is atomic.
template <int EB>
__device__ __forceinline__ void pairs_merge(const uint32_t* __restrict__ Esm, uint32_t abase, const uint4& q,
                                            uint32_t wmask, int sbits, uint32_t& cur, uint32_t& run) {
    const uint32_t v01 = emission_of<EB>(Esm, q.x, wmask) + emission_of<EB>(Esm, q.y, wmask);
    const uint32_t v23 = emission_of<EB>(Esm, q.z, wmask) + emission_of<EB>(Esm, q.w, wmask);
    const uint32_t a0 = abase + (q.x >> sbits) * 4u, a1 = abase + (q.z >> sbits) * 4u;
    bool f = a0 != cur;
    red_add_if(cur, run, f);
    run = (f ? 0u : run) + v01;
    cur = a0;
    f = a1 != cur;
    red_add_if(cur, run, f);
    run = (f ? 0u : run) + v23;
    cur = a1;
}

// Run-length step: when the advance d is non-zero, store the run as the
// in-flow of the target at shared address a (the thread owns that target:
// runs are cut at target boundaries) and start a new run (returns 0), else
// return the run.  One predicate serves the store and the reset.
__device__ __forceinline__ uint32_t run_flush(uint32_t a, uint32_t run, uint32_t d) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %2, 0;\n\t"
        "@p st.shared.u32 [%1], %3;\n\t"
        "selp.u32 %0, 0, %3, p;\n\t}"
        : "=r"(r)
        : "r"(a), "r"(d), "r"(run));
    return r;
}

__device__ __forceinline__ void st_shared_u32(uint32_t a, uint32_t v) {
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v));
}

// The same for byte accumulators (the in-flow of a target from one
// partition is at most 255 there).
__device__ __forceinline__ uint32_t run_flush8(uint32_t a, uint32_t run, uint32_t d) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.u32 p, %2, 0;\n\t"
        "@p st.shared.u8 [%1], %3;\n\t"
        "selp.u32 %0, 0, %3, p;\n\t}"
        : "=r"(r)
        : "r"(a), "r"(d), "r"(run));
    return r;
}

__device__ __forceinline__ void st_shared_u8(uint32_t a, uint32_t v) {
    asm volatile("st.shared.u8 [%0], %1;" ::"r"(a), "r"(v));
}

// Run-length layout, one 16-byte load: five 24-bit entries b << db | d,
// where b is the source's bit index in the packed emissions (source x EB)
// and d the target advance.  Each entry first advances the thread's target
// by d -- storing the run of the previous target in its accumulator when
// d > 0 -- then adds its emission to the run: word b / 32 of Esm, rotated
// by b mod 32 (the funnel shift takes its count mod 32).  `cur` is the
// shared address of the current target's accumulator.
// fl, ewords, abase, alim: the bounds-checked build's flag word, the packed
// emission words, the accumulators' shared address and byte size.
template <int EB, bool ACC8 = false>
__device__ __forceinline__ void rle_vector(const uint32_t* __restrict__ Esm, const uint4& q, int db,
                                           uint32_t& cur, uint32_t& run, uint32_t* fl = nullptr,
                                           int32_t ewords = 0, uint32_t abase = 0u, int32_t alim = 0) {
    constexpr uint32_t M = 0xFFFFFFu;
    const uint32_t e[5] = {q.x & M, __funnelshift_r(q.x, q.y, 24) & M, __funnelshift_r(q.y, q.z, 16) & M, q.z >> 8,
                           q.w & M};
    const uint32_t dmask = (1u << db) - 1u;
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const uint32_t word = Esm[SNP_IDX(fl, 1, e[i] >> (db + 5), ewords)];
        const uint32_t v = __funnelshift_r(word, word, e[i] >> db) & ((1u << EB) - 1u);
        const uint32_t d = e[i] & dmask;
#ifdef SNP_CHECK_BOUNDS
        if (d != 0u && (int32_t)(cur - abase) >= alim) {  // the accumulator a flush would write
            atomicOr(fl + kFlagBounds, 1u << 2);
            cur = abase;
        }
#endif
        if constexpr (ACC8) {
            run = run_flush8(cur, run, d) + v;
            cur += d;
        } else {
            run = run_flush(cur, run, d) + v;
            cur += d * 4u;
        }
    }
}

enum : int { kLayoutRuns = 0, kLayoutPairs = 1, kLayoutRle = 2, kLayoutRle8 = 3 };  // Rle8: byte accumulators

// ---- bulk copy of a partition's emissions into shared memory -------------
__device__ __forceinline__ void mbar_init(uint32_t bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}
// Asks L2 to fetch [p, p + bytes) from memory (16-byte aligned, a multiple
// of 16 bytes); nothing waits for it.
__device__ __forceinline__ void prefetch_l2(const void* p, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
}
__device__ __forceinline__ void prefetch_l2_range(const char* p, uint64_t bytes) {
    for (uint64_t o = 0; o < bytes; o += 32768) prefetch_l2(p + o, (uint32_t)min((uint64_t)32768, bytes - o));
}
// Waits for phase 0 of the barrier, at most `limit` polls; true when it completed.
__device__ __forceinline__ bool mbar_wait0(uint32_t bar, int limit) {
    for (int it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], 0;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar)
            : "memory");
        if (done) return true;
    }
    return false;
}
__global__ void k_wait_check(int polls, uint32_t* out) {
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(&bar);
    if (threadIdx.x == 0) {
        mbar_init(b);
        mbar_expect_tx(b, 16u);  // sixteen bytes that no copy will deliver
    }
    __syncthreads();
    const bool done = mbar_wait0(b, polls);
    if (threadIdx.x == 0) *out = done ? 1u : 2u;
}

cudaError_t launch_wait_check(int polls, uint32_t* out, cudaStream_t st) {
    k_wait_check<<<1, 32, 0, st>>>(polls, out);
    return cudaGetLastError();
}

constexpr int kBulkChunk = 32768;       // bytes per bulk copy instruction
constexpr int kWaitPolls = 1 << 20;     // each poll may suspend for a while; ~seconds in all

// One batch of D 16-byte loads of a thread: its vectors u0 .. u0+D-1 (those
// below nt), sorted indices s0 + u.  The window index k only moves forward;
// a batch inside one window (the common case) takes its base once.
template <int EB, int LAYOUT, int D>
__device__ __forceinline__ void gather_batch(const uint4 (&x)[D], int32_t u0, int32_t nt, int32_t s0,
                                             const int32_t* wb, int& k, const uint32_t* __restrict__ Esm,
                                             uint32_t acc0, int db, uint32_t wmask, int sbits, uint32_t& cur,
                                             uint32_t& run) {
    constexpr bool PAIRS = LAYOUT == kLayoutPairs;
    if constexpr (LAYOUT == kLayoutRle || LAYOUT == kLayoutRle8) {  // no target windows: the target is carried in cur
#pragma unroll
        for (int u = 0; u < D; ++u)
            if (u0 + u < nt) rle_vector<EB>(Esm, x[u], db, cur, run);
        return;
    }
    if (u0 + D <= nt && s0 + u0 + D - 1 < wb[k + 1]) {  // k <= kTiledMaxSub - 1; wb[kTiledMaxSub] = group end
        const uint32_t abase = acc0 + ((uint32_t)k << db) * 4u;
#pragma unroll
        for (int u = 0; u < D; ++u) {
            if constexpr (PAIRS)
                pairs_merge<EB>(Esm, abase, x[u], wmask, sbits, cur, run);
            else
                edges4<EB>(Esm, abase, x[u], wmask, sbits);
        }
    } else {
#pragma unroll
        for (int u = 0; u < D; ++u) {
            if (u0 + u < nt) {
                const int32_t su = s0 + u0 + u;
                int ku = k;
                while (ku + 1 < kTiledMaxSub && su >= wb[ku + 1]) ++ku;
                const uint32_t abase = acc0 + ((uint32_t)ku << db) * 4u;
                if constexpr (PAIRS)
                    pairs_merge<EB>(Esm, abase, x[u], wmask, sbits, cur, run);
                else
                    edges4<EB>(Esm, abase, x[u], wmask, sbits);
            }
        }
    }
    const int32_t snext = s0 + u0 + D;
    while (k + 1 < kTiledMaxSub && snext >= wb[k + 1]) ++k;
}

// Vectors u0 .. u0+D-1 of a thread (those below nt); vector u is at col[u * T].
template <int D>
__device__ __forceinline__ void load_batch(uint4 (&x)[D], const uint4* col, int32_t u0, int32_t nt) {
#pragma unroll
    for (int u = 0; u < D; ++u)
        if (u0 + u < nt) x[u] = ld_stream_v4(col + (size_t)(u0 + u) * kTiledThreads);
}

// Gather phase of step kg = base + t, shared by both launch forms: CTA
// g*P + h adds the emissions of partition h along the in-edges of range g
// into its shared accumulators.  The part before grid_dependency_wait
// touches only the constant layout (window bounds, the first entry vectors)
// and the CTA's own shared memory, so it overlaps the end of the launch
// before.  Returns kPhaseBlocked when the step is not executed (a fixed
// point; the same answer in every CTA), kPhaseTimeout when the bulk copy's
// wait gave up (the timeout flag is set; the accumulators are incomplete),
// else kPhaseOk.  On return the accumulators are complete in this CTA.
enum : int { kPhaseOk = 0, kPhaseBlocked = 1, kPhaseTimeout = 2 };

template <int EB, int LAYOUT>
__device__ __forceinline__ int tiled_gather_phase(const DevSys& s, const TiledSys& tl, int32_t t, uint32_t* Esm,
                                                  int* acc, int32_t* wb, unsigned long long* bar,
                                                  unsigned long long& kg_out) {
    constexpr int D = 2;  // vectors per batch; two batches in registers
    const int h = blockIdx.x % tl.P;
    const uint32_t ebar = smem_u32(bar);
    // every thread reads its own bounds (one broadcast line), so the first
    // entry loads do not wait for a barrier; the shared copy of the window
    // bounds is published by the barrier after grid_dependency_wait.  Thread
    // t streams its own run of the group's vectors (see TiledPack).
    const int32_t* subg = tl.sub + (size_t)blockIdx.x * (kTiledMaxSub + 1);
    if (threadIdx.x <= kTiledMaxSub) wb[threadIdx.x] = __ldg(subg + threadIdx.x) / 4;
    const int32_t base = __ldg(subg) / 4;
    const int32_t N = __ldg(subg + kTiledMaxSub) / 4 - base;
    const int32_t tid = (int32_t)threadIdx.x;
    const int32_t n = (N + kTiledThreads - 1) / kTiledThreads;
    const int32_t r = N - (n - 1) * kTiledThreads;
    const int32_t nt = tid < r ? n : n - 1;                       // this thread's vectors
    const int32_t s0 = base + tid * n - max(0, tid - r);          // sorted index of the first
    const uint4* col = reinterpret_cast<const uint4*>(tl.ent) + base + tid;
    uint4 qa[D], qb[D];
    constexpr bool RLE = LAYOUT == kLayoutRle || LAYOUT == kLayoutRle8;
    constexpr bool ACC8 = LAYOUT == kLayoutRle8;
    if constexpr (RLE) {
        qa[0] = ld_stream_v4(col);  // unguarded: see the gather loop below
        qa[1] = ld_stream_v4(col + kTiledThreads);
    } else {
        load_batch(qa, col, 0, nt);
    }
    const int32_t tstart = RLE ? __ldg(tl.tstart + (size_t)blockIdx.x * kTiledThreads + tid) : 0;
    if (threadIdx.x < 4) Esm[tl.part_words + threadIdx.x] = 0u;
    if (threadIdx.x == 0) mbar_init(ebar);
    for (int j = threadIdx.x; j < tl.acc_words; j += blockDim.x) acc[j] = 0;
    const int sbits = tl.src_bits;
    // target bits of a 32-bit entry; for run-length entries, the advance's bits
    const int db = RLE ? 24 - sbits - __builtin_ctz((unsigned)EB) : 32 - sbits;
    constexpr uint32_t per = 32u / EB;
    const uint32_t wmask = ((1u << sbits) - 1u) >> __builtin_ctz(per);
    const uint32_t esm = smem_u32(Esm);
    const uint32_t acc0 = smem_u32(acc);

    grid_dependency_wait();  // the launch that wrote E_k has finished
    uint32_t* fl = s.flags;
    const unsigned long long kg = s.step[kStepBase] + (unsigned long long)t;
    kg_out = kg;
    // the partition's emissions are requested before the fixed-point test, so
    // the copy overlaps the flag read (a halted step waits for it and leaves)
    const uint32_t ebytes = (uint32_t)tl.part_words * 4u;
    if (threadIdx.x == 0) {
        const char* src = reinterpret_cast<const char*>(SNP_PICK(tl.Eg, kg) + (size_t)h * tl.part_words);
        mbar_expect_tx(ebar, ebytes);
        for (uint32_t o = 0; o < ebytes; o += kBulkChunk)
            bulk_g2s(esm + o, src + o, min((uint32_t)kBulkChunk, ebytes - o), ebar);
    }
    if (step_blocked(fl, s.step, kg)) {  // its barrier also publishes wb, acc, the mbarrier
        mbar_wait0(ebar, kWaitPolls);
        return kPhaseBlocked;
    }
    allow_dependents();
    if (blockIdx.x == 0 && threadIdx.x == 0) fl[kFlagAct0 + (int)((kg + 2ull) % 3ull)] = 0u;
    const bool landed = mbar_wait0(ebar, kWaitPolls);
    if (!__syncthreads_and(landed)) {  // the same answer in every thread of the CTA
        if (threadIdx.x == 0) atomicOr(fl + kFlagTimeout, 1u);
        if (!landed) mbar_wait0(ebar, kWaitPolls);  // let the copy land before the shared memory goes away
        return kPhaseTimeout;
    }
    // paired and run-length layouts: the target being summed and its sum so far
    uint32_t cur = acc0 + (RLE ? (uint32_t)tstart * (ACC8 ? 1u : 4u) : 0u), run = 0u;
    if constexpr (RLE) {
        // one vector per iteration, loads two vectors ahead; no per-vector
        // guard: the loads past a thread's last vector read the slack rows
        // at the end of the entry buffer (or another thread's vectors) and
        // are never added
        uint4 x0 = qa[0], x1 = qa[1];
        for (int32_t u = 0; u < nt; ++u) {
            const uint4 v = x0;
            x0 = x1;
            x1 = ld_stream_v4(col + (size_t)(u + 2) * kTiledThreads);
            rle_vector<EB, ACC8>(Esm, v, db, cur, run, s.flags, tl.part_words + 4, acc0, tl.acc_words * 4);
        }
        // the last target of the run (the dummy slot for an empty run)
#ifdef SNP_CHECK_BOUNDS
        if ((int32_t)(cur - acc0) >= tl.acc_words * 4) {
            atomicOr(s.flags + kFlagBounds, 1u << 2);
            cur = acc0;
        }
#endif
        if constexpr (ACC8)
            st_shared_u8(cur, run);
        else
            st_shared_u32(cur, run);
        __syncthreads();
        return kPhaseOk;
    }
    // two batches in flight: the next batch loads while this one is added
    int k = 0;
    while (k + 1 < kTiledMaxSub && s0 >= wb[k + 1]) ++k;
    for (int32_t u = 0;;) {
        load_batch(qb, col, u + D, nt);
        gather_batch<EB, LAYOUT, D>(qa, u, nt, s0, wb, k, Esm, acc0, db, wmask, sbits, cur, run);
        u += D;
        if (u >= nt) break;
        load_batch(qa, col, u + D, nt);
        gather_batch<EB, LAYOUT, D>(qb, u, nt, s0, wb, k, Esm, acc0, db, wmask, sbits, cur, run);
        u += D;
        if (u >= nt) break;
    }
    if (LAYOUT != kLayoutRuns) red_add_if(cur, run, run != 0u);
    __syncthreads();
    return kPhaseOk;
}

// Two-launch form (partitions P > kTiledMaxCluster): the gather writes
// partition h's in-flow of step kg to tl.inflow; k_tiled_select sums them.
template <int EB, int LAYOUT>
__global__ void __launch_bounds__(1024, 1) k_tiled_gather(DevSys s, TiledSys tl, int32_t t) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ int32_t wb[kTiledMaxSub + 1];
    __shared__ __align__(8) unsigned long long bar;
    uint32_t* Esm = smem;                                              // part_words + a zero word
    int* acc = reinterpret_cast<int*>(smem + tl.part_words + 4);
    unsigned long long kg;
    if (tiled_gather_phase<EB, LAYOUT>(s, tl, t, Esm, acc, wb, &bar, kg) != kPhaseOk) return;
    const int range = blockIdx.x / tl.P, h = blockIdx.x % tl.P;
    const int32_t lo = __ldg(tl.cta_lo + range), hi = __ldg(tl.cta_lo + range + 1);
    const int32_t slot0 = lo * kSlice;
    const int32_t nloc = (hi - lo) * kSlice;  // a multiple of 32
    uint4* out = reinterpret_cast<uint4*>(tl.inflow + (size_t)h * s.nslices * kSlice + slot0);
    const uint4* a4 = reinterpret_cast<const uint4*>(acc);
    for (int j = threadIdx.x; j < nloc / 4; j += blockDim.x) out[j] = a4[j];
}

// ---- thread-block clusters ----------------------------------------------
// All threads of every CTA of the cluster arrive; writes to shared memory
// before it are visible to every CTA of the cluster after it.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Address of the same shared-memory location in CTA `rank` of the cluster
// (a pure function of its operands: offsets within a CTA's shared memory are
// kept, so one mapped base serves a whole array).
__device__ __forceinline__ uint32_t cluster_map(uint32_t a, uint32_t rank) {
    uint32_t r;
    asm("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
    return r;
}
// This CTA's rank in its cluster.
__device__ __forceinline__ uint32_t cluster_rank() {
    uint32_t r;
    asm("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
// Volatile, so it stays after the cluster barrier (also volatile) that
// publishes what it reads; no memory clobber, so ordinary loads and stores
// around it are scheduled freely.
__device__ __forceinline__ uint32_t ld_cluster_u32(uint32_t a) {
    uint32_t v;
    asm volatile("ld.shared::cluster.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}

__device__ __forceinline__ uint4 ld_cluster_v4(uint32_t a) {
    uint4 v;
    asm volatile("ld.shared::cluster.v4.u32 {%0, %1, %2, %3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
                 : "r"(a));
    return v;
}

// Finish of step kg and select of step kg+1 for one slice, from its in-flow.
template <int SEL, int EB>
__device__ __forceinline__ void finish_select_slice(const DevSys& s, bool select, bool compact, int32_t* Sk,
                                                    uint32_t* Ek, int32_t slice, int lane, int32_t c, uint32_t st,
                                                    const uint4& rec, long long in, unsigned long long ks,
                                                    bool& active) {
    const int32_t slot = slice * kSlice + lane;
    const bool valid = slot < s.q;
    if (valid && (st >> kPendShift) == 0u) {
        const long long nc = (long long)c + in;
        if (nc > 2147483647ll) {
            atomicOr(s.flags + kFlagOverflow, 1u);
            c = 2147483647;
        } else {
            c = (int32_t)nc;
        }
    }
    uint32_t emit = 0u;
    if (select && valid) {
        const uint32_t nid = neuron_id(s, slot);
        SelOut o;
        if (s.rec)
            o = select_compiled<SEL, true>(rec, c, st, ks, nid, s.seed, s.philox_rk);
        else if (compact)
            o = select_neuron<true, SEL>(s.rules, rule_lo(s, slot), rule_hi(s, slot), c, st, ks, nid, s.seed);
        else
            o = select_neuron<false, SEL>(s.rules, rule_lo(s, slot), rule_hi(s, slot), c, st, ks, nid, s.seed);
        c = o.c_after;
        active |= o.active;
        emit = (uint32_t)o.emit;
        Sk[slot] = o.s;
        if (o.st != st) s.st[slot] = o.st;  // most neurons stay open: skip the write
    }
    if (valid) s.C[slot] = c;
    if (select) pk_put_slice<EB>(Ek, slice, lane, emit);
}

// ---- select phase of the fused step, four slots per lane ----------------
// A warp takes 128 consecutive slots of the CTA's share at a time, lane l
// slots 4l .. 4l+3: C, the status words, the spiking vector and the in-flow
// move as 16-byte vectors, the compiled records as four 16-byte loads, and
// the lane packs its four emissions into 4 x EB bits.  The in-flow of a
// slot is at most (in-degree x largest p) <= INT32_MAX (checked when the
// tiled layout is built), so it and C + in-flow are exact in 32 bits.

// Split cluster barrier: arrive (release) and wait (acquire) apart, so a CTA
// can announce that it started and later check that its partner did.
__device__ __forceinline__ void cluster_arrive_relaxed() {
    asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void st_cluster_v4(uint32_t a, const uint4& v) {
    asm volatile("st.shared::cluster.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(a), "r"(v.x), "r"(v.y), "r"(v.z),
                 "r"(v.w)
                 : "memory");
}

// One SNP step in one launch (partitions P <= kTiledMaxCluster): the P CTAs
// of a slice range form a thread-block cluster.  Each gathers its partition
// into its shared accumulators; then every CTA finishes step kg and selects
// step kg+1 (SELECT) for its share of the range, the in-flow of a slot being
// the sum of the P accumulators.
//  * With a partner buffer (tl.rin_words > 0): after its gather a CTA
//    stores its accumulators of each partner's share into that partner's
//    in-flow buffer through distributed shared memory -- byte accumulators:
//    into the segment the partner keeps for this CTA; 32-bit accumulators
//    (two partitions): the whole buffer -- and one cluster barrier publishes
//    them; the select phase then reads only its own shared memory, so no
//    barrier follows it.  A CTA announces at its start that it runs (the
//    buffer it writes into exists), and checks the partners' announcements
//    before its remote stores.
//  * Otherwise the select phase reads the other CTAs' accumulators through
//    distributed shared memory between two cluster barriers.
// ---- the select phase of four consecutive slots of one lane -------------
// Same results as select_compiled, slot by slot, for systems with compiled
// rule records: finishes step k for the four slots (an open neuron receives
// its in-flow; a count above INT32_MAX is clamped and reported in ovf) and
// selects step k+1.  Written for instruction count, since the select phase
// issues most of the fused step's instructions outside the gather:
//  * the applicability mask is one table lookup: entry e of the record's
//    fourteen 4-bit masks sits in word x (e < 8) or y (e >= 8) at bit
//    4e mod 32, so one rotate of the right word finds it;
//  * the chosen rule's 16-bit (c, p, d) field is taken with one byte
//    permute of words z and w;
//  * Philox runs only when a slot has two or more applicable rules.  When
//    the four slots are the neurons 4g .. 4g+3 (quad_block: the system keeps
//    the caller's neuron order), one block at counter g serves all four
//    (philox_draw's word assignment), computed once per lane when any lane
//    of the warp draws; otherwise one drawing slot per lane per round, as
//    many rounds as the warp's busiest lane needs.  All 32 lanes call this
//    together: both branches are warp-uniform.
// Slots past the system's end arrive as c = 0, st = 0, in = 0 and a zero
// record: an open neuron with no applicable rule, which changes nothing.
// The lane's 4 x EB emission bits are returned in packed (slot j at EB * j).
template <int SEL, int EB, typename PT>
__device__ __forceinline__ void select_quad(const uint4 (&rec)[4], int4& c4, uint4& st4, const uint4& in4,
                                            const uint4& nid4, bool quad_block, const PhiloxHead& ph,
                                            const uint32_t* rk,
                                            const uint2* __restrict__ tab, const uint8_t* __restrict__ pick,
                                            int4& s4, PT& packed, bool& active, bool& dirty, bool& ovf) {
    uint32_t mask[4], need = 0u;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t st = (&st4.x)[j];
        const bool closed = (st >> kPendShift) != 0u;
        const uint32_t nc = (uint32_t)(&c4.x)[j] + (&in4.x)[j];
        ovf |= !closed && nc > 2147483647u;
        const uint32_t n = closed ? (uint32_t)(&c4.x)[j] : min(nc, 2147483647u);
        (&c4.x)[j] = (int32_t)n;
        const uint32_t y = rec[j].y, K = (y >> 24) & 15u, L = y >> 28;
        const uint32_t x = n - K;
        const uint2 mg = tab[L];
        const uint32_t r = x - (__umulhi(x, mg.x) >> mg.y) * L;  // x mod L when n >= K and L >= 2
        const uint32_t e = n < K ? n : K + (L > 1u ? r : 0u);
        const uint32_t w = e < 8u ? rec[j].x : y;
        mask[j] = closed ? 0u : __funnelshift_r(w, w, 4u * e) & 15u;
        if (SEL == SNP_SELECT_PHILOX) need |= ((mask[j] & (mask[j] - 1u)) != 0u ? 1u : 0u) << j;
    }
    uint32_t x0[4] = {0u, 0u, 0u, 0u};
    if (SEL == SNP_SELECT_PHILOX && quad_block) {
        if (__any_sync(0xffffffffu, need != 0u)) {
            const Philox4 w = philox_block(ph, nid4.x >> 2, rk);
            x0[0] = w.v[0];
            x0[1] = w.v[1];
            x0[2] = w.v[2];
            x0[3] = w.v[3];
        }
    } else if (SEL == SNP_SELECT_PHILOX) {
        while (__any_sync(0xffffffffu, need != 0u)) {
            const uint32_t j = need ? (uint32_t)__ffs(need) - 1u : 0u;
            const uint32_t nid = j == 0u ? nid4.x : j == 1u ? nid4.y : j == 2u ? nid4.z : nid4.w;
            const uint32_t v = philox_word(ph, nid, rk);
            x0[0] = (need & 1u) ? v : x0[0];
            x0[1] = (need & 3u) == 2u ? v : x0[1];
            x0[2] = (need & 7u) == 4u ? v : x0[2];
            x0[3] = need == 8u ? v : x0[3];
            need &= need - 1u;
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t st = (&st4.x)[j];
        const uint32_t pend = st >> kPendShift;
        const bool closed = pend != 0u;
        const bool completing = closed && (st & kDMask) == 0u;
        const uint32_t m = mask[j];
        const bool selected = m != 0u;
        const uint32_t idx = SEL == SNP_SELECT_PHILOX && (m & (m - 1u)) != 0u
                                 ? (uint32_t)(((unsigned long long)x0[j] * (uint32_t)__popc(m)) >> 32)
                                 : 0u;  // < popc <= 4
        const uint32_t t = pick[m | (idx << 4)];
        const uint32_t fi = completing ? pend - 1u : t;
        const uint32_t f = __byte_perm(rec[j].z, rec[j].w, fi * 0x22u + 0x10u);  // bytes 2fi, 2fi+1
        const uint32_t c = f & 63u, p = (f >> 6) & 31u, d = (f >> 11) & 31u;
        const int32_t n = (&c4.x)[j];
        (&s4.x)[j] = selected ? (int32_t)t : -1;
        (&c4.x)[j] = selected ? n - (int32_t)c : n;
        const uint32_t emit = (completing || (selected && d == 0u)) ? p : 0u;
        const uint32_t nst = closed ? (completing ? 0u : st - 1u)
                                    : ((selected && d > 0u) ? ((t + 1u) << kPendShift) | (d - 1u) : 0u);
        active |= closed || selected;
        dirty |= nst != st;
        (&st4.x)[j] = nst;
        packed |= (PT)emit << (EB * j);
    }
}

template <int EB, int LAYOUT, int SEL>
__global__ void __launch_bounds__(1024, 1) k_tiled_step(DevSys s, TiledSys tl, int32_t t, int select, int compact) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ int32_t wb[kTiledMaxSub + 1];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ uint2 s_mod[16];    // constants of x / L for the compiled masks
    __shared__ uint8_t s_pick[64];  // the idx-th applicable rule of a mask
    fill_mod_table(s_mod);          // both published by the gather phase's barriers
    fill_pick_table(s_pick);
    const bool push = tl.rin_words > 0;  // in-flows pushed to the share's owner (uniform)
    // the partner buffer in the emissions' region: written only after every
    // gather of the cluster is done; otherwise beside the accumulators,
    // written as soon as the partners run
    const bool early = push && !tl.rin_esm;
    if (early) cluster_arrive_relaxed();  // this CTA runs: its shared memory may be written
    uint32_t* Esm = smem;
    int* acc = reinterpret_cast<int*>(smem + tl.part_words + 4);
    int* rin = tl.rin_esm ? reinterpret_cast<int*>(smem) : acc + tl.acc_words;  // the partners' in-flows (push)
    const int range = blockIdx.x / tl.P, h = blockIdx.x % tl.P;
    const int32_t lo = __ldg(tl.cta_lo + range), hi = __ldg(tl.cta_lo + range + 1);
    const int32_t share = (hi - lo + tl.P - 1) / tl.P;
    const int32_t my_lo = min(hi, lo + h * share), my_hi = min(hi, lo + (h + 1) * share);
    if (threadIdx.x == 32) {
        // the select phase reads C, the status words and the compiled records
        // of this CTA's share: ask L2 for them now, while the gather runs
        const int32_t a = my_lo * kSlice, b = min(s.q, my_hi * kSlice);
        const uint64_t nb = b > a ? (uint64_t)(b - a) * 4u & ~(uint64_t)15 : 0u;
        if (nb) {
            prefetch_l2_range(reinterpret_cast<const char*>(s.C + a), nb);
            prefetch_l2_range(reinterpret_cast<const char*>(s.st + a), nb);
            if (s.rec) prefetch_l2_range(reinterpret_cast<const char*>(s.rec) + (size_t)a * 16u, nb * 4u);
        }
    }
    unsigned long long kg;
    const int ph = tiled_gather_phase<EB, LAYOUT>(s, tl, t, Esm, acc, wb, &bar, kg);
    if (ph == kPhaseBlocked) {  // the same answer in every CTA of the cluster
        if (early) cluster_wait();  // complete the start barrier's phase before leaving
        return;
    }
    const uint32_t acc0 = smem_u32(acc);
    const uint32_t me = cluster_rank();
    constexpr bool ACC8 = LAYOUT == kLayoutRle8;
    const int32_t seg_bytes = share * kSlice;  // byte accumulators: one sender's segment of a buffer
    if (push && ACC8) {
        if (early)
            cluster_wait();  // the partners run
        else
            cluster_sync();  // every gather of the cluster is done: the emissions' regions are free
        if (ph == kPhaseOk) {
            // this CTA's byte accumulators of each partner's share, into this
            // CTA's segment of that partner's buffer
            const uint8_t* acc8 = reinterpret_cast<const uint8_t*>(acc);
            for (int r = 0; r < tl.P; ++r) {
                if (r == h) continue;
                const int32_t p_lo = min(hi, lo + r * share), p_hi = min(hi, lo + (r + 1) * share);
                const int seg = h < r ? h : h - 1;
                const uint32_t rbase = cluster_map(smem_u32(rin), (uint32_t)r) + (uint32_t)(seg * seg_bytes);
                const int32_t n16 = (p_hi - p_lo) * (kSlice / 16);
                const int32_t a0 = (p_lo - lo) * kSlice;
                for (int32_t i = threadIdx.x; i < n16; i += blockDim.x)
                    st_cluster_v4(rbase + (uint32_t)i * 16u, *reinterpret_cast<const uint4*>(acc8 + a0 + 16 * i));
            }
        }
    } else if (push) {
        cluster_wait();  // the partner runs
        if (ph == kPhaseOk) {
            // this CTA's accumulators of the partner's share, into its buffer
            const int hp = h ^ 1;
            const int32_t p_lo = min(hi, lo + hp * share), p_hi = min(hi, lo + (hp + 1) * share);
            const uint32_t rbase = cluster_map(smem_u32(rin), me ^ 1u);
            const int32_t n4 = (p_hi - p_lo) * (kSlice / 4);
            const int32_t a0 = (p_lo - lo) * kSlice;
            for (int32_t i = threadIdx.x; i < n4; i += blockDim.x)
                st_cluster_v4(rbase + (uint32_t)i * 16u, *reinterpret_cast<const uint4*>(acc + a0 + 4 * i));
        }
    }
    cluster_sync();
    const unsigned long long ks = kg + 1ull;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const bool has_rec = s.rec != nullptr;
    bool active = false;
    if (ph == kPhaseOk) {
        if (threadIdx.x == 32) {
            // this CTA's entry words are read again by the next step: ask L2
            // for them while the select phase leaves memory bandwidth idle
            const int32_t* subg = tl.sub + (size_t)blockIdx.x * (kTiledMaxSub + 1);
            const int64_t b0 = __ldg(subg) / 4, b1 = __ldg(subg + kTiledMaxSub) / 4;
            if (b1 > b0) prefetch_l2_range(reinterpret_cast<const char*>(tl.ent) + b0 * 16, (uint64_t)(b1 - b0) * 16);
        }
        int32_t* const Sk = SNP_PICK(s.S, ks);
        uint32_t* const Ek = SNP_PICK(tl.Eg, ks);
        // the partner's accumulators when they are read remotely (two CTAs
        // without the buffer), mapped once
        const uint32_t pbase = (!push && tl.P == 2) ? cluster_map(acc0, me ^ 1u) : 0u;
        const int32_t share_end = my_hi * kSlice;   // this CTA's share: slots [my_lo * 32, share_end)
        const int32_t qend = min(share_end, s.q);
        const PhiloxHead phx = philox_head(ks, s.philox_rk);
        // a warp takes 128 slots at a time, lane l slots 4l .. 4l+3 (one
        // 32-slot slice never straddles the share's bounds)
        for (int32_t base = my_lo * kSlice + warp * 128; base < share_end; base += nw * 128) {
            const int32_t slot0 = base + 4 * lane;
            const bool mine = slot0 < share_end;
            const bool live = slot0 < qend;
            int4 c4 = make_int4(0, 0, 0, 0);
            uint4 st4 = make_uint4(0u, 0u, 0u, 0u), in4 = st4;
            const uint4* rp = reinterpret_cast<const uint4*>(s.rec) + slot0;
            if (live && ACC8) {
                c4 = *reinterpret_cast<const int4*>(s.C + slot0);
                st4 = *reinterpret_cast<const uint4*>(s.st + slot0);
                // four byte accumulators per word: even and odd bytes summed
                // in 16-bit halves (at most 8 x 255 each)
                const uint8_t* acc8 = reinterpret_cast<const uint8_t*>(acc);
                const uint8_t* rin8 = reinterpret_cast<const uint8_t*>(rin);
                const uint32_t ow = *reinterpret_cast<const uint32_t*>(
                    acc8 + SNP_IDX(s.flags, 2, slot0 - lo * kSlice, tl.acc_words * 4 - 3));
                uint32_t ev = ow & 0x00FF00FFu, od = (ow >> 8) & 0x00FF00FFu;
                for (int r = 0; r + 1 < tl.P; ++r) {
                    const uint32_t w =
                        *reinterpret_cast<const uint32_t*>(rin8 + r * seg_bytes + (slot0 - my_lo * kSlice));
                    ev += w & 0x00FF00FFu;
                    od += (w >> 8) & 0x00FF00FFu;
                }
                in4 = make_uint4(ev & 0xFFFFu, od & 0xFFFFu, ev >> 16, od >> 16);
            } else if (live) {
                c4 = *reinterpret_cast<const int4*>(s.C + slot0);
                st4 = *reinterpret_cast<const uint4*>(s.st + slot0);
                const int32_t li = (int32_t)SNP_IDX(s.flags, 2, slot0 - lo * kSlice, tl.acc_words - 3);
                in4 = *reinterpret_cast<const uint4*>(acc + li);
                uint4 pv = make_uint4(0u, 0u, 0u, 0u);
                if (push) {
                    pv = *reinterpret_cast<const uint4*>(rin + (slot0 - my_lo * kSlice));
                } else if (tl.P == 2) {
                    pv = ld_cluster_v4(pbase + (uint32_t)li * 4u);
                } else {
                    for (int r = 0; r < tl.P; ++r) {
                        if ((uint32_t)r == me) continue;
                        const uint4 rv = ld_cluster_v4(cluster_map(acc0 + (uint32_t)li * 4u, (uint32_t)r));
                        pv.x += rv.x;
                        pv.y += rv.y;
                        pv.z += rv.z;
                        pv.w += rv.w;
                    }
                }
                in4.x += pv.x;
                in4.y += pv.y;
                in4.z += pv.z;
                in4.w += pv.w;
            }
            using PT = typename std::conditional<EB == 16, unsigned long long, uint32_t>::type;
            PT packed = 0u;
            int4 s4 = make_int4(-1, -1, -1, -1);
            bool dirty = false, ovf = false;
            if (has_rec && select) {  // warp-uniform
                const int32_t nv = qend - slot0;  // the lane's slots inside the system (<= 0: none)
                uint4 rq[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) rq[j] = j < nv ? __ldg(rp + j) : make_uint4(0u, 0u, 0u, 0u);
                if (nv < 4) {  // the system's last quad, or past its end
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        if (j >= nv) {
                            (&c4.x)[j] = 0;
                            (&st4.x)[j] = 0u;
                            (&in4.x)[j] = 0u;
                        }
                    }
                }
                uint4 nid4 = make_uint4((uint32_t)slot0, (uint32_t)slot0 + 1u, (uint32_t)slot0 + 2u,
                                        (uint32_t)slot0 + 3u);
                if (!s.identity) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) (&nid4.x)[j] = j < nv ? (uint32_t)__ldg(s.orig + slot0 + j) : 0u;
                }
                select_quad<SEL, EB, PT>(rq, c4, st4, in4, nid4, s.identity, phx, s.philox_rk, s_mod, s_pick, s4,
                                         packed, active, dirty, ovf);
            } else {
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int32_t slot = slot0 + j;
                    const bool v = slot < qend;
                    int32_t c = (&c4.x)[j];
                    const uint32_t st = (&st4.x)[j];
                    // an open neuron receives; a count above INT32_MAX is clamped
                    // and reported
                    const uint32_t nc = (uint32_t)c + (&in4.x)[j];
                    const bool open = v && (st >> kPendShift) == 0u;
                    ovf |= open && nc > 2147483647u;
                    c = open ? (int32_t)min(nc, 2147483647u) : c;
                    if (select && v) {
                        const uint32_t nid = neuron_id(s, slot);
                        SelOut o;
                        if (has_rec)
                            o = select_rec_flat<SEL>(__ldg(rp + j), c, st, nid, phx, s.philox_rk, s_mod, s_pick);
                        else if (compact)
                            o = select_neuron<true, SEL>(s.rules, rule_lo(s, slot), rule_hi(s, slot), c, st, ks, nid,
                                                         s.seed);
                        else
                            o = select_neuron<false, SEL>(s.rules, rule_lo(s, slot), rule_hi(s, slot), c, st, ks, nid,
                                                          s.seed);
                        c = o.c_after;
                        active |= o.active;
                        packed |= (PT)(uint32_t)o.emit << (EB * j);
                        (&s4.x)[j] = o.s;
                        dirty |= o.st != st;
                        (&st4.x)[j] = o.st;
                    }
                    (&c4.x)[j] = c;
                }
            }
            if (__any_sync(0xffffffffu, ovf) && lane == 0) atomicOr(s.flags + kFlagOverflow, 1u);
            if (live) {
                *reinterpret_cast<int4*>(s.C + slot0) = c4;
                if (select) {
                    *reinterpret_cast<int4*>(Sk + slot0) = s4;
                    if (dirty) *reinterpret_cast<uint4*>(s.st + slot0) = st4;  // most quads stay open
                }
            }
            if (select) {  // the lane's 4 x EB bits into the packed E_{k+1}
                if constexpr (EB == 2) {
                    uint32_t w = (uint32_t)packed << (8u * (uint32_t)(lane & 3));
                    w |= __shfl_xor_sync(0xffffffffu, w, 1);
                    w |= __shfl_xor_sync(0xffffffffu, w, 2);
                    if (mine && (lane & 3) == 0) Ek[slot0 >> 4] = w;
                } else if constexpr (EB == 4) {
                    uint32_t w = (uint32_t)packed << (16u * (uint32_t)(lane & 1));
                    w |= __shfl_xor_sync(0xffffffffu, w, 1);
                    if (mine && (lane & 1) == 0) Ek[slot0 >> 3] = w;
                } else if constexpr (EB == 8) {
                    if (mine) Ek[slot0 >> 2] = (uint32_t)packed;
                } else {
                    if (mine) *reinterpret_cast<uint2*>(Ek + (slot0 >> 1)) =
                                  make_uint2((uint32_t)packed, (uint32_t)(packed >> 32));
                }
            }
        }
    }
    if (select) raise_step_activity(s.flags, ks, active);
    if (!push) cluster_sync();  // the other CTAs read this CTA's accumulators until here
}

// Finishes step kg (GATHER: adds the in-flow to open neurons) and selects
// step ks (SELECT); one warp per NS consecutive slices.  Launched as a
// programmatic dependent of the launch before it: the compiled rule records
// (constant) are loaded before grid_dependency_wait, and every load of the
// step is issued before the fixed-point test, whose flag read would
// otherwise add a round trip to memory in front of them.
template <bool GATHER, bool SELECT, bool COMPACT, int SEL, int EB, int NS>
__global__ void __launch_bounds__(256) k_tiled_select(DevSys s, TiledSys tl, int32_t t) {
    const int lane = threadIdx.x & 31;
    const int32_t sl0 = (int32_t)((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * NS;
    const bool has_rec = s.rec != nullptr;
    uint4 rec[NS];
#pragma unroll
    for (int j = 0; j < NS; ++j) {
        const int32_t slot = (sl0 + j) * kSlice + lane;
        rec[j] = make_uint4(0u, 0u, 0u, 0u);
        if (SELECT && has_rec && sl0 + j < s.nslices && slot < s.q)
            rec[j] = __ldg(reinterpret_cast<const uint4*>(s.rec) + slot);
    }

    if (SELECT && threadIdx.x == 0 && tl.ent_words > 0) {
        // the gather launch after this one streams the whole entry array;
        // this launch leaves memory bandwidth idle, so each CTA asks L2 for
        // a slice of it
        const uint64_t total = (uint64_t)tl.ent_words * 4u;
        const uint64_t per = (total / gridDim.x + 15u) & ~(uint64_t)15u;
        const uint64_t a = min(total, (uint64_t)blockIdx.x * per), b = min(total, a + per);
        if (b > a) prefetch_l2_range(reinterpret_cast<const char*>(tl.ent) + a, b - a);
    }

    grid_dependency_wait();
    uint32_t* fl = s.flags;
    const size_t pstride = (size_t)s.nslices * kSlice;
    int32_t c[NS];
    uint32_t st[NS];
    long long in[NS];
#pragma unroll
    for (int j = 0; j < NS; ++j) {
        const int32_t slot = (sl0 + j) * kSlice + lane;
        const bool valid = sl0 + j < s.nslices && slot < s.q;
        c[j] = valid ? s.C[slot] : 0;
        st[j] = valid ? s.st[slot] : 0u;
        in[j] = 0;
        if (GATHER && valid) {
            in[j] = tl.inflow[slot];
            if (tl.P > 1) in[j] += tl.inflow[pstride + slot];
        }
    }
    if (GATHER && tl.P > 2) {
        for (int h = 2; h < tl.P; ++h) {
#pragma unroll
            for (int j = 0; j < NS; ++j) {
                const int32_t slot = (sl0 + j) * kSlice + lane;
                if (sl0 + j < s.nslices && slot < s.q) in[j] += tl.inflow[(size_t)h * pstride + slot];
            }
        }
    }
    const unsigned long long kg = s.step[kStepBase] + (unsigned long long)t;
    const unsigned long long ks = GATHER ? kg + 1ull : kg;
    if (call_halted(fl)) return;
    allow_dependents();
    bool active = false;
#pragma unroll
    for (int j = 0; j < NS; ++j) {
        const int32_t slice = sl0 + j;
        if (slice >= s.nslices) break;  // warp-uniform
        const int32_t slot = slice * kSlice + lane;
        const bool valid = slot < s.q;
        int32_t cj = c[j];
        if (GATHER && valid && (st[j] >> kPendShift) == 0u) {
            const long long nc = (long long)cj + in[j];
            if (nc > 2147483647ll) {
                atomicOr(fl + kFlagOverflow, 1u);
                cj = 2147483647;
            } else {
                cj = (int32_t)nc;
            }
        }
        uint32_t emit = 0u;
        if (SELECT && valid) {
            const SelOut o = s.forced ? select_forced<COMPACT>(s, slot, cj, st[j])
                             : has_rec ? select_compiled<SEL>(rec[j], cj, st[j], ks, neuron_id(s, slot), s.seed)
                                     : select_neuron<COMPACT, SEL>(s.rules, rule_lo(s, slot), rule_hi(s, slot), cj,
                                                                   st[j], ks, neuron_id(s, slot), s.seed);
            cj = o.c_after;
            active |= o.active;
            emit = (uint32_t)o.emit;
            SNP_PICK(s.S, ks)[slot] = o.s;
            if (o.st != st[j]) s.st[slot] = o.st;  // most neurons stay open: skip the write
        }
        if (valid) s.C[slot] = cj;
        if (SELECT) pk_put_slice<EB>(SNP_PICK(tl.Eg, ks), slice, lane, emit);
    }
    if (SELECT) raise_step_activity(fl, ks, active);
}

// Launch with programmatic stream serialization: the kernel may start while
// the previous launch on the stream is finishing, and waits for it with
// grid_dependency_wait before touching anything that launch writes.
template <typename... P, typename... A>
static cudaError_t launch_dependent(void (*fn)(P...), unsigned grid, unsigned block, size_t smem, cudaStream_t st,
                                    A... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, args...);
}

template <int EB>
static cudaError_t launch_gather_eb(const DevSys& s, const TiledSys& tl, int32_t t, cudaStream_t st, size_t smem,
                                    int threads) {
    auto fn = tl.rle ? k_tiled_gather<EB, kLayoutRle>
                     : (tl.pairs ? k_tiled_gather<EB, kLayoutPairs> : k_tiled_gather<EB, kLayoutRuns>);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    (void)threads;
    return launch_dependent(fn, (unsigned)tl.G, (unsigned)kTiledThreads, smem, st, s, tl, t);
}

// One slice per warp: several slices per warp (more loads in flight per
// warp) measured slower on the 1M-neuron workload, as the registers they need
// lower the occupancy more than they add parallelism.
template <bool G, bool S, bool C, int SEL, int EB>
static cudaError_t launch_select_t(const DevSys& s, const TiledSys& tl, int32_t t, cudaStream_t st) {
    return launch_dependent(k_tiled_select<G, S, C, SEL, EB, 1>, (unsigned)((s.nslices + 7) / 8), 256u, 0, st, s, tl,
                            t);
}

// One fused step launch: clusters of P CTAs, programmatic dependent.
template <int EB, int SEL>
static cudaError_t launch_step_eb(const DevSys& s, const TiledSys& tl, int32_t t, cudaStream_t st, size_t smem,
                                  bool select, bool compact) {
    auto fn = tl.rle ? (tl.acc8 ? k_tiled_step<EB, kLayoutRle8, SEL> : k_tiled_step<EB, kLayoutRle, SEL>)
                     : (tl.pairs ? k_tiled_step<EB, kLayoutPairs, SEL> : k_tiled_step<EB, kLayoutRuns, SEL>);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)tl.G);
    cfg.blockDim = dim3((unsigned)kTiledThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[2];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    at[1].id = cudaLaunchAttributeClusterDimension;
    at[1].val.clusterDim.x = (unsigned)tl.P;
    at[1].val.clusterDim.y = 1;
    at[1].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 2;
    return cudaLaunchKernelEx(&cfg, fn, s, tl, t, select ? 1 : 0, compact ? 1 : 0);
}

template <int EB>
static cudaError_t launch_tiled_eb(const DevSys& s, const TiledSys& tl, int kind, int32_t t, cudaStream_t st,
                                   bool compact, int sel, size_t smem, int threads) {
    if (kind != kPullSelectOnly && tl.P <= kTiledMaxCluster) {
        const bool select = kind == kPullFused;
        return sel == SNP_SELECT_FIRST ? launch_step_eb<EB, SNP_SELECT_FIRST>(s, tl, t, st, smem, select, compact)
                                       : launch_step_eb<EB, SNP_SELECT_PHILOX>(s, tl, t, st, smem, select, compact);
    }
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

// How many thread-block clusters of P CTAs (1,024 threads, smem bytes of
// dynamic shared memory each) the device runs at once: clusters must fit
// inside one GPC, so this can be below the SM count / P.  0 on failure.
int tiled_clusters_per_wave(int P, size_t smem) {
    auto fn = k_tiled_step<2, kLayoutRle8, SNP_SELECT_PHILOX>;
    if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)P);
    cfg.blockDim = dim3((unsigned)kTiledThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)P;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int n = 0;
    if (cudaOccupancyMaxActiveClusters(&n, (const void*)fn, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return n;
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
