// Device helpers shared by the step kernels: rule decoding, the regular
// expression test, the counter-based generator and the per-neuron select.
#pragma once

#include <cstdint>

#include "snp_internal.h"

namespace snp {

// ---- Philox4x32-10 ------------------------------------------------------
// Counter-based generator of Salmon, Moraes, Dror and Shaw ("Parallel Random
// Numbers: As Easy as 1, 2, 3", SC'11).  Ten rounds; each round takes the
// 32x32 -> 64-bit products of words 0 and 2 with two fixed odd multipliers,
// and the new words are (hi(B*x2) ^ x1 ^ key0, lo(B*x2), hi(A*x0) ^ x3 ^ key1,
// lo(A*x0)).  Between rounds the key advances by two Weyl increments.
struct Philox4 {
    uint32_t v[4];
};

__device__ __forceinline__ Philox4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                 uint32_t key0, uint32_t key1) {
    constexpr uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
    constexpr uint32_t kBumpA = 0x9E3779B9u, kBumpB = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hiA = __umulhi(kMulA, c0), loA = kMulA * c0;
        const uint32_t hiB = __umulhi(kMulB, c2), loB = kMulB * c2;
        const uint32_t n0 = hiB ^ c1 ^ key0;
        const uint32_t n2 = hiA ^ c3 ^ key1;
        c0 = n0;
        c1 = loB;
        c2 = n2;
        c3 = loA;
        key0 += kBumpA;
        key1 += kBumpB;
    }
    Philox4 out;
    out.v[0] = c0;
    out.v[1] = c1;
    out.v[2] = c2;
    out.v[3] = c3;
    return out;
}

// ---- rules ----------------------------------------------------------------
struct RuleF {
    int32_t k, j, c, p, d;
};

template <bool COMPACT>
__device__ __forceinline__ RuleF load_rule(const uint32_t* __restrict__ rules, int32_t r) {
    RuleF f;
    if (COMPACT) {
        const uint32_t w = __ldg(rules + r);
        f.k = (int32_t)(w & 255u);
        f.j = (int32_t)((w >> 8) & 255u);
        f.c = (int32_t)((w >> 16) & 255u);
        f.p = (int32_t)((w >> 24) & 15u);
        f.d = (int32_t)(w >> 28);
    } else {
        const uint4 w = __ldg(reinterpret_cast<const uint4*>(rules) + r);
        f.k = (int32_t)w.x;
        f.j = (int32_t)w.y;
        f.c = (int32_t)w.z;
        f.p = (int32_t)(w.w & 0xffffu);
        f.d = (int32_t)(w.w >> 16);
    }
    return f;
}

// The regular expression a^k (a^j)* matches n spikes, and n covers c
// (Sec. 2 types 1-3 and the type-4 form of Sec. 7).
__device__ __forceinline__ bool rule_applies(int32_t n, const RuleF& f) {
    if (n < f.k || n < f.c) return false;
    if (f.j == 0) return n == f.k;
    if (f.j == 1) return true;
    return ((uint32_t)(n - f.k) % (uint32_t)f.j) == 0u;
}

// Result of the select phase of one neuron for one step.
struct SelOut {
    int32_t c_after;  // spikes after consumption
    uint32_t st;      // status word after the step's delay update
    int32_t emit;     // spikes sent along every synapse this step
    int32_t s;        // local index of the selected rule, -1 = none
    bool active;      // pending or selected: the system is not at a fixed point
};

// Select phase of neuron `slot` (caller's id `nid`) at absolute step k:
// completes a pending delayed rule, or counts down a closed neuron, or picks
// one applicable rule (first or Philox-uniform) and consumes its spikes.
// The status word already carries the end-of-step decrement (UPDATE_DELAYS).
template <bool COMPACT, int SEL>
__device__ __forceinline__ SelOut select_neuron(const uint32_t* __restrict__ rules, int32_t r0, int32_t r1,
                                                int32_t n, uint32_t st, unsigned long long k, uint32_t nid,
                                                uint64_t seed) {
    SelOut o;
    o.c_after = n;
    o.emit = 0;
    o.s = -1;
    const uint32_t pend = st >> kPendShift;
    if (pend != 0u) {
        o.active = true;
        if ((st & kDMask) == 0u) {  // the delayed rule fires now; neuron reopens
            o.emit = load_rule<COMPACT>(rules, r0 + (int32_t)pend - 1).p;
            o.st = 0u;
        } else {                    // still closed
            o.st = st - 1u;
        }
        return o;
    }
    o.st = 0u;
    o.active = false;
    int32_t pick = -1;
    if (SEL == SNP_SELECT_FIRST) {
        for (int32_t r = r0; r < r1; ++r) {
            if (rule_applies(n, load_rule<COMPACT>(rules, r))) {
                pick = r;
                break;
            }
        }
    } else {
        int32_t cnt = 0, first = -1;
        for (int32_t r = r0; r < r1; ++r) {
            if (rule_applies(n, load_rule<COMPACT>(rules, r))) {
                if (cnt == 0) first = r;
                ++cnt;
            }
        }
        if (cnt == 1) {
            pick = first;
        } else if (cnt > 1) {
            const Philox4 x = philox4x32_10((uint32_t)k, nid, (uint32_t)(k >> 32), 0u, (uint32_t)seed,
                                            (uint32_t)(seed >> 32));
            int32_t idx = (int32_t)(((unsigned long long)x.v[0] * (unsigned long long)cnt) >> 32);
            for (int32_t r = first; r < r1; ++r) {
                if (rule_applies(n, load_rule<COMPACT>(rules, r))) {
                    if (idx == 0) {
                        pick = r;
                        break;
                    }
                    --idx;
                }
            }
        }
    }
    if (pick >= 0) {
        const RuleF f = load_rule<COMPACT>(rules, pick);
        o.active = true;
        o.s = pick - r0;
        o.c_after = n - f.c;
        if (f.d == 0) {
            o.emit = f.p;
        } else {
            o.st = ((uint32_t)(o.s + 1) << kPendShift) | (uint32_t)(f.d - 1);
        }
    }
    return o;
}

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) {
    return *reinterpret_cast<const volatile uint32_t*>(p);
}

}  // namespace snp
