// Device helpers shared by the step kernels: rule decoding, the regular
// expression test, the counter-based generator and the per-neuron select.
#pragma once

#include <cstdint>

#include "snp_internal.h"

// One of two buffers by step parity.  A ternary, not arr[k & 1]: indexing a
// kernel-parameter array with a run-time value makes every thread copy the
// parameter block into local memory.
#define SNP_PICK(arr, k) ((((k) & 1ull) != 0ull) ? (arr)[1] : (arr)[0])

namespace snp {

// ---- bounds-checked builds -----------------------------------------------
// Built with SNP_CHECK_BOUNDS, every index passed through SNP_IDX is compared
// with its limit; an index outside [0, limit) is replaced by 0, so the access
// stays inside its buffer, and bit `site` is OR-ed into the system's
// kFlagBounds word, which snp_step reports as SNP_ERR_INVALID.  Built
// without it SNP_IDX is the index itself.  Sites: 0 an in-list entry's
// emission index, 1 a packed emission word in shared memory, 2 a shared
// accumulator, 3 a push target, 4 an ELL (rule, p) pair's rule.
#ifdef SNP_CHECK_BOUNDS
__device__ __forceinline__ long long snp_idx(uint32_t* flags, int site, long long i, long long limit) {
    if (i < 0 || i >= limit) {
        atomicOr(flags + kFlagBounds, 1u << site);
        return 0;
    }
    return i;
}
#define SNP_IDX(flags, site, i, limit) (::snp::snp_idx((flags), (site), (long long)(i), (long long)(limit)))
#else
#define SNP_IDX(flags, site, i, limit) (i)
#endif

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
        const unsigned long long pA = (unsigned long long)kMulA * c0;  // one wide multiply each
        const unsigned long long pB = (unsigned long long)kMulB * c2;
        const uint32_t hiA = (uint32_t)(pA >> 32), loA = (uint32_t)pA;
        const uint32_t hiB = (uint32_t)(pB >> 32), loB = (uint32_t)pB;
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

// The same generator with the ten round keys given (rk[2r], rk[2r+1] = the
// key after r Weyl increments, see philox_round_keys): kernels that take the
// keys from their parameter block read them as constant operands.
__device__ __forceinline__ Philox4 philox4x32_10_rk(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                    const uint32_t* rk) {
    constexpr uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long pA = (unsigned long long)kMulA * c0;
        const unsigned long long pB = (unsigned long long)kMulB * c2;
        const uint32_t n0 = (uint32_t)(pB >> 32) ^ c1 ^ rk[2 * r];
        const uint32_t n2 = (uint32_t)(pA >> 32) ^ c3 ^ rk[2 * r + 1];
        c0 = n0;
        c1 = (uint32_t)pB;
        c2 = n2;
        c3 = (uint32_t)pA;
    }
    Philox4 out;
    out.v[0] = c0;
    out.v[1] = c1;
    out.v[2] = c2;
    out.v[3] = c3;
    return out;
}

// The uniform 32-bit word a neuron draws its choice from (SAMPLE_ONE of
// Sec. 5 picks uniformly among the applicable rules; the generator is this
// library's choice): the four words of one Philox4x32-10 block at counter
// (k mod 2^32, nid / 4, k >> 32, 0) go to the four neurons 4(nid / 4) ..
// 4(nid / 4) + 3, neuron nid taking word nid mod 4 -- so four consecutive
// neurons can share one evaluation.
__device__ __forceinline__ uint32_t philox_word_of(const Philox4& x, uint32_t nid) {
    const uint32_t j = nid & 3u;
    return j == 0u ? x.v[0] : j == 1u ? x.v[1] : j == 2u ? x.v[2] : x.v[3];
}
__device__ __forceinline__ uint32_t philox_draw(unsigned long long k, uint32_t nid, uint64_t seed) {
    return philox_word_of(philox4x32_10((uint32_t)k, nid >> 2, (uint32_t)(k >> 32), 0u, (uint32_t)seed,
                                        (uint32_t)(seed >> 32)),
                          nid);
}
__device__ __forceinline__ uint32_t philox_draw_rk(unsigned long long k, uint32_t nid, const uint32_t* rk) {
    return philox_word_of(philox4x32_10_rk((uint32_t)k, nid >> 2, (uint32_t)(k >> 32), 0u, rk), nid);
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

// Divisibility by a small j without a division: for 32-bit x and j >= 2,
// j divides x exactly when x * c <= c - 1 modulo 2^64, c = floor((2^64-1)/j)
// + 1 (Lemire, Kaser and Kurz, "Faster remainder by direct computation",
// 2019).  The constants for j < 256 are built at compile time.
struct DivMagic {
    unsigned long long c[256];
    constexpr DivMagic() : c() {
        for (int j = 2; j < 256; ++j) c[j] = ~0ull / (unsigned long long)j + 1ull;
    }
};
__constant__ DivMagic kDivMagic = DivMagic();

__device__ __forceinline__ bool divides(uint32_t x, uint32_t j) {
    if ((j & (j - 1u)) == 0u) return (x & (j - 1u)) == 0u;  // j a power of two (incl. 1)
    if (j < 256u) {
        const unsigned long long c = kDivMagic.c[j];
        return (unsigned long long)x * c <= c - 1ull;
    }
    return x % j == 0u;
}

// The regular expression a^k (a^j)* matches n spikes, and n covers c
// (Sec. 2 types 1-3 and the type-4 form of Sec. 7).
__device__ __forceinline__ bool rule_applies(int32_t n, const RuleF& f) {
    if (n < f.k || n < f.c) return false;
    if (f.j == 0) return n == f.k;
    return divides((uint32_t)(n - f.k), (uint32_t)f.j);
}

// Rule r of a rule table applies to n spikes.  In the general (4-word)
// table a rule whose expression is a union of terms has the top bit of word
// 0 set: the low bits index its first (k, j) term record (8-byte units from
// the start of the table), word 1 counts its terms, and the rule applies
// when n >= c and n is in any term's language (see pack_union_rules).
template <bool COMPACT>
__device__ __forceinline__ bool rule_applies_at(const uint32_t* __restrict__ rules, int32_t r, int32_t n) {
    if (COMPACT) return rule_applies(n, load_rule<true>(rules, r));
    const uint4 w = __ldg(reinterpret_cast<const uint4*>(rules) + r);
    if ((w.x & 0x80000000u) == 0u) {
        RuleF f;
        f.k = (int32_t)w.x;
        f.j = (int32_t)w.y;
        f.c = (int32_t)w.z;
        f.p = 0;
        f.d = 0;
        return rule_applies(n, f);
    }
    if (n < (int32_t)w.z) return false;
    const uint2* term = reinterpret_cast<const uint2*>(rules) + (w.x & 0x7fffffffu);
    for (uint32_t u = 0; u < w.y; ++u) {
        const uint2 kj = __ldg(term + u);
        const int32_t k = (int32_t)kj.x;
        if (n >= k && (kj.y == 0u ? n == k : divides((uint32_t)(n - k), kj.y))) return true;
    }
    return false;
}

// Rule range of a slot and the caller's id of a slot.
__device__ __forceinline__ int32_t rule_lo(const DevSys& s, int32_t slot) {
    return s.rules_per_neuron > 0 ? slot * s.rules_per_neuron : __ldg(s.rule_off + slot);
}
__device__ __forceinline__ int32_t rule_hi(const DevSys& s, int32_t slot) {
    return s.rules_per_neuron > 0 ? (slot + 1) * s.rules_per_neuron : __ldg(s.rule_off + slot + 1);
}
__device__ __forceinline__ uint32_t neuron_id(const DevSys& s, int32_t slot) {
    return s.identity ? (uint32_t)slot : (uint32_t)__ldg(s.orig + slot);
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
    if (COMPACT && r1 - r0 <= 4) {
        // up to four one-word rules held in registers (one 16-byte load when
        // the neuron's four rules are 16-byte aligned); bit t of `mask` =
        // rule r0 + t applies
        const int32_t R = r1 - r0;
        uint32_t w0 = 0u, w1 = 0u, w2 = 0u, w3 = 0u;
        if (R == 4 && (r0 & 3) == 0) {
            const uint4 v = __ldg(reinterpret_cast<const uint4*>(rules) + (r0 >> 2));
            w0 = v.x;
            w1 = v.y;
            w2 = v.z;
            w3 = v.w;
        } else {
            if (R > 0) w0 = __ldg(rules + r0);
            if (R > 1) w1 = __ldg(rules + r0 + 1);
            if (R > 2) w2 = __ldg(rules + r0 + 2);
            if (R > 3) w3 = __ldg(rules + r0 + 3);
        }
        auto applies_w = [&](uint32_t w) {
            RuleF f;
            f.k = (int32_t)(w & 255u);
            f.j = (int32_t)((w >> 8) & 255u);
            f.c = (int32_t)((w >> 16) & 255u);
            return rule_applies(n, f);
        };
        uint32_t mask = 0u;
        if (R > 0 && applies_w(w0)) mask |= 1u;
        if (R > 1 && applies_w(w1)) mask |= 2u;
        if (R > 2 && applies_w(w2)) mask |= 4u;
        if (R > 3 && applies_w(w3)) mask |= 8u;
        if (mask == 0u) return o;
        if (SEL == SNP_SELECT_PHILOX && (mask & (mask - 1u)) != 0u) {
            const int32_t cnt = __popc(mask);
            const uint32_t x = philox_draw(k, nid, seed);
            int32_t idx = (int32_t)(((unsigned long long)x * (unsigned long long)cnt) >> 32);
            for (; idx > 0; --idx) mask &= mask - 1u;
        }
        const int32_t t = __ffs(mask) - 1;  // FIRST: the lowest applicable rule
        const uint32_t w = t == 0 ? w0 : t == 1 ? w1 : t == 2 ? w2 : w3;
        const int32_t c = (int32_t)((w >> 16) & 255u), p = (int32_t)((w >> 24) & 15u), d = (int32_t)(w >> 28);
        o.active = true;
        o.s = t;
        o.c_after = n - c;
        if (d == 0)
            o.emit = p;
        else
            o.st = ((uint32_t)(t + 1) << kPendShift) | (uint32_t)(d - 1);
        return o;
    }
    if (SEL == SNP_SELECT_FIRST) {
        for (int32_t r = r0; r < r1; ++r) {
            if (rule_applies_at<COMPACT>(rules, r, n)) {
                pick = r;
                break;
            }
        }
    } else if (r1 - r0 <= 32) {
        // one pass: bit i of `mask` = rule r0 + i applies; the draw picks
        // the idx-th set bit
        uint32_t mask = 0u;
        for (int32_t r = r0; r < r1; ++r)
            if (rule_applies_at<COMPACT>(rules, r, n)) mask |= 1u << (r - r0);
        const int32_t cnt = __popc(mask);
        if (cnt == 1) {
            pick = r0 + __ffs(mask) - 1;
        } else if (cnt > 1) {
            const uint32_t x = philox_draw(k, nid, seed);
            int32_t idx = (int32_t)(((unsigned long long)x * (unsigned long long)cnt) >> 32);
            for (; idx > 0; --idx) mask &= mask - 1u;  // drop the lowest set bits
            pick = r0 + __ffs(mask) - 1;
        }
    } else {
        int32_t cnt = 0, first = -1;
        for (int32_t r = r0; r < r1; ++r) {
            if (rule_applies_at<COMPACT>(rules, r, n)) {
                if (cnt == 0) first = r;
                ++cnt;
            }
        }
        if (cnt == 1) {
            pick = first;
        } else if (cnt > 1) {
            const uint32_t x = philox_draw(k, nid, seed);
            int32_t idx = (int32_t)(((unsigned long long)x * (unsigned long long)cnt) >> 32);
            for (int32_t r = first; r < r1; ++r) {
                if (rule_applies_at<COMPACT>(rules, r, n)) {
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

// ---- compiled rule records (see compile_rules) ---------------------------
// x / L for x < 2^31 and L in 2..15 by one high multiply (Granlund and
// Montgomery, PLDI 1994): with c = ceil(log2 L) and M = ceil(2^(31+c) / L),
// M < 2^32 and M*L - 2^(31+c) < L <= 2^c, so floor(x / L) = floor(x * M /
// 2^(31+c)) = umulhi(x, M) >> (c - 1) for every such x.  L = 1 is handled
// apart (x mod 1 = 0).
struct ModMagic32 {
    uint32_t m[16];
    uint32_t sh[16];
    constexpr ModMagic32() : m(), sh() {
        for (int l = 2; l < 16; ++l) {
            int c = 0;
            while ((1 << c) < l) ++c;
            m[l] = (uint32_t)((((unsigned long long)1 << (31 + c)) + (unsigned long long)l - 1ull) / (unsigned long long)l);
            sh[l] = (uint32_t)(c - 1);
        }
    }
};
__constant__ ModMagic32 kMod32 = ModMagic32();

// Applicable rules of an idle neuron with n spikes from its compiled record:
// bit t set when rule t applies (n indexes the table directly below K and
// by K + (n - K) mod L from K on).
__device__ __forceinline__ uint32_t compiled_mask(const uint4& rec, int32_t n) {
    const uint32_t K = (rec.y >> 24) & 15u, L = rec.y >> 28;
    uint32_t e = (uint32_t)n;
    if (e >= K) {
        const uint32_t x = e - K;
        const uint32_t qq = __umulhi(x, kMod32.m[L]) >> kMod32.sh[L];
        e = K + (L > 1u ? x - qq * L : 0u);
    }
    return e < 8u ? (rec.x >> (4u * e)) & 15u : (rec.y >> (4u * (e - 8u))) & 15u;
}

// The same with the constants of x / L read from a table in shared memory
// (tab[L] = {kMod32.m[L], kMod32.sh[L]}, see fill_mod_table): lanes with
// different L then read different words of one small table, where an
// indexed __constant__ read is serialised over the warp's distinct addresses.
__device__ __forceinline__ uint32_t compiled_mask_tab(const uint4& rec, int32_t n, const uint2* __restrict__ tab) {
    const uint32_t K = (rec.y >> 24) & 15u, L = rec.y >> 28;
    uint32_t e = (uint32_t)n;
    if (e >= K) {
        const uint32_t x = e - K;
        const uint2 mg = tab[L];
        const uint32_t qq = __umulhi(x, mg.x) >> mg.y;
        e = K + (L > 1u ? x - qq * L : 0u);
    }
    return e < 8u ? (rec.x >> (4u * e)) & 15u : (rec.y >> (4u * (e - 8u))) & 15u;
}

// Fills tab[0..15] for compiled_mask_tab (threads 0..15 of the block; the
// caller publishes it with a barrier).
__device__ __forceinline__ void fill_mod_table(uint2* tab) {
    const uint32_t l = threadIdx.x;
    if (l < 16u) tab[l] = l >= 2u ? make_uint2(kMod32.m[l], kMod32.sh[l]) : make_uint2(0u, 0u);
}

// The 16-bit (c, p, d) field of rule t of a compiled record.
__device__ __forceinline__ uint32_t compiled_field(const uint4& rec, uint32_t t) {
    return ((t < 2u ? rec.z : rec.w) >> (16u * (t & 1u))) & 0xffffu;
}

// RK: take the Philox round keys from rk (else derive them from seed).
// tab: the shared-memory table of compiled_mask_tab, or NULL.
template <int SEL, bool RK = false>
__device__ __forceinline__ SelOut select_compiled(const uint4 rec, int32_t n, uint32_t st, unsigned long long k,
                                                  uint32_t nid, uint64_t seed, const uint32_t* rk = nullptr,
                                                  const uint2* tab = nullptr) {
    SelOut o;
    o.c_after = n;
    o.emit = 0;
    o.s = -1;
    const uint32_t pend = st >> kPendShift;
    if (pend != 0u) {
        o.active = true;
        if ((st & kDMask) == 0u) {
            o.emit = (int32_t)((compiled_field(rec, pend - 1u) >> 6) & 31u);
            o.st = 0u;
        } else {
            o.st = st - 1u;
        }
        return o;
    }
    o.st = 0u;
    o.active = false;
    uint32_t mask = tab ? compiled_mask_tab(rec, n, tab) : compiled_mask(rec, n);
    if (mask == 0u) return o;
    if (SEL == SNP_SELECT_PHILOX && (mask & (mask - 1u)) != 0u) {
        const uint32_t cnt = (uint32_t)__popc(mask);
        const uint32_t x = RK ? philox_draw_rk(k, nid, rk) : philox_draw(k, nid, seed);
        const uint32_t idx = (uint32_t)(((unsigned long long)x * cnt) >> 32);  // < cnt <= 4
        // drop the idx lowest set bits, without a loop
        mask = idx > 0u ? mask & (mask - 1u) : mask;
        mask = idx > 1u ? mask & (mask - 1u) : mask;
        mask = idx > 2u ? mask & (mask - 1u) : mask;
    }
    const uint32_t t = (uint32_t)(__ffs(mask) - 1);
    const uint32_t f = compiled_field(rec, t);
    const int32_t c = (int32_t)(f & 63u), p = (int32_t)((f >> 6) & 31u), d = (int32_t)(f >> 11);
    o.active = true;
    o.s = (int32_t)t;
    o.c_after = n - c;
    if (d == 0)
        o.emit = p;
    else
        o.st = ((t + 1u) << kPendShift) | (uint32_t)(d - 1);
    return o;
}

// select_compiled without data-dependent branches except around the Philox
// draw (taken when any lane of the warp needs it): the pending, closed,
// idle and selecting cases are all computed and the result picked by
// selects, so the lanes of a warp stay converged.  Same results as
// select_compiled<SEL, true> with the round keys rk and the table tab.
template <int SEL>
__device__ __forceinline__ SelOut select_compiled_flat(const uint4 rec, int32_t n, uint32_t st, unsigned long long k,
                                                       uint32_t nid, const uint32_t* rk, const uint2* tab) {
    const uint32_t pend = st >> kPendShift;
    const bool closed = pend != 0u;
    const bool completing = closed && (st & kDMask) == 0u;
    uint32_t mask = closed ? 0u : compiled_mask_tab(rec, n, tab);
    if (SEL == SNP_SELECT_PHILOX) {
        const bool draw = (mask & (mask - 1u)) != 0u;
        if (__any_sync(__activemask(), draw)) {
            const uint32_t cnt = (uint32_t)__popc(mask);
            const uint32_t x = philox_draw_rk(k, nid, rk);
            uint32_t idx = draw ? (uint32_t)(((unsigned long long)x * cnt) >> 32) : 0u;  // < cnt <= 4
            mask = idx > 0u ? mask & (mask - 1u) : mask;
            mask = idx > 1u ? mask & (mask - 1u) : mask;
            mask = idx > 2u ? mask & (mask - 1u) : mask;
        }
    }
    const bool selected = mask != 0u;
    const uint32_t t = (uint32_t)(__ffs(mask) - 1);          // the chosen rule (FIRST: the lowest)
    const uint32_t f = compiled_field(rec, completing ? pend - 1u : t);
    const int32_t c = (int32_t)(f & 63u), p = (int32_t)((f >> 6) & 31u), d = (int32_t)(f >> 11);
    SelOut o;
    o.active = closed || selected;
    o.s = selected ? (int32_t)t : -1;
    o.c_after = selected ? n - c : n;
    o.emit = (completing || (selected && d == 0)) ? p : 0;
    o.st = closed ? (completing ? 0u : st - 1u)
                  : ((selected && d > 0) ? ((t + 1u) << kPendShift) | (uint32_t)(d - 1) : 0u);
    return o;
}

// ---- the select of one slot from its compiled record, for the fused step --
// Philox4x32-10 at counter (k mod 2^32, g, k >> 32, 0), g = nid / 4: only
// word 1 of the counter (the block) differs between the blocks of one step,
// so in rounds 1 to 3 most products and XORs are the same for every block.
// PhiloxHead holds those parts (computed once per step), philox_block
// finishes the ten rounds from them -- the same words as
// philox4x32_10_rk(k, g, k >> 32, 0, rk) -- and philox_word takes neuron
// nid's word of its block (philox_draw_rk's value).
struct PhiloxHead {
    uint32_t u1;    // round 1: c0 = u1 ^ g
    uint32_t u4k;   // round 2: c2 = hi(A c0) ^ u4k
    uint32_t u6k;   // round 3: c0 = hi(B c2) ^ u6k
    uint32_t w;     // round 3: c2 = w ^ lo(A c0 of round 2)
    uint32_t loA3;  // round 3: c3
};

__device__ __forceinline__ PhiloxHead philox_head(unsigned long long k, const uint32_t* rk) {
    constexpr uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
    const uint32_t k0 = (uint32_t)k, k1 = (uint32_t)(k >> 32);
    // round 1 on (k0, g, k1, 0)
    const unsigned long long pA1 = (unsigned long long)kMulA * k0, pB1 = (unsigned long long)kMulB * k1;
    const uint32_t u1 = (uint32_t)(pB1 >> 32) ^ rk[0];  // c0 = u1 ^ g
    const uint32_t u2 = (uint32_t)pB1;                   // c1
    const uint32_t u3 = (uint32_t)(pA1 >> 32) ^ rk[1];   // c2
    const uint32_t u4 = (uint32_t)pA1;                   // c3
    // round 2: B c2 does not depend on g
    const unsigned long long pB2 = (unsigned long long)kMulB * u3;
    const uint32_t u5 = (uint32_t)(pB2 >> 32) ^ u2 ^ rk[2];  // c0
    const uint32_t u6 = (uint32_t)pB2;                        // c1
    // round 3: A c0 does not depend on g
    const unsigned long long pA3 = (unsigned long long)kMulA * u5;
    PhiloxHead h;
    h.u1 = u1;
    h.u4k = u4 ^ rk[3];
    h.u6k = u6 ^ rk[4];
    h.w = (uint32_t)(pA3 >> 32) ^ rk[5];
    h.loA3 = (uint32_t)pA3;
    return h;
}

__device__ __forceinline__ Philox4 philox_block(const PhiloxHead& h, uint32_t g, const uint32_t* rk) {
    constexpr uint32_t kMulA = 0xD2511F53u, kMulB = 0xCD9E8D57u;
    // rounds 2 and 3: the parts that depend on g
    const unsigned long long pA2 = (unsigned long long)kMulA * (h.u1 ^ g);
    const uint32_t c2r2 = (uint32_t)(pA2 >> 32) ^ h.u4k, c3r2 = (uint32_t)pA2;
    const unsigned long long pB3 = (unsigned long long)kMulB * c2r2;
    uint32_t c0 = (uint32_t)(pB3 >> 32) ^ h.u6k, c1 = (uint32_t)pB3, c2 = h.w ^ c3r2, c3 = h.loA3;
#pragma unroll
    for (int r = 3; r < 10; ++r) {
        const unsigned long long pA = (unsigned long long)kMulA * c0;
        const unsigned long long pB = (unsigned long long)kMulB * c2;
        const uint32_t n0 = (uint32_t)(pB >> 32) ^ c1 ^ rk[2 * r];
        const uint32_t n2 = (uint32_t)(pA >> 32) ^ c3 ^ rk[2 * r + 1];
        c0 = n0;
        c1 = (uint32_t)pB;
        c2 = n2;
        c3 = (uint32_t)pA;
    }
    Philox4 out;
    out.v[0] = c0;
    out.v[1] = c1;
    out.v[2] = c2;
    out.v[3] = c3;
    return out;
}

__device__ __forceinline__ uint32_t philox_word(const PhiloxHead& h, uint32_t nid, const uint32_t* rk) {
    return philox_word_of(philox_block(h, nid >> 2, rk), nid);
}

// The compiled applicability mask without branches: the period's remainder
// is computed for every n (discarded below K), and the table of K + L
// four-bit masks is read as one 64-bit value.  tab as for compiled_mask_tab.
__device__ __forceinline__ uint32_t compiled_mask_flat(const uint4& rec, int32_t n, const uint2* __restrict__ tab) {
    const uint32_t K = (rec.y >> 24) & 15u, L = rec.y >> 28;
    const uint32_t x = (uint32_t)n - K;
    const uint2 mg = tab[L];
    const uint32_t r = x - (__umulhi(x, mg.x) >> mg.y) * L;  // x mod L when n >= K and L >= 2
    const uint32_t e = (uint32_t)n < K ? (uint32_t)n : K + (L > 1u ? r : 0u);
    const unsigned long long t64 = ((unsigned long long)rec.y << 32) | rec.x;
    return (uint32_t)(t64 >> (4u * e)) & 15u;
}

// pick[mask | idx << 4] = the position of the idx-th (0-based) set bit of a
// four-bit mask (0 where idx >= popc(mask)); threads 0..63 fill it.
__device__ __forceinline__ void fill_pick_table(uint8_t* pick) {
    const uint32_t i = threadIdx.x;
    if (i < 64u) {
        uint32_t m = i & 15u, idx = i >> 4, pos = 0u;
        for (uint32_t b = 0; b < 4u; ++b) {
            if (m & (1u << b)) {
                if (idx == 0u) {
                    pos = b;
                    break;
                }
                --idx;
            }
        }
        pick[i] = (uint8_t)pos;
    }
}

// The select of a slot from its compiled record (same result as
// select_compiled): every case computed without data-dependent branches
// except the Philox draw, which runs when any lane of the warp draws.
template <int SEL>
__device__ __forceinline__ SelOut select_rec_flat(const uint4 rec, int32_t n, uint32_t st, uint32_t nid,
                                                  const PhiloxHead& ph, const uint32_t* rk,
                                                  const uint2* __restrict__ tab, const uint8_t* __restrict__ pick) {
    const uint32_t pend = st >> kPendShift;
    const bool closed = pend != 0u;
    const bool completing = closed && (st & kDMask) == 0u;
    const uint32_t mask = closed ? 0u : compiled_mask_flat(rec, n, tab);
    uint32_t idx = 0u;
    if (SEL == SNP_SELECT_PHILOX) {
        const bool draw = (mask & (mask - 1u)) != 0u;
        if (__any_sync(__activemask(), draw)) {
            const uint32_t x0 = philox_word(ph, nid, rk);
            idx = draw ? (uint32_t)(((unsigned long long)x0 * (uint32_t)__popc(mask)) >> 32) : 0u;  // < popc <= 4
        }
    }
    const bool selected = mask != 0u;
    const uint32_t t = pick[mask | (idx << 4)];
    const uint32_t fi = completing ? pend - 1u : t;
    const uint32_t f = (uint32_t)((((unsigned long long)rec.w << 32) | rec.z) >> (16u * fi)) & 0xffffu;
    const int32_t c = (int32_t)(f & 63u), p = (int32_t)((f >> 6) & 31u), d = (int32_t)(f >> 11);
    SelOut o;
    o.active = closed || selected;
    o.s = selected ? (int32_t)t : -1;
    o.c_after = selected ? n - c : n;
    o.emit = (completing || (selected && d == 0)) ? p : 0;
    o.st = closed ? (completing ? 0u : st - 1u)
                  : ((selected && d > 0) ? ((t + 1u) << kPendShift) | (uint32_t)(d - 1) : 0u);
    return o;
}

// ---- forced choices (computation-tree exploration) ----------------------
// Applicable rules of an idle neuron with n spikes, in index order: bit t of
// the result (up to 32 rules) and the count.
template <bool COMPACT>
__device__ __forceinline__ int32_t count_applicable(const uint32_t* __restrict__ rules, int32_t r0, int32_t r1,
                                                    int32_t n) {
    int32_t cnt = 0;
    for (int32_t r = r0; r < r1; ++r) cnt += rule_applies_at<COMPACT>(rules, r, n) ? 1 : 0;
    return cnt;
}

// The same for neuron `slot`, through its compiled record when the system
// has one (always so for rules given as unions of terms).
template <bool COMPACT>
__device__ __forceinline__ int32_t count_applicable_slot(const DevSys& s, int32_t slot, int32_t n) {
    if (s.rec) return __popc(compiled_mask(__ldg(reinterpret_cast<const uint4*>(s.rec) + slot), n));
    return count_applicable<COMPACT>(s.rules, rule_lo(s, slot), rule_hi(s, slot), n);
}

// How many rules neuron `slot` may choose at the step about to run: the
// applicable rules of an idle neuron, 0 while a rule is pending.
template <bool COMPACT>
__device__ __forceinline__ int32_t choices_of(const DevSys& s, int32_t slot) {
    if ((s.st[slot] >> kPendShift) != 0u) return 0;
    return count_applicable_slot<COMPACT>(s, slot, s.C[slot]);
}

// The select phase with the choice given: an idle neuron with applicable
// rules takes the fidx-th of them (0-based, index order); an index outside
// 0 .. count-1 raises kFlagChoice and takes the first.  Pending neurons
// complete or count down as in select_neuron.
template <bool COMPACT>
__device__ SelOut select_forced_idx(const DevSys& s, int32_t slot, int32_t n, uint32_t st, int32_t fidx,
                                    bool& bad) {
    const int32_t r0 = rule_lo(s, slot), r1 = rule_hi(s, slot);
    SelOut o;
    o.c_after = n;
    o.emit = 0;
    o.s = -1;
    o.st = 0u;
    o.active = false;
    const uint32_t pend = st >> kPendShift;
    if (s.rec) {  // compiled record: mask of applicable rules, fields inline
        const uint4 rec = __ldg(reinterpret_cast<const uint4*>(s.rec) + slot);
        if (pend != 0u) {
            o.active = true;
            if ((st & kDMask) == 0u)
                o.emit = (int32_t)((compiled_field(rec, pend - 1u) >> 6) & 31u);
            else
                o.st = st - 1u;
            return o;
        }
        uint32_t mask = compiled_mask(rec, n);
        const int32_t cnt = __popc(mask);
        if (cnt == 0) return o;
        int32_t idx = fidx;
        if (idx < 0 || idx >= cnt) {
            bad = true;
            idx = 0;
        }
        for (; idx > 0; --idx) mask &= mask - 1u;  // drop the idx lowest applicable rules
        const uint32_t t = (uint32_t)(__ffs(mask) - 1);
        const uint32_t f = compiled_field(rec, t);
        const int32_t c = (int32_t)(f & 63u), p = (int32_t)((f >> 6) & 31u), d = (int32_t)(f >> 11);
        o.active = true;
        o.s = (int32_t)t;
        o.c_after = n - c;
        if (d == 0)
            o.emit = p;
        else
            o.st = ((t + 1u) << kPendShift) | (uint32_t)(d - 1);
        return o;
    }
    if (pend != 0u) {
        o.active = true;
        if ((st & kDMask) == 0u) {
            o.emit = load_rule<COMPACT>(s.rules, r0 + (int32_t)pend - 1).p;
        } else {
            o.st = st - 1u;
        }
        return o;
    }
    const int32_t cnt = count_applicable<COMPACT>(s.rules, r0, r1, n);
    if (cnt == 0) return o;
    int32_t idx = fidx;
    if (idx < 0 || idx >= cnt) {
        bad = true;
        idx = 0;
    }
    int32_t pick = -1;
    for (int32_t r = r0; r < r1 && pick < 0; ++r)
        if (rule_applies_at<COMPACT>(s.rules, r, n) && idx-- == 0) pick = r;
    const RuleF f = load_rule<COMPACT>(s.rules, pick);
    o.active = true;
    o.s = pick - r0;
    o.c_after = n - f.c;
    if (f.d == 0)
        o.emit = f.p;
    else
        o.st = ((uint32_t)(o.s + 1) << kPendShift) | (uint32_t)(f.d - 1);
    return o;
}

// The same with the index from the system's forced-choice array; an index
// out of range raises kFlagChoice.
template <bool COMPACT>
__device__ __forceinline__ SelOut select_forced(const DevSys& s, int32_t slot, int32_t n, uint32_t st) {
    bool bad = false;
    const SelOut o = select_forced_idx<COMPACT>(s, slot, n, st, s.forced[slot], bad);
    if (bad) atomicOr(s.flags + kFlagChoice, 1u);
    return o;
}

// The select phase of a slot through its compiled record when the system has
// one, else through its rule table; with forced choices set (only for the
// first step of a call, see snp_set_choices) through select_forced.
template <bool COMPACT, int SEL>
__device__ __forceinline__ SelOut select_slot(const DevSys& s, int32_t slot, int32_t n, uint32_t st,
                                              unsigned long long k) {
    if (s.forced) return select_forced<COMPACT>(s, slot, n, st);
    if (s.rec)
        return select_compiled<SEL>(__ldg(reinterpret_cast<const uint4*>(s.rec) + slot), n, st, k, neuron_id(s, slot),
                                    s.seed);
    return select_neuron<COMPACT, SEL>(s.rules, rule_lo(s, slot), rule_hi(s, slot), n, st, k, neuron_id(s, slot),
                                       s.seed);
}

// Programmatic dependent launch: wait until the grids this launch depends on
// have finished and their writes are visible; let the next launch on the
// stream start its own prologue.  Without the launch attribute both are
// no-ops.
__device__ __forceinline__ void grid_dependency_wait() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
}
__device__ __forceinline__ void allow_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) {
    return *reinterpret_cast<const volatile uint32_t*>(p);
}

// ---- fixed-point protocol of the per-step launches -----------------------
// Word kFlagAct0 + (k mod 3) is raised by the launch that selects step k when
// any neuron is pending or selected; the launch that finishes step k reads
// it, and if it is clear the system is at a fixed point: the step does not
// run and kFlagHalted stays set for the rest of the call.  The words are
// read once per CTA by thread 0 through the non-coherent cache and shared
// with the CTA: every warp reading them would queue tens of thousands of
// requests on one L2 line.  The activity word of step k is never written by
// the launch that reads it, and kFlagHalted is written in a launch only when
// that launch's activity word is clear, so a stale read cannot change what a
// CTA decides.  The reads go to L2 (ld.global.cg): launches may overlap the
// end of the launch before them, and L2 is where its writes are visible.

// Block-uniform: true if the launch finishing step kg must return at once.
__device__ __forceinline__ bool step_blocked(uint32_t* fl, unsigned long long* steps, unsigned long long kg) {
    __shared__ int s_blocked;
    if (threadIdx.x == 0) {
        int b = __ldcg(fl + kFlagHalted) != 0u;
        if (!b && __ldcg(fl + kFlagAct0 + (int)(kg % 3ull)) == 0u) {
            b = 1;
            if (blockIdx.x == 0 && blockIdx.y == 0) {
                steps[kStepHalt] = kg;
                __threadfence();
                atomicExch(fl + kFlagHalted, 1u);
            }
        }
        s_blocked = b;
    }
    __syncthreads();
    return s_blocked != 0;
}

// Block-uniform: true if an earlier launch of this call found a fixed point.
__device__ __forceinline__ bool call_halted(const uint32_t* fl) {
    __shared__ int s_halted;
    if (threadIdx.x == 0) s_halted = __ldcg(fl + kFlagHalted) != 0u;
    __syncthreads();
    return s_halted != 0;
}

// End of a select launch: raise step ks's activity word if this CTA saw a
// pending or selecting neuron (one store per CTA, skipped once raised).
__device__ __forceinline__ void raise_step_activity(uint32_t* fl, unsigned long long ks, bool active) {
    if (__syncthreads_or(active) && threadIdx.x == 0) {
        uint32_t* a = fl + kFlagAct0 + (int)(ks % 3ull);
        if (__ldcg(a) == 0u) *reinterpret_cast<volatile uint32_t*>(a) = 1u;
    }
}

}  // namespace snp
