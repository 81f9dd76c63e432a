// Host check of the tiled engine's packed layout (pack_tiled), no GPU needed.
//
// Builds a seeded random system, packs it for a device of 152 SMs with the
// cluster counts per wave that a GB300 reports at about 225 KB of shared
// memory per CTA, then decodes every CTA's entries back into (target,
// source) in-edges and checks:
//   * every in-edge of the system appears exactly once, in the CTA of its
//     target's range and its source's partition;
//   * (run-length layout) all in-edges of one target from one partition lie
//     in one thread's run, so that thread alone writes the accumulator;
//   * the entry buffer carries two rows of slack past the last CTA's block
//     (the gather loads two vectors ahead);
//   * the CTA's shared memory fits the budget.
// Prints one line "key=value ..." that the Python test parses.
//
// usage: tiled_layout_check q deg_lo deg_hi p_max zipf(0/1) seed
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <string>
#include <vector>

#include "snp_internal.h"

using namespace snp;

static uint64_t mix64(uint64_t x) {  // splitmix64 finaliser
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

int main(int argc, char** argv) {
    if (argc < 7) {
        std::fprintf(stderr, "usage: %s q deg_lo deg_hi p_max zipf seed\n", argv[0]);
        return 2;
    }
    const int32_t q = std::atoi(argv[1]);
    const int lo = std::atoi(argv[2]), hi = std::atoi(argv[3]), pmax = std::atoi(argv[4]);
    const bool zipf = std::atoi(argv[5]) != 0;
    uint64_t st = (uint64_t)std::atoll(argv[6]);
    auto rnd = [&]() { return mix64(st++); };

    // out-degree: uniform on [lo, hi], or Zipf(2.1) truncated to [1, 4096]
    std::vector<double> cdf;
    if (zipf) {
        double acc = 0;
        for (int x = 1; x <= 4096; ++x) cdf.push_back(acc += 1.0 / std::pow((double)x, 2.1));
        for (double& v : cdf) v /= acc;
    }
    std::vector<int64_t> so((size_t)q + 1, 0), ro((size_t)q + 1, 0);
    std::vector<int32_t> tg, C0((size_t)q, 1);
    for (int32_t i = 0; i < q; ++i) {
        int deg;
        if (zipf) {
            const double u = (double)(rnd() >> 11) / 9007199254740992.0;
            deg = 1 + (int)(std::lower_bound(cdf.begin(), cdf.end(), u) - cdf.begin());
            deg = std::min(deg, 4096);
        } else {
            deg = lo + (int)(rnd() % (uint64_t)(hi - lo + 1));
        }
        deg = std::min(deg, q - 1);
        std::vector<int32_t> t;
        while ((int)t.size() < deg) {
            const int32_t x = (int32_t)(rnd() % (uint64_t)q);
            if (x != i && std::find(t.begin(), t.end(), x) == t.end()) t.push_back(x);
        }
        tg.insert(tg.end(), t.begin(), t.end());
        so[(size_t)i + 1] = (int64_t)tg.size();
        ro[(size_t)i + 1] = ro[i] + 1;
    }
    // one firing rule a+/a -> a^p per neuron, p in 1..pmax
    std::vector<int32_t> rk((size_t)q, 1), rj((size_t)q, 1), rc((size_t)q, 1), rp((size_t)q), rd((size_t)q, 0);
    for (int32_t i = 0; i < q; ++i) rp[i] = 1 + (int32_t)(rnd() % (uint64_t)pmax);
    snp_desc d = {};
    d.q = q;
    d.init_spikes = C0.data();
    d.rule_offsets = ro.data();
    d.rule_k = rk.data();
    d.rule_j = rj.data();
    d.rule_c = rc.data();
    d.rule_p = rp.data();
    d.rule_d = rd.data();
    d.num_syn = (int64_t)tg.size();
    d.syn_offsets = so.data();
    d.syn_targets = tg.data();

    HostPack hp;
    if (pack_system(&d, false, false, 0, &hp)) return 3;
    TiledPack tp;
    const int cpw[kTiledMaxCluster + 1] = {0, 152, 76, 46, 36, 28, 23, 15, 15};
    const size_t budget = 227 * 1024 - 2048;
    if (pack_tiled(&d, hp, 152, budget, &tp, cpw)) return 4;

    const int T = kTiledThreads, eb = tp.e_bits, NR = tp.G / tp.P;
    // the in-lists the layout must hold: per target, its sources, sorted
    std::vector<std::vector<int32_t>> in((size_t)q);
    for (int32_t i = 0; i < q; ++i)
        for (int64_t e = so[i]; e < so[(size_t)i + 1]; ++e) in[(size_t)tg[(size_t)e]].push_back(i);
    long long mismatched = 0, edges = 0, split_targets = 0, positions = 0;
    int64_t last_end = 0;
    for (int g = 0; g < NR; ++g) {
        const int64_t s0 = (int64_t)tp.cta_lo[g] * kSlice;
        const int64_t s1 = std::min<int64_t>(q, (int64_t)tp.cta_lo[(size_t)g + 1] * kSlice);
        for (int h = 0; h < tp.P; ++h) {
            const int c = g * tp.P + h;
            const int32_t* sb = tp.sub.data() + (size_t)c * (kTiledMaxSub + 1);
            const int32_t src_lo = h * tp.part_size;
            std::map<int64_t, std::vector<int32_t>> got;  // target slot -> decoded sources
            std::map<int64_t, int> owner;
            if (tp.rle) {
                const int db = 24 - (tp.src_bits + __builtin_ctz((unsigned)eb));
                const int64_t base = sb[0] / 4, nvec = (sb[kTiledMaxSub] / 4 - base) / T;
                last_end = std::max<int64_t>(last_end, sb[kTiledMaxSub]);
                positions += nvec * T * 5;
                for (int t = 0; t < T; ++t) {
                    int64_t cur = tp.tstart[(size_t)c * T + t];
                    for (int64_t u = 0; u < nvec; ++u) {
                        const uint32_t* w = tp.ent.data() + (size_t)(base + u * T + t) * 4;
                        const uint32_t e5[5] = {w[0] & 0xFFFFFFu, ((w[0] >> 24) | (w[1] << 8)) & 0xFFFFFFu,
                                                ((w[1] >> 16) | (w[2] << 16)) & 0xFFFFFFu, w[2] >> 8,
                                                w[3] & 0xFFFFFFu};
                        for (uint32_t x : e5) {
                            cur += x & ((1u << db) - 1u);
                            const uint32_t src = (x >> db) / (uint32_t)eb;
                            if (src == (uint32_t)tp.part_size) continue;  // a pad entry
                            got[cur].push_back((int32_t)src + src_lo);
                            auto it = owner.find(cur);
                            if (it == owner.end())
                                owner[cur] = t;
                            else if (it->second != t)
                                ++split_targets;
                        }
                    }
                }
            } else {
                // target words, (target within its window << src_bits) |
                // source; window w holds the block's words sb[w] .. sb[w+1]
                // in target order, and the block's 16-byte vectors are stored
                // thread-contiguously: vector s0_t + u of thread t's run sits
                // at row u, column t
                const int wb = 32 - tp.src_bits;
                const int64_t base = sb[0] / 4, N = sb[kTiledMaxSub] / 4 - base;
                last_end = std::max<int64_t>(last_end, sb[kTiledMaxSub]);
                if (N > 0) {
                    const int64_t n = (N + T - 1) / T, r = N - (n - 1) * T;
                    for (int64_t t = 0; t < T; ++t) {
                        const int64_t v0 = t * n - std::max<int64_t>(0, t - r), nt = t < r ? n : n - 1;
                        for (int64_t u = 0; u < nt; ++u) {
                            const int64_t word0 = (base + v0 + u) * 4;  // position in target order
                            int win = 0;
                            while (win + 1 < kTiledMaxSub && sb[win + 1] <= word0) ++win;
                            for (int i = 0; i < 4; ++i) {
                                const uint32_t w = tp.ent[(size_t)((base + u * T + t) * 4 + i)];
                                const uint32_t src = w & ((1u << tp.src_bits) - 1u);
                                if (src == (uint32_t)tp.part_size) continue;  // padding
                                got[((int64_t)win << wb) + (w >> tp.src_bits)].push_back((int32_t)src + src_lo);
                            }
                        }
                    }
                }
            }
            const int32_t src_hi = (int32_t)std::min<int64_t>(q, (int64_t)(h + 1) * tp.part_size);
            long long decoded = 0;
            for (auto& kv : got) decoded += (long long)kv.second.size();
            long long wanted = 0;
            for (int64_t s = s0; s < s1; ++s) {
                std::vector<int32_t> want;
                for (int32_t x : in[(size_t)s])
                    if (x >= src_lo && x < src_hi) want.push_back(x);
                auto it = got.find(s - s0);
                std::vector<int32_t> have = it == got.end() ? std::vector<int32_t>() : it->second;
                std::sort(have.begin(), have.end());
                if (have != want) ++mismatched;
                wanted += (long long)want.size();
            }
            if (decoded != wanted) ++mismatched;  // edges decoded onto targets outside the range
            edges += wanted;
        }
    }
    const bool slack = !tp.rle || (int64_t)tp.ent.size() >= last_end + (int64_t)2 * T * 4;
    const bool smem_ok = tiled_smem_bytes(tp) <= budget;
    std::printf(
        "P=%d G=%d rle=%d pairs=%d acc8=%d rin_esm=%d e_bits=%d edges=%lld num_syn=%lld mismatched=%lld "
        "split_targets=%lld slack=%d smem_ok=%d positions=%lld\n",
        tp.P, tp.G, tp.rle, tp.pairs, tp.acc8, tp.rin_esm, tp.e_bits, edges, (long long)d.num_syn, mismatched,
        split_targets, slack ? 1 : 0, smem_ok ? 1 : 0, positions);
    return (mismatched || split_targets || !slack || !smem_ok || edges != d.num_syn) ? 1 : 0;
}
