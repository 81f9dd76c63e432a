// Validation of a system description and packing into the device layouts.
//
// The paper builds a dense transition matrix first and compresses it
// afterwards (Sec. 5, "Initialization"), which it names as the reason ELL
// could not reach the largest subset-sum instances (Sec. 6).  Here every
// layout is built straight from the edge list in O(|syn| + m) memory.
//
// Layouts (all in slot order, see below):
//  * rule table: N_Pi offsets (Sec. 2) and one compact word per rule when
//    every field fits (k, j, c < 256, p, d < 16), else four words per rule;
//  * in-lists (pull): sliced ELL.  Slots are grouped by 32 (one warp); a slice
//    stores its in-neighbour columns column-major, padded to the widest list
//    in the slice with the dummy slot q (whose emission is always 0).  This is
//    the transpose of the paper's synapse matrix Sy_Pi (Sec. 4) cut into
//    warp-sized slices;
//  * out-lists (push): the paper's Sy_Pi in the same sliced layout, padded
//    with -1 (the null entry that ends a column in Alg. 5).
//
// Slot order: inside windows of `window` neurons, neurons are stably sorted
// by decreasing in-degree so that the 32 lists of a slice have similar
// lengths and padding stays small.  The caller never sees slot numbers.
#include <algorithm>
#include <climits>
#include <cstring>
#include <numeric>

#include "snp_internal.h"

namespace snp {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }
int fail(int status, const std::string& msg) {
    g_err = msg;
    return status;
}
const char* last_error() { return g_err.c_str(); }

int validate_desc(const snp_desc* d) {
    if (!d) return fail(SNP_ERR_INVALID, "desc is NULL");
    if (d->q < 1) return fail(SNP_ERR_INVALID, "q must be >= 1");
    if (d->q > INT32_MAX - 64) return fail(SNP_ERR_INVALID, "q too large");
    if (!d->init_spikes || !d->rule_offsets || !d->syn_offsets)
        return fail(SNP_ERR_INVALID, "init_spikes, rule_offsets and syn_offsets are required");
    const int32_t q = d->q;
    if (d->rule_offsets[0] != 0) return fail(SNP_ERR_INVALID, "rule_offsets[0] != 0");
    for (int32_t i = 0; i < q; ++i) {
        int64_t a = d->rule_offsets[i], b = d->rule_offsets[i + 1];
        if (b < a) return fail(SNP_ERR_INVALID, "rule_offsets not monotone at neuron " + std::to_string(i));
        if (b - a > kMaxRulesPerNeuron)
            return fail(SNP_ERR_INVALID, "more than 32766 rules in neuron " + std::to_string(i));
        if (d->init_spikes[i] < 0) return fail(SNP_ERR_INVALID, "negative initial spikes at neuron " + std::to_string(i));
    }
    const int64_t m = d->rule_offsets[q];
    if (m > INT32_MAX - 1) return fail(SNP_ERR_INVALID, "too many rules");
    const bool unions = d->rule_term_offsets != nullptr;
    if (m > 0 && ((!unions && (!d->rule_k || !d->rule_j)) || !d->rule_c || !d->rule_p || !d->rule_d))
        return fail(SNP_ERR_INVALID, "rule arrays are required when m > 0");
    if (!unions && (d->term_k || d->term_j))
        return fail(SNP_ERR_INVALID, "term_k/term_j given without rule_term_offsets");
    if (unions) {
        if (d->rule_term_offsets[0] != 0) return fail(SNP_ERR_INVALID, "rule_term_offsets[0] != 0");
        for (int64_t r = 0; r < m; ++r)
            if (d->rule_term_offsets[r + 1] <= d->rule_term_offsets[r])
                return fail(SNP_ERR_INVALID, "rule " + std::to_string(r) + " has no term (rule_term_offsets must increase)");
        const int64_t T = d->rule_term_offsets[m];
        if (T > 0 && (!d->term_k || !d->term_j)) return fail(SNP_ERR_INVALID, "term_k and term_j are required");
        for (int64_t t = 0; t < T; ++t)
            if (d->term_k[t] < 0 || d->term_j[t] < 0)
                return fail(SNP_ERR_INVALID, "negative term_k or term_j in term " + std::to_string(t));
    }
    for (int64_t r = 0; r < m; ++r) {
        if ((!unions && (d->rule_k[r] < 0 || d->rule_j[r] < 0)) || d->rule_c[r] < 0)
            return fail(SNP_ERR_INVALID, "negative k, j or c in rule " + std::to_string(r));
        if (d->rule_p[r] < 0 || d->rule_p[r] > kMaxP)
            return fail(SNP_ERR_INVALID, "p out of [0, 65535] in rule " + std::to_string(r));
        if (d->rule_d[r] < 0 || d->rule_d[r] > kMaxDelay)
            return fail(SNP_ERR_INVALID, "d out of [0, 65535] in rule " + std::to_string(r));
        if (d->rule_p[r] == 0 && d->rule_d[r] != 0)
            return fail(SNP_ERR_INVALID, "forgetting rule with a delay: rule " + std::to_string(r));
    }
    if (d->syn_offsets[0] != 0) return fail(SNP_ERR_INVALID, "syn_offsets[0] != 0");
    if (d->syn_offsets[q] != d->num_syn) return fail(SNP_ERR_INVALID, "syn_offsets[q] != num_syn");
    if (d->num_syn > 0 && !d->syn_targets) return fail(SNP_ERR_INVALID, "syn_targets is NULL");
    std::vector<int32_t> row;
    for (int32_t i = 0; i < q; ++i) {
        int64_t a = d->syn_offsets[i], b = d->syn_offsets[i + 1];
        if (b < a) return fail(SNP_ERR_INVALID, "syn_offsets not monotone at neuron " + std::to_string(i));
        row.assign(d->syn_targets + a, d->syn_targets + b);
        for (int32_t t : row) {
            if (t < 0 || t >= q) return fail(SNP_ERR_INVALID, "synapse target out of range from neuron " + std::to_string(i));
            if (t == i) return fail(SNP_ERR_INVALID, "self-loop at neuron " + std::to_string(i));
        }
        std::sort(row.begin(), row.end());
        if (std::adjacent_find(row.begin(), row.end()) != row.end())
            return fail(SNP_ERR_INVALID, "duplicate synapse from neuron " + std::to_string(i));
    }
    if (d->out_neuron < -1 || d->out_neuron >= q) return fail(SNP_ERR_INVALID, "out_neuron out of range");
    return SNP_OK;
}

void pack_in_lists(const snp_desc* d, HostPack* hp) {
    const int32_t q = hp->q;
    const int32_t nslices = (q + kSlice - 1) / kSlice;
    hp->in_idx.assign((size_t)hp->slice_ptr[nslices] * kSlice, q);
    std::vector<int32_t> fill(q, 0);
    for (int32_t i = 0; i < q; ++i) {
        const int32_t si = hp->inv[i];
        for (int64_t e = d->syn_offsets[i]; e < d->syn_offsets[i + 1]; ++e) {
            const int32_t s = hp->inv[d->syn_targets[e]];
            const int32_t col = fill[s]++;
            const int64_t sl = s / kSlice, lane = s % kSlice;
            hp->in_idx[((int64_t)hp->slice_ptr[sl] + col) * kSlice + lane] = si;
        }
    }
}

// Rules given as unions that the compiled records cannot hold are stepped
// through the general (4-word) rule table.  A union rule's record keeps c
// and (p, d) in words 2 and 3 as any rule does; word 0 holds 0x80000000 |
// the index of its first term record and word 1 the number of terms.  The
// term records, two words (k, j) each, follow the 4m rule words in the same
// buffer, in slot order of their rules, so the index in word 0 counts
// 8-byte records from the start of the buffer (the first one is 2m).
static int pack_union_rules(const snp_desc* d, HostPack* hp) {
    const int32_t q = hp->q;
    const int64_t m = hp->m;
    const int64_t T = d->rule_term_offsets[m];
    if (2 * m + T >= ((int64_t)1 << 31))
        return fail(SNP_ERR_UNSUPPORTED, "too many rules and union terms for the rule table");
    hp->compact = false;
    hp->rules.assign((size_t)(4 * m + 2 * T), 0u);
    int64_t next = 2 * m;  // the next term record (8-byte units)
    for (int32_t s = 0; s < q; ++s) {
        const int32_t i = hp->perm[s];
        const int64_t r0 = d->rule_offsets[i];
        const int32_t R = hp->rule_off[s + 1] - hp->rule_off[s];
        for (int32_t t = 0; t < R; ++t) {
            const int64_t r = r0 + t, dst = hp->rule_off[s] + t;
            const int64_t u0 = d->rule_term_offsets[r], u1 = d->rule_term_offsets[r + 1];
            uint32_t* w = hp->rules.data() + dst * 4;
            w[0] = 0x80000000u | (uint32_t)next;
            w[1] = (uint32_t)(u1 - u0);
            w[2] = (uint32_t)d->rule_c[r];
            w[3] = (uint32_t)d->rule_p[r] | ((uint32_t)d->rule_d[r] << 16);
            for (int64_t u = u0; u < u1; ++u, ++next) {
                hp->rules[(size_t)next * 2] = (uint32_t)d->term_k[u];
                hp->rules[(size_t)next * 2 + 1] = (uint32_t)d->term_j[u];
            }
        }
    }
    return SNP_OK;
}

int pack_system(const snp_desc* d, bool want_out_lists, bool want_in_lists, int window, HostPack* hp) {
    const int32_t q = d->q;
    const int64_t m = d->rule_offsets[q];
    const int64_t nsyn = d->num_syn;
    hp->q = q;
    hp->m = m;
    hp->nsyn = nsyn;
    const bool sort_slots = window > 0;
    if (sort_slots && window < kSlice) window = kSlice;

    // in-degrees
    std::vector<int32_t> indeg(q, 0);
    for (int64_t e = 0; e < nsyn; ++e) indeg[d->syn_targets[e]]++;
    hp->max_in = q ? *std::max_element(indeg.begin(), indeg.end()) : 0;
    hp->max_out = 0;
    for (int32_t i = 0; i < q; ++i)
        hp->max_out = std::max<int32_t>(hp->max_out, (int32_t)(d->syn_offsets[i + 1] - d->syn_offsets[i]));

    // slot order: stable sort by decreasing in-degree inside windows
    hp->perm.resize(q);
    std::iota(hp->perm.begin(), hp->perm.end(), 0);
    for (int64_t w0 = 0; sort_slots && w0 < q; w0 += window) {
        int64_t w1 = std::min<int64_t>(q, w0 + window);
        std::stable_sort(hp->perm.begin() + w0, hp->perm.begin() + w1,
                         [&](int32_t a, int32_t b) { return indeg[a] > indeg[b]; });
    }
    hp->inv.assign(q, 0);
    for (int32_t s = 0; s < q; ++s) hp->inv[hp->perm[s]] = s;

    // rule table in slot order
    hp->rule_off.assign((size_t)q + 1, 0);
    hp->rule_base.assign(q, 0);
    int32_t max_rules = 0, max_p = 0, max_d = 0;
    bool compact = true;
    for (int32_t s = 0; s < q; ++s) {
        int32_t i = hp->perm[s];
        int32_t R = (int32_t)(d->rule_offsets[i + 1] - d->rule_offsets[i]);
        hp->rule_off[s + 1] = hp->rule_off[s] + R;
        hp->rule_base[s] = (int32_t)d->rule_offsets[i];
        max_rules = std::max(max_rules, R);
    }
    // with union expressions the rule table carries (k, j) = (0, 0): every
    // kernel then reads the compiled records (compile_rules) instead
    const bool unions = d->rule_term_offsets != nullptr;
    auto rk = [&](int64_t r) { return unions ? 0 : d->rule_k[r]; };
    auto rj = [&](int64_t r) { return unions ? 0 : d->rule_j[r]; };
    for (int64_t r = 0; r < m; ++r) {
        max_p = std::max(max_p, d->rule_p[r]);
        max_d = std::max(max_d, d->rule_d[r]);
        if (rk(r) > 255 || rj(r) > 255 || d->rule_c[r] > 255 || d->rule_p[r] > 15 || d->rule_d[r] > 15)
            compact = false;
    }
    hp->max_rules = max_rules;
    hp->uniform_rules = max_rules;
    for (int32_t i = 0; i < q; ++i)
        if (d->rule_offsets[i + 1] - d->rule_offsets[i] != max_rules) {
            hp->uniform_rules = 0;
            break;
        }
    hp->identity = !sort_slots;
    hp->max_p = max_p;
    hp->max_d = max_d;
    hp->compact = compact;
    hp->rules.assign(compact ? (size_t)m : (size_t)m * 4, 0);
    for (int32_t s = 0; s < q; ++s) {
        int32_t i = hp->perm[s];
        int64_t r0 = d->rule_offsets[i];
        int32_t R = hp->rule_off[s + 1] - hp->rule_off[s];
        for (int32_t t = 0; t < R; ++t) {
            int64_t r = r0 + t;
            int64_t dst = hp->rule_off[s] + t;
            if (compact) {
                hp->rules[dst] = pack_rule_compact(rk(r), rj(r), d->rule_c[r], d->rule_p[r], d->rule_d[r]);
            } else {
                hp->rules[dst * 4 + 0] = (uint32_t)rk(r);
                hp->rules[dst * 4 + 1] = (uint32_t)rj(r);
                hp->rules[dst * 4 + 2] = (uint32_t)d->rule_c[r];
                hp->rules[dst * 4 + 3] = (uint32_t)d->rule_p[r] | ((uint32_t)d->rule_d[r] << 16);
            }
        }
    }

    // in-lists: sliced ELL, pad = q
    const int32_t nslices = (q + kSlice - 1) / kSlice;
    hp->slice_ptr.assign((size_t)nslices + 1, 0);
    int64_t acc = 0;
    for (int32_t sl = 0; sl < nslices; ++sl) {
        int32_t w = 0;
        for (int32_t l = 0; l < kSlice; ++l) {
            int64_t s = (int64_t)sl * kSlice + l;
            if (s < q) w = std::max(w, indeg[hp->perm[s]]);
        }
        hp->slice_ptr[sl] = (int32_t)acc;
        acc += w;
        if (acc > INT32_MAX) return fail(SNP_ERR_INVALID, "in-lists too large for 32-bit slice offsets");
    }
    hp->slice_ptr[nslices] = (int32_t)acc;
    if (want_in_lists) pack_in_lists(d, hp);

    // out-lists (push): sliced ELL by source slot, pad = -1
    if (want_out_lists) {
        hp->out_ptr.assign((size_t)nslices + 1, 0);
        int64_t oacc = 0;
        for (int32_t sl = 0; sl < nslices; ++sl) {
            int32_t w = 0;
            for (int32_t l = 0; l < kSlice; ++l) {
                int64_t s = (int64_t)sl * kSlice + l;
                if (s < q) {
                    int32_t i = hp->perm[s];
                    w = std::max<int32_t>(w, (int32_t)(d->syn_offsets[i + 1] - d->syn_offsets[i]));
                }
            }
            hp->out_ptr[sl] = (int32_t)oacc;
            oacc += w;
            if (oacc > INT32_MAX) return fail(SNP_ERR_INVALID, "out-lists too large for 32-bit slice offsets");
        }
        hp->out_ptr[nslices] = (int32_t)oacc;
        hp->out_idx.assign((size_t)oacc * kSlice, -1);
        for (int32_t s = 0; s < q; ++s) {
            int32_t i = hp->perm[s];
            const int64_t sl = s / kSlice, lane = s % kSlice;
            int32_t col = 0;
            for (int64_t e = d->syn_offsets[i]; e < d->syn_offsets[i + 1]; ++e, ++col)
                hp->out_idx[((int64_t)hp->out_ptr[sl] + col) * kSlice + lane] = hp->inv[d->syn_targets[e]];
        }
    }

    if (!compile_rules(d, hp) && d->rule_term_offsets) {
        const int st = pack_union_rules(d, hp);
        if (st) return st;
    }

    hp->C0.resize(q);
    for (int32_t s = 0; s < q; ++s) hp->C0[s] = d->init_spikes[hp->perm[s]];
    return SNP_OK;
}

int pack_ell(const snp_desc* d, const HostPack& hp, bool want_pull, bool want_push, EllPack* ep) {
    const int32_t q = hp.q;
    const int64_t m = hp.m;
    const int32_t nslices = (q + kSlice - 1) / kSlice;
    // firing rules (p > 0) of every source slot, as (slot rule id, p)
    auto rule_id = [&](int32_t i, int64_t r) { return (int32_t)(hp.rule_off[hp.inv[i]] + (r - d->rule_offsets[i])); };
    std::vector<int32_t> nfire(q, 0);
    for (int32_t i = 0; i < q; ++i)
        for (int64_t r = d->rule_offsets[i]; r < d->rule_offsets[i + 1]; ++r) nfire[i] += d->rule_p[r] > 0;
    if (want_pull) {
        std::vector<int64_t> len(q, 0);  // pairs per target slot
        for (int32_t i = 0; i < q; ++i)
            for (int64_t e = d->syn_offsets[i]; e < d->syn_offsets[i + 1]; ++e) len[hp.inv[d->syn_targets[e]]] += nfire[i];
        ep->in_ptr.assign((size_t)nslices + 1, 0);
        int64_t acc = 0;
        for (int32_t sl = 0; sl < nslices; ++sl) {
            int64_t w = 0;
            for (int l = 0; l < kSlice; ++l) {
                const int64_t s = (int64_t)sl * kSlice + l;
                if (s < q) w = std::max(w, len[s]);
            }
            ep->in_ptr[sl] = (int32_t)acc;
            acc += w;
            if (acc * kSlice * 2 > INT32_MAX) return fail(SNP_ERR_UNSUPPORTED, "ELL in-lists too large");
        }
        ep->in_ptr[nslices] = (int32_t)acc;
        ep->in_ent.assign((size_t)acc * kSlice * 2, 0);
        for (int64_t x = 0; x < acc * kSlice; ++x) ep->in_ent[2 * x] = (int32_t)m;  // pad (m, 0)
        std::vector<int32_t> fill(q, 0);
        for (int32_t i = 0; i < q; ++i)
            for (int64_t e = d->syn_offsets[i]; e < d->syn_offsets[i + 1]; ++e) {
                const int32_t s = hp.inv[d->syn_targets[e]];
                const int64_t sl = s / kSlice, lane = s % kSlice;
                for (int64_t r = d->rule_offsets[i]; r < d->rule_offsets[i + 1]; ++r) {
                    if (d->rule_p[r] <= 0) continue;
                    const int64_t x = ((int64_t)ep->in_ptr[sl] + fill[s]++) * kSlice + lane;
                    ep->in_ent[2 * x] = rule_id(i, r);
                    ep->in_ent[2 * x + 1] = d->rule_p[r];
                }
            }
    }
    if (want_push) {
        const int64_t nrs = (m + kSlice - 1) / kSlice;
        // owner slot of every slot rule id
        std::vector<int32_t> owner((size_t)m);
        for (int32_t s = 0; s < q; ++s)
            for (int32_t r = hp.rule_off[s]; r < hp.rule_off[s + 1]; ++r) owner[r] = s;
        ep->out_ptr.assign((size_t)nrs + 1, 0);
        int64_t acc = 0;
        auto col_len = [&](int64_t r) -> int64_t {
            const int32_t i = hp.perm[owner[r]];
            const int64_t rr = d->rule_offsets[i] + (r - hp.rule_off[owner[r]]);
            return d->rule_p[rr] > 0 ? d->syn_offsets[i + 1] - d->syn_offsets[i] : 0;
        };
        for (int64_t rs = 0; rs < nrs; ++rs) {
            int64_t w = 0;
            for (int l = 0; l < kSlice; ++l) {
                const int64_t r = rs * kSlice + l;
                if (r < m) w = std::max(w, col_len(r));
            }
            ep->out_ptr[rs] = (int32_t)acc;
            acc += w;
            if (acc * kSlice * 2 > INT32_MAX) return fail(SNP_ERR_UNSUPPORTED, "ELL out-lists too large");
        }
        ep->out_ptr[nrs] = (int32_t)acc;
        ep->out_ent.assign((size_t)acc * kSlice * 2, 0);
        for (int64_t x = 0; x < acc * kSlice; ++x) ep->out_ent[2 * x] = -1;  // pad (-1, 0)
        for (int64_t r = 0; r < m; ++r) {
            const int32_t i = hp.perm[owner[r]];
            const int64_t rr = d->rule_offsets[i] + (r - hp.rule_off[owner[r]]);
            if (d->rule_p[rr] <= 0) continue;
            const int64_t rs = r / kSlice, lane = r % kSlice;
            int64_t row = 0;
            for (int64_t e = d->syn_offsets[i]; e < d->syn_offsets[i + 1]; ++e, ++row) {
                const int64_t x = ((int64_t)ep->out_ptr[rs] + row) * kSlice + lane;
                ep->out_ent[2 * x] = hp.inv[d->syn_targets[e]];
                ep->out_ent[2 * x + 1] = d->rule_p[rr];
            }
        }
    }
    return SNP_OK;
}

int pack_dense(const snp_desc* d, const HostPack& hp, std::vector<int32_t>* M) {
    const int64_t q = hp.q, m = hp.m;
    if (m * q > ((int64_t)1 << 31)) return fail(SNP_ERR_UNSUPPORTED, "dense matrix too large (m q > 2^31)");
    M->assign((size_t)(m * q), 0);
    for (int32_t i = 0; i < hp.q; ++i)
        for (int64_t r = d->rule_offsets[i]; r < d->rule_offsets[i + 1]; ++r) {
            const int64_t row = hp.rule_off[hp.inv[i]] + (r - d->rule_offsets[i]);
            for (int64_t e = d->syn_offsets[i]; e < d->syn_offsets[i + 1]; ++e)
                (*M)[(size_t)(row * q + hp.inv[d->syn_targets[e]])] = d->rule_p[r];
        }
    return SNP_OK;
}

static int64_t gcd64(int64_t a, int64_t b) {
    while (b) {
        const int64_t t = a % b;
        a = b;
        b = t;
    }
    return a;
}

bool compile_rules(const snp_desc* d, HostPack* hp) {
    const int32_t q = hp->q;
    hp->rec.clear();
    if (hp->max_rules > 4) return false;
    // the terms of rule r: its own (k, j), or its union's terms
    const bool unions = d->rule_term_offsets != nullptr;
    auto t_lo = [&](int64_t r) { return unions ? d->rule_term_offsets[r] : r; };
    auto t_hi = [&](int64_t r) { return unions ? d->rule_term_offsets[r + 1] : r + 1; };
    auto t_k = [&](int64_t u) { return unions ? d->term_k[u] : d->rule_k[u]; };
    auto t_j = [&](int64_t u) { return unions ? d->term_j[u] : d->rule_j[u]; };
    std::vector<uint32_t> rec((size_t)q * 4, 0u);
    for (int32_t s = 0; s < q; ++s) {
        const int32_t i = hp->perm[s];
        const int64_t r0 = d->rule_offsets[i], R = d->rule_offsets[i + 1] - r0;
        int64_t K = 1, L = 1;
        for (int64_t t = 0; t < R; ++t) {
            const int64_t r = r0 + t;
            if (d->rule_c[r] >= 64 || d->rule_p[r] >= 32 || d->rule_d[r] >= 32) return false;
            K = std::max<int64_t>(K, 1 + (int64_t)d->rule_c[r]);
            for (int64_t u = t_lo(r); u < t_hi(r); ++u) {
                if (t_k(u) >= 14) return false;
                K = std::max<int64_t>(K, 1 + (int64_t)t_k(u));
                if (t_j(u) > 0) {
                    if (t_j(u) > 14) return false;
                    L = L / gcd64(L, t_j(u)) * t_j(u);
                    if (L > 14) return false;
                }
            }
        }
        if (K + L > 14) return false;
        uint64_t table = 0;
        for (int64_t e = 0; e < K + L; ++e) {
            const int64_t n = e;  // entries K.. stand for n = K + (n - K) mod L; n = e is such an n
            uint32_t mask = 0;
            for (int64_t t = 0; t < R; ++t) {
                const int64_t r = r0 + t, c = d->rule_c[r];
                bool ok = false;
                for (int64_t u = t_lo(r); u < t_hi(r) && !ok; ++u) {
                    const int64_t k = t_k(u), j = t_j(u);
                    ok = n >= k && (j == 0 ? n == k : (n - k) % j == 0);
                }
                if (ok && n >= c) mask |= 1u << t;
            }
            table |= (uint64_t)mask << (4 * e);
        }
        uint32_t* w = rec.data() + (size_t)s * 4;
        w[0] = (uint32_t)table;
        w[1] = (uint32_t)((table >> 32) & 0xffffffu) | ((uint32_t)K << 24) | ((uint32_t)L << 28);
        for (int64_t t = 0; t < R; ++t) {
            const int64_t r = r0 + t;
            const uint32_t f = (uint32_t)d->rule_c[r] | ((uint32_t)d->rule_p[r] << 6) | ((uint32_t)d->rule_d[r] << 11);
            w[2 + t / 2] |= f << (16 * (t % 2));
        }
    }
    hp->rec.swap(rec);
    return true;
}

int tiled_e_bits(int max_p) {
    if (max_p <= 3) return 2;
    if (max_p <= 15) return 4;
    if (max_p <= 255) return 8;
    return 16;
}

size_t tiled_smem_bytes(const TiledPack& tp) {
    return (size_t)tp.part_words * 4 + 16 + (size_t)tp.acc_words * 4 + (tp.rin_esm ? 0 : (size_t)tp.rin_words * 4);
}

static int bits_for(int64_t n) {  // bits to hold 0..n
    int b = 0;
    while (((int64_t)1 << b) <= n) ++b;
    return b;
}

int pack_tiled(const snp_desc* d, const HostPack& hp, int G, size_t smem_budget, TiledPack* tp,
               const int* cpw) {
    const int32_t q = hp.q;
    const int32_t nslices = (q + kSlice - 1) / kSlice;
    const int eb = tiled_e_bits(hp.max_p);
    if (G < 1) G = 1;
    if (G > nslices) G = nslices;

    // in-neighbour lists by target slot, sources as slots, sorted
    std::vector<int64_t> ioff((size_t)q + 1, 0);
    for (int64_t e = 0; e < hp.nsyn; ++e) ioff[(size_t)hp.inv[d->syn_targets[e]] + 1]++;
    for (int32_t s = 0; s < q; ++s) ioff[s + 1] += ioff[s];
    std::vector<int32_t> isrc((size_t)hp.nsyn);
    {
        std::vector<int64_t> fill(ioff.begin(), ioff.end() - 1);
        for (int32_t i = 0; i < q; ++i) {
            const int32_t si = hp.inv[i];
            for (int64_t e = d->syn_offsets[i]; e < d->syn_offsets[i + 1]; ++e)
                isrc[(size_t)fill[hp.inv[d->syn_targets[e]]]++] = si;
        }
        for (int32_t s = 0; s < q; ++s) std::sort(isrc.begin() + ioff[s], isrc.begin() + ioff[s + 1]);
    }

    // Slice ranges balanced by entries plus a per-slice cost.  The launch has
    // one CTA per (range, partition), so a CTA loads one partition's
    // emissions once; with P partitions there are G / P ranges.
    std::vector<int64_t> cost((size_t)nslices + 1, 0);
    for (int32_t sl = 0; sl < nslices; ++sl) {
        const int64_t a = ioff[std::min<int64_t>(q, (int64_t)sl * kSlice)];
        const int64_t b = ioff[std::min<int64_t>(q, (int64_t)(sl + 1) * kSlice)];
        cost[sl + 1] = cost[sl] + (b - a) + 64;
    }
    auto split = [&](int nr, std::vector<int32_t>& lo) {
        lo.assign((size_t)nr + 1, nslices);
        int32_t sl = 0;
        for (int g = 0; g < nr; ++g) {
            lo[g] = sl;
            const int64_t target = cost[nslices] * (g + 1) / nr;
            while (sl < nslices && cost[sl + 1] <= target) ++sl;
        }
        lo[nr] = nslices;
    };
    std::vector<int32_t> cta_lo;
    int P = 0, NR = 0, part_size = 0, part_words = 0, src_bits = 0, acc_words = 0, max_slices = 0;
    int64_t max_slots = 0;
    bool acc8 = false, rin_esm = false;
    int rin_words = 0;
    // Byte accumulators when every target's in-flow from one partition fits
    // a byte (in-degree x largest p <= 255): a range then holds four times the
    // targets of 32-bit accumulators, and the partitions of a range exchange
    // their in-flows through per-sender byte buffers (rin); they need the
    // run-length entries (a bit index of at most 21 bits) and one cluster per
    // range.  Otherwise 32-bit accumulators.  Either way: one CTA per SM
    // first, more CTAs (several waves) when the accumulators of fewer, larger
    // ranges would not fit next to a partition's emissions.
    const bool acc8_ok = (int64_t)hp.max_in * (int64_t)std::max(1, hp.max_p) <= 255;
    // One configuration: p partitions, gm waves.  Returns the CTAs of one
    // wave it would use (0: it does not fit); with commit, takes it.
    auto try_cfg = [&](int p, int gm, bool a8, bool commit) -> int {
        // ranges of one wave: the clusters of p CTAs the device holds at once
        const int per_wave = (cpw && p <= kTiledMaxCluster && cpw[p] > 0) ? std::min(cpw[p], G / p) : G / p;
        const int nr = std::max(1, std::min(nslices, std::max(1, per_wave) * gm));
        std::vector<int32_t> lo;
        split(nr, lo);
        int32_t ms = 0;
        for (int g = 0; g < nr; ++g) ms = std::max(ms, lo[g + 1] - lo[g]);
        const int64_t slots = (int64_t)ms * kSlice;  // local slot `slots` is the dummy
        const int aw = a8 ? (int)(((slots + 1 + 3) / 4 + 3) / 4 * 4) : (int)((slots + 1 + 3) / 4 * 4);
        int64_t ps = ((int64_t)q + p - 1) / p;
        ps = (ps + 511) / 512 * 512;
        const int64_t words = ps * eb / 32;
        const int sb = bits_for(ps);  // sources 0..part_size; part_size reads a zero word
        // the partner buffers: (P - 1) senders x the largest share
        const int64_t share_slots = (int64_t)((ms + p - 1) / p) * kSlice;
        const int64_t rw = a8 ? (p > 1 ? (int64_t)(p - 1) * share_slots / 4 : 0) : (p == 2 ? share_slots : 0);
        const size_t need = (size_t)words * 4 + 16 + (size_t)aw * 4;
        bool ok, in_esm = false;
        if (a8) {
            // the partner buffer beside the rest, or else in the emissions'
            // region (free once the cluster's gathers are done)
            in_esm = need + (size_t)rw * 4 > smem_budget && rw <= words + 4;
            ok = (need + (size_t)(in_esm ? 0 : rw) * 4 <= smem_budget) && p <= kTiledMaxCluster &&
                 sb + __builtin_ctz((unsigned)eb) <= 21;
        } else {
            const int db = 32 - sb;
            const int64_t nsub = (slots + ((int64_t)1 << db) - 1) >> db;
            ok = need <= smem_budget && db >= 5 && nsub <= kTiledMaxSub;
        }
        if (!ok) return 0;
        if (commit) {
            P = p;
            G = G * gm;
            NR = nr;
            cta_lo = lo;
            part_size = (int)ps;
            part_words = (int)words;
            src_bits = sb;
            acc_words = aw;
            max_slices = ms;
            max_slots = slots;
            acc8 = a8;
            // 32-bit accumulators: the partner buffer only where it fits
            rin_words = (a8 || need + (size_t)rw * 4 <= smem_budget) ? (int)rw : 0;
            rin_esm = in_esm;
        }
        return std::min(nr, std::max(1, per_wave)) * p;
    };
    if (acc8_ok) {
        // one wave if any cluster size allows it: the one using the most SMs
        int best = 0, best_ctas = 0;
        for (int p = 1; p <= kTiledMaxCluster; ++p) {
            const int c = try_cfg(p, 1, true, false);
            if (c > best_ctas) {
                best_ctas = c;
                best = p;
            }
        }
        if (best) try_cfg(best, 1, true, true);
    }
    for (int pass = acc8_ok ? 0 : 1; pass < 2 && P == 0; ++pass)
        for (int p = 1, gm = 1; gm <= 8 && P == 0; p = (p == 64 ? (++gm, 1) : p + 1))
            try_cfg(p, gm, pass == 0, true);
    if (P == 0) return fail(SNP_ERR_UNSUPPORTED, "no source partitioning fits shared memory and 32-bit entries");
    G = NR * P;  // CTAs of the launch

    tp->e_bits = eb;
    tp->P = P;
    tp->part_size = part_size;
    tp->part_words = part_words;
    tp->G = G;
    tp->max_slices = max_slices;
    tp->acc_words = acc_words;
    tp->src_bits = src_bits;
    tp->acc8 = acc8 ? 1 : 0;
    // The partitions' in-flows of a CTA's share arrive in a buffer of its
    // own (the fused step then needs no barrier after its select phase):
    // with byte accumulators always, (P - 1) byte segments, one per sender;
    // with 32-bit accumulators for two partitions when it fits.
    tp->rin_words = rin_words;
    tp->rin_esm = rin_esm ? 1 : 0;
    tp->cta_lo = cta_lo;
    const int db = 32 - src_bits;
    // run-length layout when a source's bit index in the packed emissions
    // (source x e_bits) fits 21 bits, leaving at least 3 bits for the target
    // advance; otherwise the paired layout unless too many (target,
    // partition) groups have an odd number of words
    const int rle_bits = src_bits + __builtin_ctz((unsigned)eb);  // bits of a bit index 0 .. part_size * eb
    tp->rle = rle_bits <= 21 ? 1 : 0;  // always so with byte accumulators
    int64_t odd = 0;
    {
        for (int32_t s = 0; s < q; ++s) {
            auto b = isrc.begin() + ioff[s], e = isrc.begin() + ioff[s + 1];
            for (int h = 0; h < P && b != e; ++h) {
                auto m = std::lower_bound(b, e, (int32_t)std::min<int64_t>(q, (int64_t)(h + 1) * part_size));
                odd += (m - b) & 1;
                b = m;
            }
        }
        tp->pairs = (double)odd <= kTiledPairSlack * (double)std::max<int64_t>(1, hp.nsyn) ? 1 : 0;
    }
    tp->sub.assign((size_t)G * (kTiledMaxSub + 1), 0);
    tp->ent.clear();
    tp->ent.reserve((size_t)hp.nsyn + (size_t)q + (size_t)G * kTiledMaxSub * 4);
    const uint32_t pad = (uint32_t)part_size;  // target 0 of the window, source = the zero word
    const int rle_db = 24 - rle_bits;          // run-length entries: bit index << rle_db | advance
    std::vector<int64_t> cur(kSlice), end(kSlice);
    // the words of the other layouts, for the run-length layout to beat
    const double other_words = (double)hp.nsyn + (tp->pairs ? (double)odd : 0.0) + 12.0 * G * kTiledMaxSub;
    if (tp->rle) {
        tp->tstart.assign((size_t)G * kTiledThreads, 0);
        const int64_t T = kTiledThreads;
        const uint32_t max_delta = (1u << rle_db) - 1u;
        const uint32_t rle_pad = (pad * (uint32_t)eb) << rle_db;  // the zero word, no advance
        std::vector<std::pair<uint32_t, uint32_t>> seq;  // (target local to the range, source local to the partition)
        std::vector<int64_t> bnd;                          // run t = seq[bnd[t] .. bnd[t+1])
        std::vector<int64_t> gstart;                       // first entry of each target group
        std::vector<std::vector<std::pair<uint32_t, int64_t>>> tmpl(T);  // per run: (advance, seq index or -1)
        const uint32_t dummy = (uint32_t)max_slots;       // the accumulator no slot reads
        for (int g = 0; g < NR; ++g) {
            for (int h = 0; h < P; ++h) {
                const int c = g * P + h;
                int32_t* sb = tp->sub.data() + (size_t)c * (kTiledMaxSub + 1);
                const int32_t lo_src = h * part_size;
                const int32_t hi_src = (int32_t)std::min<int64_t>(q, (int64_t)(h + 1) * part_size);
                seq.clear();
                for (int64_t s = (int64_t)cta_lo[g] * kSlice; s < std::min<int64_t>(q, (int64_t)cta_lo[g + 1] * kSlice); ++s) {
                    auto b = isrc.begin() + ioff[s], e = isrc.begin() + ioff[s + 1];
                    const int64_t x0 = std::lower_bound(b, e, lo_src) - isrc.begin();
                    const int64_t x1 = std::lower_bound(b, e, hi_src) - isrc.begin();
                    const uint32_t local = (uint32_t)(s - (int64_t)cta_lo[g] * kSlice);
                    for (int64_t x = x0; x < x1; ++x) seq.push_back({local, (uint32_t)(isrc[(size_t)x] - lo_src)});
                }
                // Cut into T runs of nearly equal length at target boundaries:
                // all in-edges of a target from this partition fall in one
                // run, so the thread of that run owns the target's
                // accumulator and writes it with a plain store.
                const int64_t n_e = (int64_t)seq.size();
                // target groups and what each costs in a run after another
                // group (its entries plus the pad entries of a long gap)
                gstart.clear();
                for (int64_t x = 0; x < n_e; ++x)
                    if (x == 0 || seq[x].first != seq[x - 1].first) gstart.push_back(x);
                gstart.push_back(n_e);
                const int64_t ng = (int64_t)gstart.size() - 1;
                auto cost = [&](int64_t k, bool first) {
                    const int64_t sz = gstart[k + 1] - gstart[k];
                    if (first || k == 0) return sz;
                    const int64_t d = (int64_t)seq[gstart[k]].first - (int64_t)seq[gstart[k - 1]].first;
                    return sz + (d + max_delta - 1) / max_delta - 1;
                };
                // the smallest longest run: whole groups, at most T runs
                auto fits = [&](int64_t cap, bool cut) {
                    int64_t t = 0, len = 0;
                    if (cut) bnd[0] = 0;
                    for (int64_t k = 0; k < ng; ++k) {
                        int64_t c_ = cost(k, len == 0);
                        if (len > 0 && len + c_ > cap) {
                            if (++t >= T) return false;
                            if (cut) bnd[t] = gstart[k];
                            len = 0;
                            c_ = cost(k, true);
                        }
                        len += c_;
                    }
                    if (cut)
                        for (int64_t r = t + 1; r <= T; ++r) bnd[r] = n_e;
                    return true;
                };
                bnd.assign((size_t)T + 1, n_e);
                int64_t lo_c = 1, hi_c = 1;
                for (int64_t k = 0; k < ng; ++k) {
                    lo_c = std::max(lo_c, cost(k, true));
                    hi_c += cost(k, false);
                }
                lo_c = std::max(lo_c, (n_e + T - 1) / T);
                while (lo_c < hi_c) {
                    const int64_t mid = (lo_c + hi_c) / 2;
                    if (fits(mid, false))
                        hi_c = mid;
                    else
                        lo_c = mid + 1;
                }
                fits(lo_c, true);
                // the positions of every run: the advance of each entry and the
                // target group whose source goes there (-1: a pad entry)
                size_t nvec = 0;
                for (int64_t t = 0; t < T; ++t) {
                    std::vector<std::pair<uint32_t, int64_t>>& pos = tmpl[t];
                    pos.clear();
                    const int64_t a0 = bnd[t], a1 = bnd[t + 1];
                    uint32_t cur = a0 < a1 ? seq[a0].first : dummy;
                    tp->tstart[(size_t)c * T + t] = (int32_t)cur;
                    for (int64_t x = a0; x < a1; ++x) {
                        uint32_t d = seq[x].first - cur;
                        while (d > max_delta) {  // a long gap: advance with pad entries
                            pos.push_back({max_delta, -1});
                            d -= max_delta;
                        }
                        pos.push_back({d, x});
                        cur = seq[x].first;
                    }
                    while (pos.size() % 5) pos.push_back({0u, -1});  // zero delta, zero emission
                    nvec = std::max(nvec, pos.size() / 5);
                }
                // Sources within a target's group may go in any order (the sum
                // does not depend on it).  The lanes of a warp read position u
                // of their runs in the same shared-memory load, so each
                // position takes, lane by lane, the group's remaining source
                // whose bank the warp's other lanes use least there (a word
                // already read at that position costs nothing: broadcast).
                std::vector<int32_t> srcs(seq.size());
                for (size_t x = 0; x < seq.size(); ++x) srcs[x] = (int32_t)seq[x].second;
                const size_t npos = nvec * 5;
                for (int64_t t = 0; t < T; ++t) tmpl[t].resize(npos, {0u, -1});
                const uint32_t pad_word = (pad * (uint32_t)eb) >> 5;
                for (int64_t w0 = 0; w0 < T; w0 += 32) {
                    for (size_t p = 0; p < npos; ++p) {
                        int bank_n[32] = {0};
                        uint32_t words[32];
                        int nwords = 0;
                        auto take = [&](uint32_t word) {
                            for (int i = 0; i < nwords; ++i)
                                if (words[i] == word) return;
                            words[nwords++] = word;
                            ++bank_n[word & 31u];
                        };
                        // forced lanes first (a pad, or one source left in the group)
                        for (int pass = 0; pass < 2; ++pass) {
                            for (int64_t t = w0; t < std::min<int64_t>(T, w0 + 32); ++t) {
                                const int64_t x = tmpl[t][p].second;
                                if (x < 0) {
                                    if (pass == 0) take(pad_word);
                                    continue;
                                }
                                // remaining sources of this group: srcs[x .. group end)
                                int64_t e = x + 1;
                                while (e < bnd[t + 1] && seq[e].first == seq[x].first) ++e;
                                if ((pass == 0) != (e - x == 1)) continue;
                                int64_t best = x;
                                int best_cost = 1 << 30;
                                for (int64_t y = x; y < e; ++y) {
                                    const uint32_t word = ((uint32_t)srcs[y] * (uint32_t)eb) >> 5;
                                    int cost = bank_n[word & 31u];
                                    for (int i = 0; i < nwords; ++i)
                                        if (words[i] == word) cost = 0;
                                    if (cost < best_cost) {
                                        best_cost = cost;
                                        best = y;
                                    }
                                }
                                std::swap(srcs[x], srcs[best]);
                                take(((uint32_t)srcs[x] * (uint32_t)eb) >> 5);
                            }
                        }
                    }
                }
                const size_t base = tp->ent.size() / 4;
                sb[0] = (int32_t)(base * 4);
                tp->ent.resize((base + nvec * T) * 4, 0u);
                for (int64_t t = 0; t < T; ++t) {
                    const std::vector<std::pair<uint32_t, int64_t>>& pos = tmpl[t];
                    for (size_t u = 0; u < nvec; ++u) {
                        uint32_t e[5];
                        for (int i = 0; i < 5; ++i) {
                            const auto& ps = pos[u * 5 + (size_t)i];
                            e[i] = (ps.second < 0 ? rle_pad : (((uint32_t)srcs[ps.second] * (uint32_t)eb) << rle_db)) |
                                   ps.first;
                        }
                        uint32_t* w = tp->ent.data() + (base + u * T + (size_t)t) * 4;
                        w[0] = e[0] | (e[1] << 24);
                        w[1] = (e[1] >> 8) | (e[2] << 16);
                        w[2] = (e[2] >> 16) | (e[3] << 8);
                        w[3] = e[4];
                    }
                }
                for (int k = 1; k <= kTiledMaxSub; ++k) sb[k] = (int32_t)tp->ent.size();
                if (tp->ent.size() > (size_t)INT32_MAX) return fail(SNP_ERR_UNSUPPORTED, "too many entries");
            }
        }
        // short runs spend most of their words on padding: keep the run-length
        // layout only when it is clearly smaller
        if (tp->acc8 || (double)tp->ent.size() <= 0.9 * other_words) {
            tp->pairs = 0;
            // slack: the gather loads two vectors ahead of the one it adds,
            // so the last CTA's threads read up to two rows past its block
            tp->ent.resize(tp->ent.size() + (size_t)2 * T * 4, rle_pad);
            return SNP_OK;
        }
        tp->rle = 0;
        tp->tstart.clear();
        tp->ent.clear();
        std::fill(tp->sub.begin(), tp->sub.end(), 0);
    }
    for (int g = 0; g < NR; ++g) {
        for (int h = 0; h < P; ++h) {
            int32_t* sb = tp->sub.data() + (size_t)(g * P + h) * (kTiledMaxSub + 1);
            int win = 0;  // current target window
            sb[0] = (int32_t)tp->ent.size();
            const int32_t lo_src = h * part_size;
            const int32_t hi_src = (int32_t)std::min<int64_t>(q, (int64_t)(h + 1) * part_size);
            for (int32_t sl = cta_lo[g]; sl < cta_lo[g + 1]; ++sl) {
                int64_t maxn = 0;
                for (int l = 0; l < kSlice; ++l) {
                    const int64_t s = (int64_t)sl * kSlice + l;
                    if (s >= q) {
                        cur[l] = end[l] = 0;
                        continue;
                    }
                    auto b = isrc.begin() + ioff[s], e = isrc.begin() + ioff[s + 1];
                    cur[l] = std::lower_bound(b, e, lo_src) - isrc.begin();
                    end[l] = std::lower_bound(b, e, hi_src) - isrc.begin();
                    maxn = std::max(maxn, end[l] - cur[l]);
                }
                // target-major; in the paired layout each target's words are
                // padded to an even count, so a 16-byte load holds two
                // (target, two sources) pairs
                (void)maxn;
                const uint32_t local0 = (uint32_t)(sl - cta_lo[g]) * kSlice;
                for (int l = 0; l < kSlice; ++l) {
                    const uint32_t local = local0 + (uint32_t)l;
                    while ((int)(local >> db) > win) {  // close the window: pad to 16 bytes
                        while (tp->ent.size() % 4) tp->ent.push_back(pad);
                        sb[++win] = (int32_t)tp->ent.size();
                    }
                    const uint32_t dst = local & (((uint32_t)1 << db) - 1u);
                    for (int64_t x = cur[l]; x < end[l]; ++x)
                        tp->ent.push_back((dst << src_bits) | (uint32_t)(isrc[(size_t)x] - lo_src));
                    if (tp->pairs && ((end[l] - cur[l]) & 1)) tp->ent.push_back((dst << src_bits) | pad);  // complete the pair
                }
            }
            while (tp->ent.size() % 4) tp->ent.push_back(pad);
            while (win < kTiledMaxSub) sb[++win] = (int32_t)tp->ent.size();
            if (tp->ent.size() > (size_t)INT32_MAX) return fail(SNP_ERR_UNSUPPORTED, "too many entries");
            // thread-contiguous storage order of the group's vectors
            const int64_t base = sb[0] / 4, N = (int64_t)tp->ent.size() / 4 - base;
            if (N > 0) {
                const int64_t T = kTiledThreads, n = (N + T - 1) / T, r = N - (n - 1) * T;
                std::vector<uint32_t> srt(tp->ent.begin() + base * 4, tp->ent.end());
                for (int64_t t = 0; t < T; ++t) {
                    const int64_t s0 = t * n - std::max<int64_t>(0, t - r), nt = t < r ? n : n - 1;
                    for (int64_t u = 0; u < nt; ++u)
                        std::copy_n(srt.begin() + (s0 + u) * 4, 4, tp->ent.begin() + (base + u * T + t) * 4);
                }
            }
        }
    }
    return SNP_OK;
}

}  // namespace snp

// ---- paper formats on the host (inspection / memory accounting) ---------

extern "C" int snp_export_dense(const snp_desc* d, int32_t* M, int64_t capacity) {
    int st = snp::validate_desc(d);
    if (st) return st;
    const int64_t q = d->q, m = d->rule_offsets[q];
    if (!M || capacity < m * q) return snp::fail(SNP_ERR_INVALID, "dense output too small");
    std::memset(M, 0, sizeof(int32_t) * (size_t)(m * q));
    for (int64_t i = 0; i < q; ++i)
        for (int64_t r = d->rule_offsets[i]; r < d->rule_offsets[i + 1]; ++r) {
            M[r * q + i] -= d->rule_c[r];
            for (int64_t e = d->syn_offsets[i]; e < d->syn_offsets[i + 1]; ++e)
                M[r * q + d->syn_targets[e]] += d->rule_p[r];
        }
    return SNP_OK;
}

extern "C" int snp_export_ell(const snp_desc* d, int32_t* values, int32_t* neurons, int64_t capacity,
                              int64_t* rows_out) {
    int st = snp::validate_desc(d);
    if (st) return st;
    const int64_t q = d->q, m = d->rule_offsets[q];
    int64_t z = 0;
    for (int64_t i = 0; i < q; ++i) z = std::max<int64_t>(z, d->syn_offsets[i + 1] - d->syn_offsets[i]);
    const int64_t rows = z + 1;
    if (rows_out) *rows_out = rows;
    if (!values && !neurons) return SNP_OK;
    if (!values || !neurons || capacity < rows * m) return snp::fail(SNP_ERR_INVALID, "ELL output too small");
    for (int64_t x = 0; x < rows * m; ++x) {
        values[x] = 0;
        neurons[x] = -1;
    }
    for (int64_t i = 0; i < q; ++i)
        for (int64_t r = d->rule_offsets[i]; r < d->rule_offsets[i + 1]; ++r) {
            values[r] = -d->rule_c[r];   // row 0: consumption at the owner
            neurons[r] = (int32_t)i;
            if (d->rule_p[r] == 0) continue;  // forgetting rules have no +p entries
            int64_t row = 1;
            for (int64_t e = d->syn_offsets[i]; e < d->syn_offsets[i + 1]; ++e, ++row) {
                values[row * m + r] = d->rule_p[r];
                neurons[row * m + r] = d->syn_targets[e];
            }
        }
    return SNP_OK;
}

extern "C" int snp_export_compressed(const snp_desc* d, int32_t* sy, int64_t capacity, int64_t* rows_out) {
    int st = snp::validate_desc(d);
    if (st) return st;
    const int64_t q = d->q;
    int64_t z = 0;
    for (int64_t i = 0; i < q; ++i) z = std::max<int64_t>(z, d->syn_offsets[i + 1] - d->syn_offsets[i]);
    if (rows_out) *rows_out = z;
    if (!sy) return SNP_OK;
    if (capacity < z * q) return snp::fail(SNP_ERR_INVALID, "compressed output too small");
    for (int64_t x = 0; x < z * q; ++x) sy[x] = -1;
    for (int64_t i = 0; i < q; ++i) {
        int64_t row = 0;
        for (int64_t e = d->syn_offsets[i]; e < d->syn_offsets[i + 1]; ++e, ++row) sy[row * q + i] = d->syn_targets[e];
    }
    return SNP_OK;
}

extern "C" int64_t snp_paper_format_elements(int32_t form, int64_t q, int64_t m, int64_t z) {
    switch (form) {
        case SNP_FORM_DENSE: return m * q + 3 * m + 2 * q + 1;
        case SNP_FORM_ELL: return m * (2 * z + 5) + 2 * q + 1;
        case SNP_FORM_OPT: return q * (z + 3) + 4 * m + 1;
        default: return -1;
    }
}
