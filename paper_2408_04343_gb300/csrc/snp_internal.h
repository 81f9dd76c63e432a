// Internal declarations shared by the host code and the kernels of libsnp.
#pragma once

#include <cstdint>
#include <cstddef>
#include <string>
#include <vector>

#include "../../include/snp.h"

#if defined(__CUDACC__)
#define SNP_HD __host__ __device__
#else
#define SNP_HD
#endif

namespace snp {

// Neurons are processed in slices of 32 (one warp, one neuron per lane).
constexpr int kSlice = 32;
// Status word of a neuron: low 16 bits = D (steps until it reopens), high
// bits = 1 + local index of its pending delayed rule (0 = none).
constexpr int kPendShift = 16;
constexpr uint32_t kDMask = 0xffffu;
constexpr int kMaxRulesPerNeuron = 32766;
constexpr int kMaxDelay = 65535;
constexpr int kMaxP = 65535;

// Device flag words of one system (uint32).
enum Flag : int {
    kFlagAct0 = 0,     // activity of absolute step k lives in word k mod 3 (3 words)
    kFlagHalted = 3,   // set when a step found the system at a fixed point
    kFlagOverflow = 4, // a spike count left the int32 range (sticky until reported)
    kFlagTimeout = 5,  // a bounded wait gave up
    kFlagChoice = 6,   // a forced choice index was out of range (snp_set_choices)
    kFlagImport = 7,   // smallest neuron whose imported state is invalid (snp_set_state)
    kFlagBounds = 8,   // bounds-checked builds: bit per site of an out-of-range index (SNP_IDX)
    kNumFlags = 9
};
// Device step counters of one system (uint64).
enum StepWord : int {
    kStepBase = 0,      // absolute step counter k
    kStepCallStart = 1, // k when the current snp_step call began
    kStepExec = 2,      // steps executed by the last call
    kStepHalt = 3,      // step at which the last call found a fixed point
    kNumStepWords = 4
};

// Compact rule word: k(8) | j(8) << 8 | c(8) << 16 | p(4) << 24 | d(4) << 28.
// General rule: 4 words {k, j, c, p | d << 16}.
SNP_HD inline uint32_t pack_rule_compact(uint32_t k, uint32_t j, uint32_t c,
                                                      uint32_t p, uint32_t d) {
    return k | (j << 8) | (c << 16) | (p << 24) | (d << 28);
}

// Everything a kernel needs about one system (device pointers, slot order).
struct DevSys {
    int32_t q;           // neurons (slots); slot q is a dummy that never emits
    int32_t nslices;     // ceil(q / 32)
    const int32_t* slice_ptr;  // [nslices+1] in-list slice starts, units of 32 entries
    const int32_t* in_idx;     // in-lists, sliced ELL column-major, pad = q
    const int32_t* out_ptr;    // [nslices+1] out-list slice starts (push), units of 32
    const int32_t* out_idx;    // out-lists, sliced ELL column-major, pad = -1
    const int32_t* rule_off;   // [q+1] rule offsets in slot order
    const uint32_t* rules;     // compact words or 4 words per rule
    const int32_t* orig;       // [q] slot -> caller's neuron id
    int32_t* C;                // [q] spikes
    uint32_t* st;              // [q] status word
    int32_t* E[2];             // [q+1] emissions of step k in E[k & 1]
    int32_t* S[2];             // [q] local index of the selected rule, -1
    uint32_t* flags;           // [kNumFlags]
    unsigned long long* step;  // [kNumStepWords] step counters
    uint64_t seed;
    int32_t select;
    int32_t max_p;
    const void* rec;           // [q] 16-byte compiled rule records, or NULL (see compile_rules)
    uint32_t philox_rk[20];    // Philox4x32-10 round keys of seed (philox_round_keys)
    const int32_t* forced;     // [q] slot order: forced choice index of each neuron, or NULL (see select_forced)
    int32_t rules_per_neuron;  // > 0: every neuron has this many rules (rule r0 = slot * R)
    int32_t identity;          // 1: slot order is the caller's order (orig[slot] = slot)
};

// Host-side packed form of a system (slot order).
struct HostPack {
    int32_t q = 0;
    int64_t m = 0, nsyn = 0;
    int32_t max_rules = 0, max_p = 0, max_d = 0, max_out = 0, max_in = 0;
    int32_t uniform_rules = 0;  // > 0: every neuron has this many rules
    bool identity = false;      // slot order == caller's order
    bool compact = true;
    std::vector<int32_t> perm;        // slot -> neuron
    std::vector<int32_t> inv;         // neuron -> slot
    std::vector<int32_t> rule_off;    // [q+1] slot order
    std::vector<uint32_t> rules;      // compact: m words; general: 4m words (+ 2 per union term)
    std::vector<int32_t> rule_base;   // [q] caller's id of the slot's first rule
    std::vector<int32_t> slice_ptr;   // [nslices+1]
    std::vector<int32_t> in_idx;
    std::vector<int32_t> out_ptr;     // push only
    std::vector<int32_t> out_idx;
    std::vector<int32_t> C0;          // slot order
    std::vector<uint32_t> rec;        // compiled rule records, 4 words per slot (empty: not compiled)
};

// Compiled rule records.  For a neuron with at most four rules, which rules
// apply depends on n only through min(n, K) and (n - K) mod L once n >= K,
// with K = 1 + the largest k or c of its rules and L the least common
// multiple of its nonzero j: above K every exact rule (j = 0) fails and every
// other rule's test (n - k) mod j = 0 repeats with period L.  When K + L <= 14
// the whole applicability function fits a table of K + L four-bit masks:
//   word 0: masks of table entries 0..7 (entry e in bits 4e..4e+3);
//   word 1: masks of entries 8..13, K in bits 24..27, L in bits 28..31;
//   words 2-3: per rule t, 16 bits (c: 6, p: 5, d: 5) at bits 16(t mod 2) of
//   word 2 + t/2.
// Entry e is the mask for n = e when e < K and for n = K + ((n - K) mod L)
// otherwise.  A system is compiled only if every neuron fits (c < 64,
// p < 32, d < 32); then one 16-byte load replaces the per-rule tests.
bool compile_rules(const snp_desc* d, HostPack* hp);

// The ten round keys of Philox4x32-10 for key (seed mod 2^32, seed >> 32):
// round r uses the key advanced by r Weyl increments (0x9E3779B9,
// 0xBB67AE85), as the generator's definition (Salmon et al., SC'11) gives.
inline void philox_round_keys(uint64_t seed, uint32_t rk[20]) {
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        rk[2 * r] = k0;
        rk[2 * r + 1] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
}

constexpr int kTiledMaxSub = 8;  // target windows per CTA of the tiled engine
constexpr int kTiledThreads = 1024;  // threads of a tiled gather CTA (the entry layout depends on it)
constexpr int kTiledMaxCluster = 8;  // up to this many partitions: one fused launch per step (a cluster per range)
constexpr double kTiledPairSlack = 0.125;  // largest padding of the paired layout

// Layout of the tiled engine (shared-memory emissions, source partitions).
// Sources are cut into P partitions of part_size slots so that one
// partition's bit-packed emissions fit in shared memory.  Slices are cut into
// G/P ranges; CTA g*P + h owns range g and partition h, and the in-edges of
// its range that come from partition h form one contiguous group of 32-bit
// words (dst << src_bits) | src, src the source slot relative to the
// partition start.  A word has 32 - src_bits bits for the target, too few
// for a whole range, so the group is cut into up to kTiledMaxSub target
// windows of 2^(32 - src_bits) slots; dst is relative to its window and the
// kernel knows the window from the word's position (window boundaries in
// `sub`).  Inside a window the words are sorted by target.  In the paired
// layout each target's words are padded to an even count, so every aligned
// pair of words shares one target and the kernel adds the pair's two
// emissions with one reduction; it is used when the padding adds at most
// kTiledPairSlack of the words (systems whose targets mostly have one
// in-edge per partition would nearly double).  Otherwise the words of one
// target are merely adjacent and the kernel merges runs of equal targets
// within a 16-byte load.  Pad words have source part_size, which reads a
// zero word; windows are padded to 16 bytes with them so they load as
// 16-byte vectors.
// Storage order: the N 16-byte vectors of a CTA's group, in the sorted order
// above (window bounds in `sub` count in that order), are dealt out to the
// kTiledThreads threads of the CTA in contiguous runs -- thread t takes n or
// n - 1 consecutive vectors, n = ceil(N / T), the first r = N - (n-1)T
// threads n -- and stored so that the u-th vector of every thread is
// adjacent: vector u of thread t sits at group offset u*T + t.  A warp's
// load is then one contiguous 512-byte line set, while its lanes work on
// targets far apart (no two lanes reducing into one accumulator).
// Run-length layout (when the source field fits 20 bits): the target is not
// stored.  A CTA's target-sorted in-edges are cut into kTiledThreads runs of
// nearly equal length; each entry is 24 bits, src | delta << src_bits, delta
// (24 - src_bits bits) = how many targets to advance before this entry, 0
// on a run's first entry, whose target is tstart[thread]; longer gaps take
// pad entries (source part_size, the zero word).  Five entries fill a
// 16-byte vector (bits 24i..24i+23, the top 8 bits zero); each run is padded
// with zero-delta pads to the CTA's longest run, and the vectors are stored
// in the thread-contiguous order above (every thread has the same count).
struct TiledPack {
    int e_bits = 0;          // bits per emission (2, 4, 8, 16)
    int P = 0;               // partitions
    int part_size = 0;       // slots per partition (multiple of 512)
    int part_words = 0;      // 32-bit words of one partition's emissions
    int G = 0;               // CTAs of a launch: one per (slice range, partition)
    int max_slices = 0;      // most slices given to one CTA
    int acc_words = 0;       // shared in-flow accumulators per CTA (+ dummy)
    int src_bits = 0;        // low bits of an entry holding the source (0..part_size)
    int pairs = 0;           // 1: paired layout (every aligned word pair has one target)
    int rle = 0;             // 1: run-length layout (24-bit entries, see below)
    int rin_words = 0;       // > 0: words of the partners' in-flow buffer in shared memory
    int acc8 = 0;            // 1: byte accumulators (run-length layout, P <= kTiledMaxCluster)
    int rin_esm = 0;         // 1: the partner buffer occupies the emissions' region (after the gathers)
    std::vector<int32_t> tstart;  // run-length layout: [G][kTiledThreads] first target of each thread's run
    std::vector<int32_t> sub;     // [G][kTiledMaxSub+1] window starts in ent (CTA g*P+h: range g, partition h)
    std::vector<uint32_t> ent;    // entries
    std::vector<int32_t> cta_lo;  // [G/P + 1] first slice of each range
};

// Layouts of the ELL form (Sec. 4, M^s_Pi: a column per rule of (neuron,
// value) pairs) and of the uncompressed "Sparse" form (Table 1, M_Pi).
// Rule ids are slot-order ids (rule_off[slot] + local index).  The
// consumption pair (-c, own neuron) of M^s_Pi's row 0 is not stored: with
// delays a rule consumes when it fires and emits d steps later, so the
// consumption is applied by the select phase in every form.
//  * in-ELL (pull): per target slot, one (rule, p) pair for every firing
//    rule of every in-neighbour -- the transpose of the +p rows of M^s_Pi --
//    as sliced ELL (32 targets per slice, column-major pairs, pad (m, 0));
//  * out-ELL (push): per rule, its column's +p pairs (target slot, p) as
//    sliced ELL (32 rules per slice, column-major, pad (-1, 0));
//  * dense: M_Pi's positive part, m x q int32 row-major in slot order.
struct EllPack {
    std::vector<int32_t> in_ptr;   // [nslices+1], units of 32 pairs
    std::vector<int32_t> in_ent;   // pairs as 2 int32 (rule, p)
    std::vector<int32_t> out_ptr;  // [ceil(m/32)+1], units of 32 pairs
    std::vector<int32_t> out_ent;  // pairs as 2 int32 (target, p)
};
int pack_ell(const snp_desc* d, const HostPack& hp, bool want_pull, bool want_push, EllPack* out);
int pack_dense(const snp_desc* d, const HostPack& hp, std::vector<int32_t>* M);

// Bits per packed emission for the largest p of a system.
int tiled_e_bits(int max_p);
// Builds the tiled layout; returns SNP_ERR_UNSUPPORTED when no partitioning
// fits the shared-memory budget and the 32-bit entry encoding.
// cpw[P] (P = 1 .. kTiledMaxCluster, may be NULL): clusters of P CTAs the
// device runs at once; a wave has that many ranges (else G / P).
int pack_tiled(const snp_desc* d, const HostPack& hp, int G, size_t smem_budget, TiledPack* out,
               const int* cpw = nullptr);
size_t tiled_smem_bytes(const TiledPack& tp);

// Thread-local error text for snp_last_error().
void set_error(const std::string& msg);
int fail(int status, const std::string& msg);
const char* last_error();

// Validation and packing (pack.cpp).  window: in-degree sort window (slots).
int validate_desc(const snp_desc* d);
int pack_system(const snp_desc* d, bool want_out_lists, bool want_in_lists, int window, HostPack* out);
// Fills hp->in_idx (sliced ELL) from an already packed slot order.
void pack_in_lists(const snp_desc* d, HostPack* hp);

}  // namespace snp
