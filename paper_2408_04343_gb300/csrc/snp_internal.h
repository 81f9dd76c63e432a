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
    kNumFlags = 8
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
};

// Host-side packed form of a system (slot order).
struct HostPack {
    int32_t q = 0;
    int64_t m = 0, nsyn = 0;
    int32_t max_rules = 0, max_p = 0, max_d = 0, max_out = 0, max_in = 0;
    bool compact = true;
    std::vector<int32_t> perm;        // slot -> neuron
    std::vector<int32_t> inv;         // neuron -> slot
    std::vector<int32_t> rule_off;    // [q+1] slot order
    std::vector<uint32_t> rules;      // compact: m words; general: 4m words
    std::vector<int32_t> rule_base;   // [q] caller's id of the slot's first rule
    std::vector<int32_t> slice_ptr;   // [nslices+1]
    std::vector<int32_t> in_idx;
    std::vector<int32_t> out_ptr;     // push only
    std::vector<int32_t> out_idx;
    std::vector<int32_t> C0;          // slot order
};

// Layout of the tiled engine (shared-memory emissions, source partitions).
// Sources are cut into P partitions of part_size slots so that one
// partition's bit-packed emissions fit in shared memory.  For slice s and
// partition h, the in-neighbours of the 32 lanes that lie in h form one
// block: lane l has cnt[(s*P+h)*32+l] of them, stored "jagged column-major":
// column t holds, in lane order, the t-th entry of every lane with more than
// t entries, so a warp reads each column with one coalesced load and no
// padding.  Entries are source slots relative to the partition start.
struct TiledPack {
    int e_bits = 0;          // bits per emission (2, 4, 8, 16)
    int P = 0;               // partitions
    int part_size = 0;       // slots per partition (multiple of 512)
    int part_words = 0;      // 32-bit words of one partition's emissions
    int G = 0;               // CTAs of a launch (one range of slices each)
    int max_slices = 0;      // most slices given to one CTA
    std::vector<int32_t> blk;   // [nslices*P + 1] block starts in ent
    std::vector<uint8_t> cnt;   // [nslices*P*32] entries per lane and block
    std::vector<int32_t> ent;   // entries
    std::vector<int32_t> cta_lo;  // [G + 1] first slice of each CTA
};

// Bits per packed emission for the largest p of a system.
int tiled_e_bits(int max_p);
// Builds the tiled layout; returns SNP_ERR_UNSUPPORTED when the system does
// not fit it (a lane with more than 255 in-neighbours in one partition, or no
// partitioning fits the shared-memory budget).
int pack_tiled(const snp_desc* d, const HostPack& hp, int G, size_t smem_budget, TiledPack* out);
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
