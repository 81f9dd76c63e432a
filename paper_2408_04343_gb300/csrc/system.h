// The snp_system handle (internal).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <memory>
#include <utility>
#include <vector>

#include "kernels.h"
#include "snp_internal.h"

namespace snp {

constexpr int kChunk = 48;                 // steps per captured CUDA graph
constexpr int kMaxGraphedCall = 256;       // longest call run_steps_graphed captures whole
constexpr int kSortWindow = 8192;          // in-degree sort window (slots)
constexpr int kAutoResidentMaxQ = 8192;    // AUTO picks the resident engine up to here
constexpr int64_t kAutoResidentMaxRules = 65536;  // ... and up to this many rules (one CTA does all the work)
constexpr int kBranchMaxQ = 8192;           // snp_branch_step: one configuration per CTA, state in shared memory

// Host-side layouts of a system kept until they are uploaded.
struct HostImage {
    HostPack hp;
    TiledPack tp;
    EllPack ep;
    std::vector<int32_t> dense;
};

// One device buffer of a system: where its pointer goes, its source (or a
// fill byte when src is NULL) and its size.
struct Piece {
    void** dst;
    const void* src;
    size_t bytes;
    int fill;
};

}  // namespace snp

struct snp_system {
    snp_options opt{};
    snp_allocator alloc{};
    cudaStream_t stream = nullptr;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t chunk_exec = nullptr;
    cudaGraphExec_t call_exec = nullptr;  // a whole call of call_n steps (run_steps_graphed)
    int64_t call_n = 0;
    snp::DevSys dev{};
    snp::DevSys* d_self = nullptr;     // device copy of dev (resident engine)
    long long* d_nsteps = nullptr;
    unsigned int* d_work = nullptr;
    int32_t* d_rule_base = nullptr;
    int32_t* scratch = nullptr;
    std::vector<std::pair<void*, size_t>> allocs;
    size_t device_bytes = 0;
    int32_t q = 0;
    int64_t m = 0, nsyn = 0;
    int32_t max_p = 0, max_rules = 0;
    bool compact = true;
    bool compiled = false;     // compiled rule records uploaded (OPT form, or any form with unions)
    bool unions = false;       // rules given as unions of terms (need the compiled records)
    int32_t* d_forced = nullptr;  // [q] forced choices in slot order (allocated by snp_set_choices)
    bool choices_pending = false; // the next snp_step's first step takes d_forced
    int32_t uniform_rules = 0;
    bool identity = false;
    int64_t in_entries = 0, out_entries = 0, rule_words = 0;
    std::vector<int32_t> perm;          // slot -> caller's neuron
    std::vector<int64_t> rule_offsets;  // caller's N_Pi (for set_state checks)
    unsigned long long host_step = 0;   // last step counter read back
    std::atomic<int> busy{0};
    // tiled engine
    bool has_tiled = false;
    bool has_in_lists = false;
    snp::TiledSys tiled{};
    size_t tiled_smem = 0;
    int64_t tiled_entries = 0;
    int32_t tiled_threads = 1024;
    int32_t tiled_P = 0, tiled_G = 0, tiled_layout = 0, tiled_acc_bits = 0;  // launch shape (snp_get_info)
    // ELL and dense forms
    snp::EllSys ell{};
    // deferred upload
    std::unique_ptr<snp::HostImage> img;  // host layouts until uploaded
    bool materialized = false;
    size_t planned_bytes = 0;             // device bytes the upload will take
    struct snp_batch* owner = nullptr;    // batch that uploaded it (memory accounting)
    bool own_stream = false;              // stream created by the library
};

namespace snp {
size_t plan_bytes(const std::vector<Piece>& plan);
void build_plan(snp_system* s, std::vector<Piece>& plan);
int materialize(snp_system* s);
void batch_release(snp_system* s);
void* sys_alloc(snp_system* s, size_t bytes);
bool is_device_ptr(const void* p);
bool resident_fits(const snp_system* s, ResidentPlan* plan);
int effective_engine(const snp_system* s);
int read_flags(snp_system* s, int64_t* exec);
int run_steps(snp_system* s, int64_t n);
// The same as run_steps, for callers that run calls of one length again and
// again (the batch's rounds): a pull call on a grid-wide engine is captured
// once as one graph and replayed, one launch instead of one per step.
int run_steps_graphed(snp_system* s, int64_t n);
}  // namespace snp
