/*
 * libsnp -- a GB300 (sm_103a) simulator of spiking neural P systems with
 * delays over compressed sparse representations.
 *
 * Paper: J. Hernandez-Tello, M.A. Martinez-del-Amor, D. Orellana-Martin,
 * F.G.C. Cabarle, "Sparse Spiking Neural-like Membrane Systems on Graphics
 * Processing Units", IJNS 34(7) 2450038, 2024 (arXiv 2408.04343).
 *
 * Conventions for every call below:
 *  - Every call returns an int status: SNP_OK (0) or one of SNP_ERR_*.  No
 *    C++ exception crosses this boundary.  snp_last_error() returns a
 *    thread-local message about the last failure on the calling thread.
 *  - Input arrays are owned by the caller and copied before the call returns.
 *  - Handles (snp_system, snp_batch) are owned by the library and released
 *    with the matching destroy call.
 *  - Output pointers may be host or device memory; the library asks the
 *    CUDA runtime which one it was given.  Copies to host memory complete
 *    before the call returns; copies to device memory are ordered on the
 *    system's stream.
 *  - All device work of a system is ordered on the stream given at creation
 *    (options.stream; NULL = the legacy default stream).
 *  - Neuron and rule numbering at this boundary is the caller's: neuron i
 *    is position i of init_spikes, rule r is position r of the rule arrays.
 *    Internally neurons are renumbered (sorted by in-degree); that order
 *    never leaks out.
 */
#ifndef SNP_H
#define SNP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define SNP_OK 0
#define SNP_ERR_INVALID 1     /* bad argument or malformed system          */
#define SNP_ERR_OOM 2         /* device or host allocation failed          */
#define SNP_ERR_CUDA 3        /* a CUDA runtime call failed                */
#define SNP_ERR_TIMEOUT 4     /* a bounded device-side wait gave up        */
#define SNP_ERR_OVERFLOW 5    /* a spike count left the int32 range        */
#define SNP_ERR_BUSY 6        /* system is owned by an unfinished batch    */
#define SNP_ERR_UNSUPPORTED 7 /* option combination not available          */

/* ---- options ----------------------------------------------------------- */
/* Representation of the transition matrix (Sec. 4):
 *   SNP_FORM_OPT   -- the "Compressed"/"optimized" form: rule vector with
 *                     (c, p) per rule plus per-neuron synapse lists;
 *   SNP_FORM_ELL   -- the ELL form: per-rule columns of (neuron, value);
 *   SNP_FORM_DENSE -- the uncompressed m x q matrix (the paper's "Sparse"
 *                     format), a baseline for small systems only.          */
#define SNP_FORM_OPT 0
#define SNP_FORM_ELL 1
#define SNP_FORM_DENSE 2
/* Direction of spike propagation:
 *   SNP_PROP_PULL -- every neuron sums over its in-neighbours (no atomics);
 *   SNP_PROP_PUSH -- every emitter adds into its targets with atomics, as
 *                    Algorithms 4 and 5 do (warp-aggregated).              */
#define SNP_PROP_PULL 0
#define SNP_PROP_PUSH 1
/* Choice of one applicable rule per neuron (Sec. 5, SV_CALC/SAMPLE_ONE):
 *   SNP_SELECT_FIRST  -- the lowest-index applicable rule (the paper's
 *                        deterministic choice);
 *   SNP_SELECT_PHILOX -- uniform over the applicable rules, drawn from
 *                        Philox4x32-10 (Salmon et al., SC'11): the four
 *                        words of the block at counter (k mod 2^32, i / 4,
 *                        k >> 32, 0) and key (seed mod 2^32, seed >> 32)
 *                        serve neurons 4(i / 4) .. 4(i / 4) + 3 at step k,
 *                        neuron i taking word x = word i mod 4; the index
 *                        into the applicable list is floor(x |A| / 2^32). */
#define SNP_SELECT_FIRST 0
#define SNP_SELECT_PHILOX 1
/* How snp_step runs its steps:
 *   SNP_ENGINE_AUTO     -- library's choice by size;
 *   SNP_ENGINE_LAUNCH   -- one grid-wide launch per step (CUDA graph of
 *                          launches), every CTA working on one step;
 *   SNP_ENGINE_RESIDENT -- one CTA owns the whole system and runs all steps
 *                          in one launch with the spike emissions kept in
 *                          shared memory (systems whose two bit-packed
 *                          emission vectors fit in one CTA's shared memory,
 *                          about 460,000 neurons at 4 bits).               */
#define SNP_ENGINE_AUTO 0
#define SNP_ENGINE_LAUNCH 1
#define SNP_ENGINE_RESIDENT 2
/*   SNP_ENGINE_TILED    -- one grid-wide launch per step like LAUNCH, but
 *                          every CTA copies the bit-packed emission vector
 *                          into shared memory (in source partitions when it
 *                          does not fit at once) so in-neighbour reads are
 *                          shared-memory reads; the default for large
 *                          systems under AUTO.                              */
#define SNP_ENGINE_TILED 3

/* Optional device allocator (e.g. a framework's caching allocator).  Both
 * callbacks are called on the thread that calls into the library, except
 * for a system that a batch uploads at admission (SNP_FLAG_DEFER_UPLOAD):
 * its alloc runs on the batch's upload thread.                            */
typedef struct snp_allocator {
    void* (*alloc)(void* ctx, size_t bytes, void* stream); /* NULL = OOM */
    void (*release)(void* ctx, void* ptr, size_t bytes, void* stream);
    void* ctx;
} snp_allocator;

typedef struct snp_options {
    int32_t form;     /* SNP_FORM_*                                   */
    int32_t prop;     /* SNP_PROP_*                                   */
    int32_t select;   /* SNP_SELECT_*                                 */
    int32_t engine;   /* SNP_ENGINE_*                                 */
    uint64_t seed;    /* Philox key of this system                    */
    void* stream;     /* cudaStream_t; NULL = legacy default stream   */
    const snp_allocator* alloc; /* NULL = cudaMalloc/cudaFree         */
    int32_t threads;  /* CTA size hint for the kernels; 0 = default   */
    int32_t flags;    /* SNP_FLAG_* bits                              */
} snp_options;

/* snp_create packs the system on the host but allocates and uploads nothing
 * until the system is first stepped, read, or admitted by a batch (which
 * then counts its memory against the batch budget).                       */
#define SNP_FLAG_DEFER_UPLOAD 1

/* A system Pi = (O, syn, sigma_1..sigma_q, i_out) (Sec. 2) as the user
 * defines it (Sec. 5, "Initialization").  All arrays are HOST memory.
 *
 *   init_spikes[q]     n_i, the initial configuration C_0 (>= 0).
 *   rule_offsets[q+1]  N_Pi: the rules of neuron i are rule_offsets[i] ..
 *                      rule_offsets[i+1]-1 (rule_offsets[0] = 0, monotone,
 *                      at most 32766 rules per neuron).
 *   rule_k/j/c/p/d[m]  rule r is E/a^c -> a^p; d with the regular expression
 *                      E = a^k (a^j)* (j = 0: exactly a^k).  The paper's
 *                      three regex types map to (k = n, j = 0) for a^n,
 *                      (k = 0, j = 1) for a* and (k = 1, j = 1) for a+.
 *                      A forgetting rule a^s -> lambda is k = c = s, j = 0,
 *                      p = 0, d = 0.  Ranges: k, j, c >= 0; 0 <= p <= 65535;
 *                      0 <= d <= 65535; p = 0 requires d = 0.
 *   num_syn            |syn|.
 *   syn_offsets[q+1]   out-list of neuron i: syn_targets[syn_offsets[i] ..
 *   syn_targets[]      syn_offsets[i+1]-1]; no self-loops, no duplicates.
 *   out_neuron         i_out (kept, not used by the step).
 *   rule_term_offsets  optional (NULL: every rule has the single term
 *     [m+1]            (rule_k, rule_j)).  When set, rule r's expression is
 *   term_k/term_j[]    the finite union of a^term_k[t] (a^term_j[t])* over
 *                      t = rule_term_offsets[r] .. rule_term_offsets[r+1]-1
 *                      (the type-4 form of Sec. 7, several terms per rule):
 *                      the rule applies to n spikes when n >= c and n is in
 *                      any term's language.  rule_k and rule_j are then not
 *                      read and may be NULL.  rule_term_offsets[0] = 0,
 *                      monotone, at least one term per rule; term_k, term_j
 *                      >= 0.  When every neuron has at most 4 rules,
 *                      c < 64, p < 32, d < 32 and K + L <= 14 (K = 1 + the
 *                      largest term_k or c of the neuron, L the lcm of its
 *                      non-zero term_j) the step reads one compiled 16-byte
 *                      applicability table per neuron; otherwise it tests
 *                      each rule's terms (any number of rules and terms,
 *                      the ranges above).
 *                      Zero-initialise the struct so that callers unaware
 *                      of these fields leave them NULL.                  */
typedef struct snp_desc {
    int32_t q;
    const int32_t* init_spikes;
    const int64_t* rule_offsets;
    const int32_t* rule_k;
    const int32_t* rule_j;
    const int32_t* rule_c;
    const int32_t* rule_p;
    const int32_t* rule_d;
    int64_t num_syn;
    const int64_t* syn_offsets;
    const int32_t* syn_targets;
    int32_t out_neuron;
    const int64_t* rule_term_offsets;
    const int32_t* term_k;
    const int32_t* term_j;
} snp_desc;

/* Sizes of a created system, for accounting and roofline arithmetic. */
typedef struct snp_info {
    int32_t q;
    int32_t form, prop, select, engine;
    int64_t m;
    int64_t num_syn;
    int64_t in_entries;      /* stored in-list entries incl. padding       */
    int64_t out_entries;     /* stored out-list entries incl. padding      */
    int64_t rule_words;      /* 32-bit words of the stored rule table      */
    int64_t device_bytes;    /* device memory held by the system           */
    int32_t max_rules;       /* largest |R_i|                              */
    int32_t max_p;           /* largest p                                  */
    int32_t compact_rules;   /* 1 if rules are stored in one word each     */
    int32_t e_bits;          /* bits per stored emission in shared memory  */
    uint64_t step;           /* absolute step counter k                    */
    int32_t compiled_rules;  /* 1 if the select phase reads one 16-byte    */
                             /* applicability record per neuron instead    */
                             /* of testing each rule (Compressed form with */
                             /* at most 4 small rules per neuron)          */
    /* The tiled engine's launch shape (all 0 when the system has none):   */
    int32_t tiled_partitions; /* source partitions P = CTAs per cluster    */
    int32_t tiled_ctas;       /* CTAs of one step launch (ranges x P)      */
    int32_t tiled_layout;     /* in-edge entries: 0 target words, 1 paired */
                              /* target words, 2 run-length entries        */
    int32_t tiled_acc_bits;   /* width of the in-flow accumulators: 8, 32  */
    int64_t tiled_smem_bytes; /* dynamic shared memory per CTA            */
} snp_info;

typedef struct snp_system snp_system;
typedef struct snp_batch snp_batch;

/* Builds a system from its description (Sec. 5, "Initialization"): validates
 * it, packs the rule vector RV_Pi, the neuron-rule map N_Pi and the synapse
 * lists straight from the edge list (no dense intermediate), uploads them
 * and sets C = C_0, D = 0, no pending rules, k = 0 (Alg. 1, INIT).
 * Returns SNP_ERR_INVALID for malformed input (self-loop, duplicate synapse,
 * out-of-range id or field), SNP_ERR_OOM when memory runs out.            */
int snp_create(const snp_desc* desc, const snp_options* opts, snp_system** out);

/* Releases a system and its device memory.  NULL is accepted.            */
int snp_destroy(snp_system* sys);

/* Runs up to n transition steps (Alg. 1's loop body: SV_CALC with the
 * choice, STEP and UPDATE_DELAYS) and stops early at a fixed point, i.e.
 * when no neuron is pending and no open neuron has an applicable rule.
 * If steps_done is not NULL the call waits for the device and stores the
 * number of steps executed; if it is NULL the call returns once the work is
 * queued on the system's stream.  Returns SNP_ERR_OVERFLOW when a spike
 * count left the int32 range (checked when the call waits).              */
int snp_step(snp_system* sys, int64_t n, int64_t* steps_done);

/* C_k: spikes per neuron, out[q].                                          */
int snp_get_config(const snp_system* sys, int32_t* out, int64_t len);
/* S_k of the last executed step: per neuron the global id of the rule it
 * selected at that step, or -1 (Sec. 4, the Compressed spiking vector of
 * length q with 0-based rule ids).  All -1 before the first step.         */
int snp_get_spiking(const snp_system* sys, int32_t* out, int64_t len);
/* D_k: per neuron the number of steps before it reopens, 0 = open (Sec. 2,
 * delays vector).                                                          */
int snp_get_status(const snp_system* sys, int32_t* out, int64_t len);
/* Pending delayed rule per neuron (global rule id) or -1.                 */
int snp_get_pending(const snp_system* sys, int32_t* out, int64_t len);
/* Checkpoint: (C, D, P) as above plus the absolute step counter k.  Any
 * of C, D, P may be NULL for get_state.  set_state takes all three, in host
 * (pageable or pinned) or device memory, and validates them on the device
 * (C >= 0; 0 <= D <= 65535; a pending rule must belong to its neuron; D > 0
 * only with a pending rule): SNP_ERR_INVALID names the smallest offending
 * neuron and leaves C, D, P and k unchanged.  Either way the spiking vector
 * then reads all -1.                                                       */
int snp_get_state(const snp_system* sys, int32_t* C, int32_t* D, int32_t* P, int64_t len,
                  uint64_t* step);
int snp_set_state(snp_system* sys, const int32_t* C, const int32_t* D, const int32_t* P,
                  int64_t len, uint64_t step);
int snp_get_info(const snp_system* sys, snp_info* info);

/* ---- computation-tree exploration (Sec. 2 SV_k; Sec. 5's future work) ----
 * The paper's semantics are nondeterministic: at step k every idle open
 * neuron with applicable rules picks one of them, and each combination is a
 * spiking vector of SV_k, one branch of the computation tree.  These two
 * calls let a caller walk that tree with the library's own step:
 *
 * snp_count_choices: out[i] (caller's neuron ids, host or device buffer,
 *   len >= q) = how many rules neuron i may choose at the next step -- the
 *   applicable rules of an idle open neuron, 0 while a rule is pending.  The
 *   branches of the next step are the products of these counts.
 * snp_set_choices: idx[i] (host or device, len >= q, copied) = which of
 *   neuron i's applicable rules (0-based, in rule order) the FIRST step of
 *   the next snp_step call takes, instead of the system's selection; neurons
 *   with no applicable rule ignore their entry.  The call's later steps
 *   select as usual.  An index outside 0 .. count-1 makes that snp_step
 *   return SNP_ERR_INVALID (the step has run, with the neuron's first rule).
 * Both return SNP_ERR_BUSY while a batch owns the system.                  */
int snp_count_choices(const snp_system* sys, int32_t* out, int64_t len);
int snp_set_choices(snp_system* sys, const int32_t* idx, int64_t len);

/* snp_branch_step: one forced step of nb configurations of the system at
 * once (a level of the computation tree in one launch), leaving the
 * system's own state untouched.  Arrays are [nb][q] int32 in the caller's
 * neuron order, host or device: C, D (steps until the neuron reopens), P
 * (global id of the pending rule, -1 none) and choices (as snp_set_choices)
 * in; C_out, D_out, P_out out; executed[nb] = 1, or 0 for a configuration
 * at a fixed point (copied unchanged); bad[nb] = 1 when one of its choice
 * indices was out of range (that neuron took its first applicable rule);
 * counts (optional, NULL to skip) = snp_count_choices of each resulting
 * configuration, the branching of the next level.
 * Needs the optimized form with in-neighbour lists (the launch or resident
 * engine, or AUTO) and q <= 8192: SNP_ERR_UNSUPPORTED otherwise.
 * SNP_ERR_OVERFLOW if a spike count left the int32 range.                 */
int snp_branch_step(snp_system* sys, int32_t nb, const int32_t* C, const int32_t* D, const int32_t* P,
                    const int32_t* choices, int32_t* C_out, int32_t* D_out, int32_t* P_out, int32_t* executed,
                    int32_t* bad, int32_t* counts);

/* ---- batched and served forms ----------------------------------------- */
/* A batch runs many independent systems in one persistent launch, each
 * system owned by one CTA for all its steps, systems taken largest first
 * from a device work counter.  Admitted systems are uploaded by a thread of
 * the batch while the systems already running keep stepping; they join the
 * next round once uploaded.  mem_budget (bytes) bounds the device memory
 * of the systems the batch uploaded (created with SNP_FLAG_DEFER_UPLOAD)
 * and that are not yet destroyed; 0 = no bound.  The bound is hard: the
 * first waiting system is admitted only when it fits beside them.  A
 * finished system keeps its memory until snp_destroy (its state is still
 * read), so callers make room by destroying finished systems.             */
int snp_batch_create(const snp_options* opts, size_t mem_budget, snp_batch** out);
int snp_batch_destroy(snp_batch* b);
/* Queues count systems, each to advance steps[i] steps (stopping early at
 * a fixed point).  The systems must have been created with the same form
 * and must not be stepped or read until the ticket completes (calls on them
 * return SNP_ERR_BUSY meanwhile).  Work is admitted as memory allows and
 * overlaps with work already running.                                     */
int snp_batch_submit(snp_batch* b, snp_system* const* sys, const int64_t* steps, int32_t count,
                     int64_t* ticket);
int snp_batch_poll(snp_batch* b, int64_t ticket, int* done);
/* Blocks until the ticket completes (SNP_OK, or the first error of its
 * systems).  Returns SNP_ERR_BUSY instead of blocking forever when the
 * ticket waits for memory that only a destroy can free: nothing runs and
 * the first waiting system does not fit beside the finished ones still
 * held.  Destroy finished systems, then wait again.  Systems still waiting
 * when the batch is destroyed are released unrun (their tickets complete
 * with SNP_ERR_BUSY).                                                      */
int snp_batch_wait(snp_batch* b, int64_t ticket);
/* Executed steps of system `index` of a completed ticket.                 */
int snp_batch_steps_done(snp_batch* b, int64_t ticket, int32_t index, int64_t* steps_done);
/* Counters of a batch: device bytes of the systems it holds now and at most
 * so far, rounds run, systems admitted / finished / waiting / running, and
 * where its worker's time went since creation (seconds, host clock unless
 * noted): uploading admitted systems; queueing the grid-wide systems' steps
 * of each round; the CTA-resident launches of each round from table upload
 * to results (their device time by CUDA events beside it); waiting for the
 * grid-wide systems after those launches; idle (nothing admissible and
 * nothing running); whole rounds.                                         */
typedef struct snp_batch_info {
    uint64_t budget_bytes;
    uint64_t resident_bytes;
    uint64_t peak_resident_bytes;
    int64_t rounds;
    int64_t admitted;
    int64_t finished;
    int64_t waiting;
    int64_t running;
    double admit_seconds;
    double launch_seconds;
    double resident_seconds;
    double resident_device_seconds;
    double large_tail_seconds;
    double idle_seconds;
    double round_seconds;
} snp_batch_info;
int snp_batch_get_info(snp_batch* b, snp_batch_info* info);

/* ---- the neuron-sharded step (one system over several devices) ----------
 * The paper simulates a system on one GPU; its future work names larger
 * systems.  A system too large for one device is split by neuron range into
 * shards, one per device.  Each step of the definition needs data of other
 * neurons at one point only -- the in-flow of phase 2 (Sec. 2: a neuron
 * receives the spikes its in-neighbours emit) -- so a step of the sharded
 * system is, on every shard: snp_shard_select (phase 1 for the shard's
 * neurons: complete / count down / choose a rule and consume, the delay
 * status; their emissions go into the shard's slice [lo, hi) of its
 * emission vector), then the caller exchanges the slices so that every
 * shard's vector holds all q emissions (an allgather, 2 bytes per neuron)
 * and ORs the shards' `active` flags (the fixed point of Alg. 1: no shard
 * active means the step is not executed and nothing changed), then
 * snp_shard_gather (phase 2 for the shard's neurons from the whole vector).
 * Results equal the unsharded system's, step for step (the Philox counter
 * keeps the global neuron id).
 *
 * snp_shard_create: the shard of neurons lo..hi-1 (0 <= lo < hi <= q) of
 *   the system desc (validated as by snp_create; the whole desc is read,
 *   the shard keeps its neurons' rules, state and in-lists with global
 *   source ids).  E: the emission vector, DEVICE memory of at least q + 1
 *   uint16 entries owned by the caller (so that a collective library can
 *   write into it), or NULL to let the shard allocate it.  opts: select,
 *   seed, stream (form, engine, allocator and flags are not used).  The
 *   state starts at C_0, no delays, step counter chosen by the caller.
 * snp_shard_emissions: the device address of the emission vector.
 * snp_shard_select(k): phase 1 of step k; waits for the device and sets
 *   *active.  SNP_ERR_OVERFLOW if an earlier phase 2 left int32 range.
 * snp_shard_gather: phase 2 of the step last selected (queued on the
 *   stream); marks that step executed.
 * snp_shard_get_state: C, D, P and the spiking vector of the last executed
 *   step (global rule ids, -1 none) of the shard's neurons, hi - lo entries
 *   each (host or device).                                                */
typedef struct snp_shard snp_shard;
int snp_shard_create(const snp_desc* desc, int32_t lo, int32_t hi, const snp_options* opts, uint16_t* E,
                     snp_shard** out);
int snp_shard_destroy(snp_shard* sh);
int snp_shard_emissions(snp_shard* sh, uint16_t** E);
int snp_shard_select(snp_shard* sh, uint64_t k, int32_t* active);
int snp_shard_gather(snp_shard* sh);
int snp_shard_get_state(const snp_shard* sh, int32_t* C, int32_t* D, int32_t* P, int32_t* S, int64_t len);

/* ---- paper formats, host only (inspection and memory accounting) -------- */
/* The paper's matrices for a system, written densely on the host:
 *   snp_export_dense: M_Pi, m x q row-major (Table 1 layout);
 *   snp_export_ell:   M^s_Pi, z' = max out-degree + 1 rows x m columns,
 *                     row-major, values[] and neurons[] with -1 neuron for
 *                     null; the consumption pair (-c, own neuron) is row 0
 *                     (Table 2 layout);
 *   snp_export_compressed: Sy_Pi, z = max out-degree rows x q columns,
 *                     row-major, -1 for null (Table 3 layout).
 * rows_out (may be NULL) receives the number of rows; capacity is the
 * number of int32 elements each output array holds.                       */
int snp_export_dense(const snp_desc* desc, int32_t* M, int64_t capacity);
int snp_export_ell(const snp_desc* desc, int32_t* values, int32_t* neurons, int64_t capacity,
                   int64_t* rows_out);
int snp_export_compressed(const snp_desc* desc, int32_t* sy, int64_t capacity, int64_t* rows_out);
/* Element counts of the paper's three formats (Sec. 6):
 *   SNP_FORM_DENSE: m q + 3m + 2q + 1; SNP_FORM_ELL: m (2z + 5) + 2q + 1;
 *   SNP_FORM_OPT: q (z + 3) + 4m + 1, z = max out-degree.                 */
int64_t snp_paper_format_elements(int32_t form, int64_t q, int64_t m, int64_t z);

/* ---- stepping without allocation ----------------------------------------- */
/* The paper has no counterpart to this call; it exists for callers of this
 * library that cannot call cudaMalloc: code living inside a host framework
 * that owns all device memory and hands it out only through its own pool
 * (plugins, custom operators), and latency-critical loops in which an
 * allocation could synchronize the device at an unpredictable moment.
 *
 * snp_step_noalloc runs up to n pull steps (same semantics, selection and
 * results as snp_step) on a system whose tables and state the caller keeps
 * in its own DEVICE arrays, in the caller's neuron and rule numbering:
 *   rule_offsets[q+1], rule_k/j/c/p/d[m]  as in snp_desc, but int32 and on
 *                                         the device;
 *   in_offsets[q+1], in_sources[num_in]  the in-neighbours of neuron j are
 *                                         in_sources[in_offsets[j] ..
 *                                         in_offsets[j+1]-1] (the transpose
 *                                         of the synapse lists);
 *   C, D, P [q]   the state (spikes, steps until reopening, pending rule
 *                 or -1) at absolute step `step`; read and overwritten with
 *                 the state after the executed steps;
 *   S [q]         receives the spiking vector (global rule ids, -1 none) of
 *                 the last executed step; untouched if no step executes.
 * The library allocates nothing: its working memory (two emission vectors
 * and a few flag words, about 2 MB) is one static device array that every
 * GPU which loads the library holds until the process exits, which caps q
 * at SNP_NOALLOC_MAX_Q; larger q returns SNP_ERR_INVALID.  The first call
 * on a device looks up that array's device address (cudaGetSymbolAddress,
 * with the device current) and keeps it for the life of the process; make
 * that first call before any stream capture.  A process that resets a
 * device (cudaDeviceReset) must not call snp_step_noalloc on it afterwards:
 * the kept address belonged to the destroyed context.
 * All calls share the one array and the next call overwrites it (the flag
 * words are cleared at the start of every call), so calls whose work
 * overlaps on the GPU, from any thread or stream, race and must be
 * serialised by the caller.  Work is ordered on `stream`; with steps_done
 * non-NULL the call waits for it and reports the executed step count,
 * SNP_ERR_OVERFLOW, or SNP_ERR_INVALID if the kernels found an index in the
 * device arrays out of range, a neuron with more than 32,766 rules, a
 * state outside snp_set_state's ranges (C >= 0, 0 <= D <= 65535, P = -1 or
 * a rule of its neuron, D = 0 when P = -1), or a
 * rule that a step fires with a field outside snp_desc's ranges (k, j,
 * c >= 0; p, d in [0, 65535]; d = 0 when p = 0); such a neuron is treated as
 * idle for the rest of the call.  n is at most 2^31 - 1 (SNP_ERR_INVALID
 * beyond).                                                                 */
#define SNP_NOALLOC_MAX_Q 262144
typedef struct snp_device_system {
    int32_t q;
    int64_t m;
    int64_t num_in;
    const int32_t* rule_offsets;
    const int32_t* rule_k;
    const int32_t* rule_j;
    const int32_t* rule_c;
    const int32_t* rule_p;
    const int32_t* rule_d;
    const int32_t* in_offsets;
    const int32_t* in_sources;
    int32_t* C;
    int32_t* D;
    int32_t* P;
    int32_t* S;
} snp_device_system;
int snp_step_noalloc(const snp_device_system* sys, int32_t select, uint64_t seed, uint64_t step, int64_t n,
                     void* stream, int64_t* steps_done);

/* ---- diagnostic of the device-side wait limit --------------------------
 * No counterpart in the paper.  Every wait inside the library's kernels
 * (the tiled engine waits on a shared-memory barrier for the bulk copy of an
 * emission partition) gives up after a bounded number of polls, records the
 * fact in the system's timeout flag and returns, so that a lost completion
 * surfaces as SNP_ERR_TIMEOUT with the CUDA context still usable instead of
 * a hung GPU.  This call runs one CTA that performs the same bounded wait,
 * for at most `polls` polls (1 .. 1,000,000), on a barrier that nothing
 * completes, on the current device and a private stream.
 * Returns SNP_ERR_TIMEOUT when the wait gave up (the expected outcome),
 * SNP_OK if it completed, SNP_ERR_INVALID for polls out of range,
 * SNP_ERR_CUDA on a launch or copy failure.                               */
int snp_check_bounded_wait(int32_t polls);

const char* snp_strerror(int status);
const char* snp_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* SNP_H */
