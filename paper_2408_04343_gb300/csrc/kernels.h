// Host-side launchers of the libsnp kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include "snp_internal.h"

namespace snp {

enum PullKind : int { kPullSelectOnly = 0, kPullFused = 1, kPullGatherOnly = 2 };
enum ExportWhat : int { kExportConfig = 0, kExportStatus = 1, kExportPending = 2, kExportSpiking = 3, kExportChoices = 4 };

// Grid-wide engine (kernels_step.cu).  t is the step index relative to the
// system's device base step k.
cudaError_t launch_pull(const DevSys& s, int kind, int32_t t, cudaStream_t st, bool compact, int sel);
cudaError_t launch_push_step(const DevSys& s, int32_t t, cudaStream_t st, bool compact, int sel);
cudaError_t launch_begin(const DevSys& s, cudaStream_t st);
cudaError_t launch_advance(const DevSys& s, int32_t count, cudaStream_t st);
cudaError_t launch_finish(const DevSys& s, int32_t tail, cudaStream_t st);
cudaError_t launch_export(const DevSys& s, const int32_t* rule_base, int what, int32_t* out, int parity,
                          cudaStream_t st, bool compact = true);
// State import (snp_set_state): C, D, P in the caller's neuron order, already
// on the device.  check: records the smallest neuron id whose values are out
// of range in flags[kFlagImport] (which the caller sets to 0xffffffff first);
// commit: writes C and the status words in slot order.
cudaError_t launch_import(const DevSys& s, const int32_t* rule_base, const int32_t* C, const int32_t* D,
                          const int32_t* P, bool commit, cudaStream_t st);

// CTA-resident engine (kernels_resident.cu): each CTA takes whole systems
// from `work` (largest first as listed) and runs all their steps.
struct ResidentPlan {
    int threads;     // CTA size
    int e_bits;      // bits per emission in shared memory (4, 8, 16 or 32)
    int max_q;       // largest system of the launch
    int ctas;        // grid size
    size_t smem;     // dynamic shared memory per CTA
    bool big = false;  // the 64-register instance, one 1,024-thread CTA per system
};
int resident_e_bits(int max_p);
size_t resident_smem_bytes(int max_q, int e_bits);
cudaError_t launch_resident(const DevSys* d_systems, const long long* d_nsteps, int nsys, unsigned int* d_work,
                            const ResidentPlan& plan, bool compact, int sel, cudaStream_t st);
int resident_max_smem();
// One forced step of nb configurations of one system (computation-tree
// exploration); see k_branch_step.
// Range check of the nb configurations a branch step is given (C >= 0,
// 0 <= D <= 65535, P = -1 or a rule of its neuron, D > 0 only with P):
// atomicMin of the offending index b*q + neuron into *first_bad.
cudaError_t launch_branch_check(const DevSys& s, const int32_t* rule_base, int nb, const int32_t* C0,
                                const int32_t* D0, const int32_t* P0, unsigned long long* first_bad,
                                cudaStream_t st);
size_t branch_smem_bytes(int q, int e_bits);
cudaError_t launch_branch_step(const DevSys& s, const int32_t* rule_base, int e_bits, bool compact, int nb,
                               const int32_t* C0, const int32_t* D0, const int32_t* P0, const int32_t* ch,
                               int32_t* C1, int32_t* D1, int32_t* P1, int32_t* ex, int32_t* bad, int32_t* counts,
                               cudaStream_t st);

// Tiled engine (kernels_tiled.cu): device view of a TiledPack.
struct TiledSys {
    int32_t P, part_words, e_bits, G, acc_words, src_bits, pairs, rle;
    int32_t rin_words;      // > 0: the partners' in-flows arrive in a shared buffer (see k_tiled_step)
    int32_t acc8;           // 1: byte accumulators
    int32_t rin_esm;        // 1: the partner buffer is the emissions' region (written after the gathers)
    const int32_t* tstart;  // run-length layout: first target of each thread's run, [G][kTiledThreads]
    const int32_t* sub;     // [G][kTiledMaxSub+1] window starts (words, multiples of 4); CTA g*P+h
    const uint32_t* ent;    // (dst_local << src_bits) | src_local
    int64_t ent_words;      // words of ent
    const int32_t* cta_lo;  // [G/P+1] slice ranges
    uint32_t* Eg[2];        // packed emissions of step k in Eg[k & 1]
    int32_t* inflow;        // [P][nslices*32] in-flow of the step being finished, per partition
};
cudaError_t launch_tiled(const DevSys& s, const TiledSys& tl, int kind, int32_t t, cudaStream_t st, bool compact,
                         int sel, size_t smem, int threads);
// Clusters of P CTAs of the fused step the device runs at once (0 if unknown).
int tiled_clusters_per_wave(int P, size_t smem);
// One CTA waits at most `polls` polls on a barrier nothing completes; *out = 1
// if the wait completed, 2 if it gave up.
cudaError_t launch_wait_check(int polls, uint32_t* out, cudaStream_t st);
cudaError_t launch_gather_results(const DevSys* d_systems, int nsys, unsigned long long* d_out, cudaStream_t st);

// ELL and dense forms (kernels_ell.cu).
struct EllSys {
    int64_t m;
    const int32_t* in_ptr;   // in-ELL slice starts (units of 32 pairs)
    const int2* in_ent;      // (rule, p) pairs, pad (m, 0)
    const int32_t* out_ptr;  // out-ELL rule-slice starts (units of 32 pairs)
    const int2* out_ent;     // (target, p) pairs, pad (-1, 0)
    uint8_t* Em[2];          // [m+1] rule r emits at step k: Em[k & 1][r]
    const int32_t* dense;    // m x q positive part of M_Pi (dense form)
    int32_t* inflow;         // [q] in-flow of the step being finished (dense form)
};
cudaError_t launch_ell_pull(const DevSys& s, const EllSys& e, int kind, int32_t t, cudaStream_t st, bool compact,
                            int sel);
cudaError_t launch_ell_select(const DevSys& s, const EllSys& e, bool inflow, bool select, int32_t t, cudaStream_t st,
                              bool compact, int sel);
cudaError_t launch_ell_push(const DevSys& s, const EllSys& e, int32_t t, cudaStream_t st);
cudaError_t launch_dense_accum(const DevSys& s, const EllSys& e, int32_t t, cudaStream_t st);

}  // namespace snp
