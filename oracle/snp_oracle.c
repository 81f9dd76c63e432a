/*
 * CPU oracle for one transition step of a spiking neural P system with delays.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the simulator links, imports or calls
 * this file; only the tests, the package's smoke check and the bench's CPU
 * baseline leg do.  It shares no code, header, table or constant with the CUDA
 * path: the two agree only through the definition below.
 *
 * Plain, slow and neuron by neuron.  Spike counts are kept in int64 while a
 * step is computed and checked against the int32 range before they are stored.
 *
 * Definition followed (Sec. 2, the syntax of Pi, the matrix representation
 * and Algorithm 1; Sec. 5, SV_CALC, STEP and UPDATE_DELAYS):
 *
 *   state per neuron i: C[i] spikes, D[i] steps until it reopens, P[i] the
 *   pending (delayed) rule or -1.  A neuron is closed while it has a pending
 *   rule and D[i] > 0; closed neurons neither send nor receive (Sec. 5,
 *   "Sparse": a neuron closed by a delay cannot receive or send spikes).
 *
 *   halt   : at the start of step k, if no neuron is pending and no idle
 *            neuron has an applicable rule, the system is at a fixed point
 *            (Alg. 1 stop test: empty spiking-vector set and D = 0).
 *   phase 1: every neuron, independently, from C_k:
 *            - pending with D = 0: the delayed rule completes, the neuron
 *              emits its p spikes, reopens and receives; no new selection;
 *            - pending with D > 0: closed; emits nothing, receives nothing;
 *            - idle: the applicable rules A_i (in index order) are those with
 *              n >= k_r and (j_r = 0 ? n = k_r : (n - k_r) mod j_r = 0) and
 *              n >= c_r, for the regex a^k (a^j)* (type-4 form, Sec. 7; the
 *              three types of Sec. 2 are a^n exactly, a* and a+).  A rule
 *              given as a finite union of such terms, a^k1 (a^j1)* U ...
 *              U a^kT (a^jT)*, applies when n >= c_r and n lies in any one
 *              of the terms' languages (the same test, term by term).  If A_i is
 *              empty nothing happens; else one rule r is chosen and c_r
 *              spikes are consumed.  With d_r = 0 the neuron emits p_r now;
 *              with d_r > 0 it closes (P = r, D = d_r) and emits at k + d_r.
 *   phase 2: every open (receiving) neuron j gains the sum of the emissions
 *            of its in-neighbours (C_{k+1} = C_k + S_k . M_Pi, restricted to
 *            open neurons).  Spikes sent to closed neurons are lost.
 *   phase 3: every pending neuron's counter drops by one (UPDATE_DELAYS).
 *
 *   choice : FIRST  -- the lowest-index applicable rule (Sec. 5, SV_CALC);
 *            PHILOX -- A_i[floor(x * |A_i| / 2^32)], x word i mod 4 of the
 *                      Philox4x32-10 block (Salmon et al., SC'11) at counter
 *                      (k mod 2^32, i / 4, k >> 32, 0) and key
 *                      (seed mod 2^32, seed >> 32) (orc_philox_pick);
 *            FORCED -- A_i[forced[i]] (used to enumerate branches).
 *
 * Pins (tests/test_oracle.py): Tables 1-3 and the sorting system of Sec. 6,
 * C_{k+1} = C_k + S_k . M_Pi on delay-free systems, spike bookkeeping with
 * delays, hand-written delay traces, brute-force enumeration of SV_k on tiny
 * systems, NVIDIA's host-side Philox generator.  Parity unpinned: the
 * delay-timing reading itself (a delayed rule consumes at t, keeps its
 * neuron closed for t .. t+d-1 and emits at t+d, against Alg. 4/5 read
 * literally, which consume and emit at t and close afterwards); no
 * implementation of the paper is available to confirm it, and the hand
 * traces pin this oracle to the reading, not to the paper's code.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_ERR_INVALID 1
#define ORC_ERR_OOM 2
#define ORC_ERR_OVERFLOW 5

#define ORC_FIRST 0
#define ORC_PHILOX 1
#define ORC_FORCED 2

/* ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Sec. 3.3) --------
 * A Feistel-like network of 10 rounds.  Each round multiplies two of the four
 * words by fixed odd 32-bit multipliers, keeps both halves of each 64-bit
 * product, and mixes the high halves with the other two words and the round
 * key.  The key is bumped between rounds by two Weyl constants (the golden
 * ratio and sqrt(3) - 1 as 32-bit fractions). */
static const uint32_t ORC_PHILOX_MUL_A = 0xD2511F53u;
static const uint32_t ORC_PHILOX_MUL_B = 0xCD9E8D57u;
static const uint32_t ORC_PHILOX_WEYL_A = 0x9E3779B9u;
static const uint32_t ORC_PHILOX_WEYL_B = 0xBB67AE85u;

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += ORC_PHILOX_WEYL_A;
            k1 += ORC_PHILOX_WEYL_B;
        }
        uint64_t pa = (uint64_t)ORC_PHILOX_MUL_A * x0;
        uint64_t pb = (uint64_t)ORC_PHILOX_MUL_B * x2;
        uint32_t hi_a = (uint32_t)(pa >> 32), lo_a = (uint32_t)pa;
        uint32_t hi_b = (uint32_t)(pb >> 32), lo_b = (uint32_t)pb;
        uint32_t y0 = hi_b ^ x1 ^ k0;
        uint32_t y1 = lo_b;
        uint32_t y2 = hi_a ^ x3 ^ k1;
        uint32_t y3 = lo_a;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* The uniform choice of SAMPLE_ONE (Sec. 5: one of the a applicable rules,
 * each equally likely).  The paper does not fix the generator; this library's
 * reading: the four 32-bit words of the Philox4x32-10 block at counter
 * (step mod 2^32, i / 4, step >> 32, 0) and key (seed mod 2^32, seed >> 32)
 * belong to the four neurons 4(i / 4) .. 4(i / 4) + 3, neuron i taking word
 * i mod 4, and the pick is floor(word * a / 2^32) (an index 0 .. a-1). */
static int64_t orc_philox_pick(uint64_t step, int64_t i, uint64_t seed, int64_t a) {
    uint32_t ctr[4] = {(uint32_t)step, (uint32_t)(i / 4), (uint32_t)(step >> 32), 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t x[4];
    orc_philox4x32_10(ctr, key, x);
    return (int64_t)(((uint64_t)x[i % 4] * (uint64_t)a) >> 32);
}

/* The system as the user describes it (Sec. 5, "Initialization"). */
typedef struct {
    int32_t q;
    const int64_t* rule_off;   /* [q+1] N_Pi */
    const int32_t* rk;         /* [m] regex a^k (a^j)* */
    const int32_t* rj;
    const int32_t* rc;         /* [m] consumed */
    const int32_t* rp;         /* [m] produced, 0 = forgetting */
    const int32_t* rd;         /* [m] delay */
    const int64_t* syn_off;    /* [q+1] out-lists */
    const int32_t* syn_tgt;    /* [|syn|] */
    const int64_t* term_off;   /* [m+1] or NULL: rule r's regex is the union of */
    const int32_t* tk;         /*   a^tk[t] (a^tj[t])* over t in [term_off[r],  */
    const int32_t* tj;         /*   term_off[r+1]); rk and rj are then unused   */
} orc_sys;

static int orc_applicable(int64_t n, int32_t k, int32_t j, int32_t c) {
    if (n < k) return 0;
    if (j == 0) {
        if (n != k) return 0;
    } else if ((n - k) % j != 0) {
        return 0;
    }
    return n >= c;
}

/* Rule r against n spikes: its single term, or any term of its union. */
static int orc_rule_applies(const orc_sys* s, int64_t r, int64_t n) {
    if (!s->term_off) return orc_applicable(n, s->rk[r], s->rj[r], s->rc[r]);
    for (int64_t t = s->term_off[r]; t < s->term_off[r + 1]; ++t)
        if (orc_applicable(n, s->tk[t], s->tj[t], s->rc[r])) return 1;
    return 0;
}

/* Number of applicable rules of idle neuron i with n spikes. */
static int64_t orc_count_applicable(const orc_sys* s, int32_t i, int64_t n) {
    int64_t cnt = 0;
    for (int64_t r = s->rule_off[i]; r < s->rule_off[i + 1]; ++r)
        cnt += orc_rule_applies(s, r, n);
    return cnt;
}

/* The idx-th applicable rule (0-based) of idle neuron i. */
static int64_t orc_nth_applicable(const orc_sys* s, int32_t i, int64_t n, int64_t idx) {
    for (int64_t r = s->rule_off[i]; r < s->rule_off[i + 1]; ++r) {
        if (orc_rule_applies(s, r, n)) {
            if (idx == 0) return r;
            --idx;
        }
    }
    return -1;
}

int orc_is_halted(const orc_sys* s, const int32_t* C, const int32_t* P) {
    for (int32_t i = 0; i < s->q; ++i) {
        if (P[i] != -1) return 0;
        if (orc_count_applicable(s, i, C[i]) > 0) return 0;
    }
    return 1;
}

/*
 * One transition step k.  C, D, P are updated in place.  S[i] receives the
 * global id of the rule neuron i selected at this step, or -1.  E (optional)
 * receives what each neuron emitted at this step.  *halted is set when the
 * step is not executed because the system is at a fixed point; then nothing
 * changes and S is all -1.
 */
int orc_step(const orc_sys* s, int32_t* C, int32_t* D, int32_t* P, uint64_t step,
             int mode, uint64_t seed, const int32_t* forced, int32_t* S, int32_t* E_out,
             int* halted) {
    const int32_t q = s->q;
    *halted = 0;
    for (int32_t i = 0; i < q; ++i) S[i] = -1;
    if (orc_is_halted(s, C, P)) {
        *halted = 1;
        if (E_out) memset(E_out, 0, sizeof(int32_t) * (size_t)q);
        return ORC_OK;
    }
    int64_t* Cn = (int64_t*)malloc(sizeof(int64_t) * (size_t)q);
    int64_t* E = (int64_t*)malloc(sizeof(int64_t) * (size_t)q);
    char* recv = (char*)malloc((size_t)q);
    if (!Cn || !E || !recv) {
        free(Cn); free(E); free(recv);
        return ORC_ERR_OOM;
    }
    /* phase 1 */
    for (int32_t i = 0; i < q; ++i) {
        int64_t n = C[i];
        Cn[i] = n;
        E[i] = 0;
        recv[i] = 1;
        if (P[i] != -1 && D[i] == 0) {
            E[i] = s->rp[P[i]];
            P[i] = -1;
        } else if (P[i] != -1) {
            recv[i] = 0;
        } else {
            int64_t a = orc_count_applicable(s, i, n);
            if (a == 0) continue;
            int64_t pick = 0;
            if (mode == ORC_PHILOX) {
                pick = orc_philox_pick(step, i, seed, a);
            } else if (mode == ORC_FORCED) {
                pick = forced[i];
                if (pick < 0 || pick >= a) {
                    free(Cn); free(E); free(recv);
                    return ORC_ERR_INVALID;
                }
            }
            int64_t r = orc_nth_applicable(s, i, n, pick);
            S[i] = (int32_t)r;
            Cn[i] = n - s->rc[r];
            if (s->rd[r] == 0) {
                E[i] = s->rp[r];
            } else {
                P[i] = (int32_t)r;
                D[i] = s->rd[r];
                recv[i] = 0;
            }
        }
    }
    /* phase 2: push every emission along the synapses to open neurons */
    for (int32_t i = 0; i < q; ++i) {
        if (E[i] == 0) continue;
        for (int64_t e = s->syn_off[i]; e < s->syn_off[i + 1]; ++e) {
            int32_t t = s->syn_tgt[e];
            if (recv[t]) Cn[t] += E[i];
        }
    }
    /* phase 3 */
    for (int32_t i = 0; i < q; ++i)
        if (P[i] != -1) D[i] -= 1;
    int rc = ORC_OK;
    for (int32_t i = 0; i < q; ++i) {
        if (Cn[i] > INT32_MAX || Cn[i] < INT32_MIN) rc = ORC_ERR_OVERFLOW;
        C[i] = (int32_t)Cn[i];
        if (E_out) E_out[i] = (int32_t)E[i];
    }
    free(Cn); free(E); free(recv);
    return rc;
}

/*
 * Up to nsteps steps starting at absolute step `step0`; stops at the first
 * fixed point.  *executed receives the number of steps actually taken and S
 * the spiking vector of the last executed step (left untouched if none).
 */
/* The definition's step split at its exchange point, for the neurons
 * lo..hi-1 only (one shard of a system partitioned by neuron range; test
 * infrastructure for the sharded step).  orc_range_select is phase 1 for
 * those neurons -- complete a delayed rule / count down / choose an
 * applicable rule and consume -- writing their emissions into E[lo..hi-1],
 * their spiking vector into S[lo..hi-1], whether each can receive this step
 * into recv[lo..hi-1], and *active = 1 when any of them is pending or chose
 * a rule.  The system is at a fixed point when no shard is active; then no
 * state changed.  Once E holds every shard's emissions, orc_range_receive is
 * phase 2 for the same neurons (every emission pushed along the synapses
 * into the open ones among lo..hi-1) and phase 3 (their delay counters).
 * Composed over shards covering 0..q-1 this is exactly orc_step.           */
int orc_range_select(const orc_sys* s, int32_t lo, int32_t hi, int32_t* C, int32_t* D, int32_t* P,
                     uint64_t step, int mode, uint64_t seed, int32_t* S, int32_t* E, char* recv,
                     int* active) {
    *active = 0;
    for (int32_t i = lo; i < hi; ++i) {
        const int64_t n = C[i];
        S[i] = -1;
        E[i] = 0;
        recv[i] = 1;
        if (P[i] != -1 && D[i] == 0) {
            *active = 1;
            E[i] = s->rp[P[i]];
            P[i] = -1;
        } else if (P[i] != -1) {
            *active = 1;
            recv[i] = 0;
        } else {
            const int64_t a = orc_count_applicable(s, i, n);
            if (a == 0) continue;
            *active = 1;
            int64_t pick = 0;
            if (mode == ORC_PHILOX) {
                pick = orc_philox_pick(step, i, seed, a);
            } else if (mode != ORC_FIRST) {
                return ORC_ERR_INVALID;
            }
            const int64_t r = orc_nth_applicable(s, i, n, pick);
            S[i] = (int32_t)r;
            C[i] = (int32_t)(n - s->rc[r]);
            if (s->rd[r] == 0) {
                E[i] = s->rp[r];
            } else {
                P[i] = (int32_t)r;
                D[i] = s->rd[r];
                recv[i] = 0;
            }
        }
    }
    return ORC_OK;
}

int orc_range_receive(const orc_sys* s, int32_t lo, int32_t hi, int32_t* C, int32_t* D, const int32_t* P,
                      const int32_t* E, const char* recv) {
    const int32_t q = s->q;
    int rc = ORC_OK;
    int64_t* add = (int64_t*)calloc((size_t)(hi > lo ? hi - lo : 1), sizeof(int64_t));
    if (!add) return ORC_ERR_OOM;
    /* phase 2: every emission pushed along its synapses into lo..hi-1 */
    for (int32_t i = 0; i < q; ++i) {
        if (E[i] == 0) continue;
        for (int64_t e = s->syn_off[i]; e < s->syn_off[i + 1]; ++e) {
            const int32_t t = s->syn_tgt[e];
            if (t >= lo && t < hi && recv[t]) add[t - lo] += E[i];
        }
    }
    for (int32_t t = lo; t < hi; ++t) {
        const int64_t c = (int64_t)C[t] + add[t - lo];
        if (c > INT32_MAX || c < INT32_MIN) rc = ORC_ERR_OVERFLOW;
        C[t] = (int32_t)c;
        /* phase 3 */
        if (P[t] != -1) D[t] -= 1;
    }
    free(add);
    return rc;
}

int orc_run(const orc_sys* s, int32_t* C, int32_t* D, int32_t* P, uint64_t step0,
            int64_t nsteps, int mode, uint64_t seed, int32_t* S, int64_t* executed) {
    int32_t* Stmp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(s->q > 0 ? s->q : 1));
    if (!Stmp) return ORC_ERR_OOM;
    *executed = 0;
    for (int64_t t = 0; t < nsteps; ++t) {
        int halted = 0;
        int rc = orc_step(s, C, D, P, step0 + (uint64_t)t, mode, seed, NULL, Stmp, NULL, &halted);
        if (rc != ORC_OK) { free(Stmp); return rc; }
        if (halted) break;
        memcpy(S, Stmp, sizeof(int32_t) * (size_t)s->q);
        *executed += 1;
    }
    free(Stmp);
    return ORC_OK;
}

/* ---- the same definition, pulled and in parallel ------------------------
 * orc_run_pull applies exactly the three phases above, with phase 2 written
 * as a pull over in-neighbour lists (C_{k+1}[j] gains the sum of E[i] over
 * the synapses (i, j) when j receives) instead of a push along out-lists.
 * Every phase is a loop over independent neurons; with OpenMP each loop is
 * split across threads (without it the pragmas are ignored and the loops run
 * in order).  Integer sums do not depend on order, so the result is the one
 * orc_run gives.  in_off [q+1] / in_src [|syn|]: in-lists (orc_in_lists). */
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* In-neighbour lists of every neuron, sources in increasing order. */
int orc_in_lists(const orc_sys* s, int64_t* in_off, int32_t* in_src) {
    const int32_t q = s->q;
    for (int32_t j = 0; j <= q; ++j) in_off[j] = 0;
    for (int32_t i = 0; i < q; ++i)
        for (int64_t e = s->syn_off[i]; e < s->syn_off[i + 1]; ++e) in_off[s->syn_tgt[e] + 1] += 1;
    for (int32_t j = 0; j < q; ++j) in_off[j + 1] += in_off[j];
    int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(q > 0 ? q : 1));
    if (!fill) return ORC_ERR_OOM;
    for (int32_t j = 0; j < q; ++j) fill[j] = in_off[j];
    for (int32_t i = 0; i < q; ++i)
        for (int64_t e = s->syn_off[i]; e < s->syn_off[i + 1]; ++e) in_src[fill[s->syn_tgt[e]]++] = i;
    free(fill);
    return ORC_OK;
}

int orc_run_pull(const orc_sys* s, const int64_t* in_off, const int32_t* in_src, int32_t* C, int32_t* D,
                 int32_t* P, uint64_t step0, int64_t nsteps, int mode, uint64_t seed, int32_t* S,
                 int64_t* executed) {
    const int32_t q = s->q;
    const size_t nq = (size_t)(q > 0 ? q : 1);
    int64_t* Cn = (int64_t*)malloc(sizeof(int64_t) * nq);
    int64_t* E = (int64_t*)malloc(sizeof(int64_t) * nq);
    char* recv = (char*)malloc(nq);
    int32_t* Sk = (int32_t*)malloc(sizeof(int32_t) * nq);
    if (!Cn || !E || !recv || !Sk) {
        free(Cn); free(E); free(recv); free(Sk);
        return ORC_ERR_OOM;
    }
    *executed = 0;
    int rc = ORC_OK;
    for (int64_t t = 0; t < nsteps && rc == ORC_OK; ++t) {
        const uint64_t step = step0 + (uint64_t)t;
        /* halt test */
        int busy = 0;
#pragma omp parallel for reduction(| : busy) schedule(static)
        for (int32_t i = 0; i < q; ++i)
            busy |= P[i] != -1 || orc_count_applicable(s, i, C[i]) > 0;
        if (!busy) break;
        /* phase 1 */
#pragma omp parallel for schedule(static)
        for (int32_t i = 0; i < q; ++i) {
            const int64_t n = C[i];
            Cn[i] = n;
            E[i] = 0;
            recv[i] = 1;
            Sk[i] = -1;
            if (P[i] != -1 && D[i] == 0) {
                E[i] = s->rp[P[i]];
                P[i] = -1;
            } else if (P[i] != -1) {
                recv[i] = 0;
            } else {
                const int64_t a = orc_count_applicable(s, i, n);
                if (a == 0) continue;
                int64_t pick = 0;
                if (mode == ORC_PHILOX) {
                    pick = orc_philox_pick(step, i, seed, a);
                }
                const int64_t r = orc_nth_applicable(s, i, n, pick);
                Sk[i] = (int32_t)r;
                Cn[i] = n - s->rc[r];
                if (s->rd[r] == 0) {
                    E[i] = s->rp[r];
                } else {
                    P[i] = (int32_t)r;
                    D[i] = s->rd[r];
                    recv[i] = 0;
                }
            }
        }
        /* phase 2 (pull) and phase 3 */
        int over = 0;
#pragma omp parallel for reduction(| : over) schedule(static)
        for (int32_t j = 0; j < q; ++j) {
            int64_t c = Cn[j];
            if (recv[j])
                for (int64_t e = in_off[j]; e < in_off[j + 1]; ++e) c += E[in_src[e]];
            if (P[j] != -1) D[j] -= 1;
            over |= c > INT32_MAX || c < INT32_MIN;
            C[j] = (int32_t)c;
        }
        if (over) rc = ORC_ERR_OVERFLOW;
        memcpy(S, Sk, sizeof(int32_t) * (size_t)q);
        *executed += 1;
    }
    free(Cn); free(E); free(recv); free(Sk);
    return rc;
}

/* Number of rules neuron i may choose at the next step (the definition of
 * phase 1): |A_i| for an idle neuron, 0 while a rule is pending. */
void orc_count_choices(const orc_sys* s, const int32_t* C, const int32_t* P, int32_t* out) {
    for (int32_t i = 0; i < s->q; ++i)
        out[i] = P[i] != -1 ? 0 : (int32_t)orc_count_applicable(s, i, C[i]);
}
