/*
 * ffs_oracle.c -- plain, slow, single-threaded CPU oracle for the flexible
 * flow shop (FFS) island GA hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent statement of what
 * the GPU library must compute.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline arm may load it.  It shares no code, header, table
 * or constant generator with the CUDA library; every function below is
 * written from its definition, in the order the method states it, with no
 * blocking, fusion or reordering.
 *
 * Sources (Luo & El Baz, "A Dual Heterogeneous Island Genetic Algorithm for
 * Solving Large Size Flexible Flow Shop Scheduling Problems on Hybrid
 * multi-core CPU and GPU Platforms", arXiv:1903.10722):
 *   - Section 3: the FFS problem (jobs pass all stages in order, each
 *     operation on exactly one of M_s identical machines, no preemption),
 *     release times R_j, due times D_j and the objective
 *     WT * sum_j T_j + C_max with tardiness T_j = max(0, C_j - D_j).
 *   - Section 5, Table 1: WT = 100 and the release / due time generator.
 *   - Section 4.1: the two islands (cellular GA on a 2D grid, pseudo GA with
 *     complementary parents whose children replace them).
 *   - Section 4.2: the cellular step (recombine two neighbours, mutate,
 *     replace the cell if better).
 *   - Section 4.3, Eq. (1)-(2): the penetration migration policy.
 *   - Section 5: parameter values (pc 1.00 / pm 0.05 cellular, pc 0.75
 *     pseudo, theta 1.00).
 * The schedule decoder (stage-wise list scheduling) and the operators (order
 * crossover, swap mutation, binary tournament on a von Neumann torus) are not
 * spelled out in the paper; the readings used here are listed in the header
 * comment of each function and in the design notes of the repository.
 *
 * Philox4x32-10 follows Salmon, Moraes, Dror and Shaw, "Parallel Random
 * Numbers: As Easy as 1, 2, 3", SC 2011 (Section 4, the Philox S-box).
 *
 * Parity status: the decoder (makespan and the Section 3 objective), the
 * decoder of the paper's own genotype (machine-assignment strings), the
 * operators, Philox and the migration formulas are pinned by tests
 * (hand-worked Gantt charts, closed forms, brute force, library
 * cross-checks).  The GA loop as a whole (the sequence
 * of generations) has no published trajectory: "parity unpinned" beyond
 * those component pins.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al. 2011)                                  */
/* ------------------------------------------------------------------ */

/* One call = ten rounds.  Each round multiplies the even words of the
 * counter by the two Philox multipliers, and builds the new counter from the
 * high halves xor'ed with the odd words and the round key; the key is bumped
 * by the two Weyl constants between rounds. */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                       uint32_t out[4])
{
    const uint32_t mult0 = 0xD2511F53u, mult1 = 0xCD9E8D57u;
    const uint32_t weyl0 = 0x9E3779B9u, weyl1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += weyl0;
            k1 += weyl1;
        }
        uint64_t prod0 = (uint64_t)mult0 * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)mult1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Purpose codes of the counter's fourth word (top 8 bits). */
enum { ORC_PURPOSE_INIT = 1, ORC_PURPOSE_CELLULAR = 2, ORC_PURPOSE_PSEUDO = 3,
       ORC_PURPOSE_SURROGATE = 16 /* + candidate index */,
       ORC_PURPOSE_SURROGATE_PSEUDO = 32 /* + candidate index */ };

/* Draw number d of the stream keyed by (seed, island, generation, cell):
 * counter = (d / 4, cell, generation, island | purpose << 24),
 * key = (low, high) 32-bit halves of the seed, result word = d mod 4. */
uint32_t orc_draw(uint64_t seed, uint32_t purpose, uint32_t island,
                  uint32_t generation, uint32_t cell, uint32_t d)
{
    uint32_t ctr[4] = { d / 4u, cell, generation, (island & 0xFFFFFFu) | (purpose << 24) };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t out[4];
    orc_philox4x32_10(ctr, key, out);
    return out[d % 4u];
}

/* Integer in [0, k): the high word of x * k (no rejection step). */
uint32_t orc_uniform(uint32_t x, uint32_t k)
{
    return (uint32_t)(((uint64_t)x * (uint64_t)k) >> 32);
}

/* Bernoulli event with probability threshold / 2^32 (threshold in [0, 2^32]). */
int orc_bernoulli(uint32_t x, uint64_t threshold)
{
    return (uint64_t)x < threshold;
}

/* ------------------------------------------------------------------ */
/* Schedule decoder: stage-wise list scheduling                        */
/* ------------------------------------------------------------------ */

/* Stage 1 takes the jobs in chromosome order.  Every later stage takes them
 * in ascending (completion time at the previous stage, job index) order.
 * Each job goes to the machine that is free earliest, the lowest machine
 * index on ties, and starts at max(machine free time, release from the
 * previous stage).  Stage-1 release time is R_j (0 without release times).
 *
 * Objective (Section 3): C_max, plus WT * sum_j max(0, C_j - D_j) when due
 * times are given, C_j being job j's completion at the last stage.
 *
 * p is [n][S] row-major (job-major).  If gantt is not NULL it receives
 * n*S records of 5 int64 (stage, job, machine, start, end) in dispatch
 * order, stage by stage.  A row with a gene outside [0, n) has objective
 * -1 (nothing is scheduled). */
typedef struct {
    const int32_t *release;   /* R_j [n], or NULL (all 0) */
    const int32_t *due;       /* D_j [n], or NULL (no tardiness term) */
    int64_t wt;               /* WT, the weight of the total tardiness */
} orc_objective;

typedef struct { int64_t c; int32_t j; } orc_pair;

static int orc_pair_cmp(const void *a, const void *b)
{
    const orc_pair *x = (const orc_pair *)a, *y = (const orc_pair *)b;
    if (x->c < y->c) return -1;
    if (x->c > y->c) return 1;
    if (x->j < y->j) return -1;
    if (x->j > y->j) return 1;
    return 0;
}

int64_t orc_decode_obj(int32_t n, int32_t S, const int32_t *M, const int32_t *p,
                       const orc_objective *obj, const int16_t *perm, int64_t *gantt)
{
    /* a gene that names no job makes the row invalid: objective -1 (the
     * same reading as for the machine-assignment strings below) */
    for (int32_t k = 0; k < n; ++k)
        if (perm[k] < 0 || perm[k] >= n) return -1;
    int64_t *c_prev = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    int64_t *c_cur = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    int32_t *order = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    orc_pair *pairs = (orc_pair *)malloc((size_t)n * sizeof(orc_pair));
    const int32_t *release = obj ? obj->release : NULL;
    int64_t rec = 0;
    for (int32_t s = 0; s < S; ++s) {
        if (s == 0) {
            for (int32_t k = 0; k < n; ++k) order[k] = perm[k];
        } else {
            for (int32_t j = 0; j < n; ++j) { pairs[j].c = c_prev[j]; pairs[j].j = j; }
            qsort(pairs, (size_t)n, sizeof(orc_pair), orc_pair_cmp);
            for (int32_t k = 0; k < n; ++k) order[k] = pairs[k].j;
        }
        int32_t ms = M[s];
        int64_t *free_at = (int64_t *)calloc((size_t)ms, sizeof(int64_t));
        for (int32_t k = 0; k < n; ++k) {
            int32_t j = order[k];
            int32_t best = 0;
            for (int32_t m = 1; m < ms; ++m)
                if (free_at[m] < free_at[best]) best = m;
            int64_t ready = (s == 0) ? (release ? (int64_t)release[j] : 0) : c_prev[j];
            int64_t start = free_at[best] > ready ? free_at[best] : ready;
            int64_t end = start + (int64_t)p[(int64_t)j * S + s];
            c_cur[j] = end;
            free_at[best] = end;
            if (gantt) {
                gantt[rec * 5 + 0] = s;
                gantt[rec * 5 + 1] = j;
                gantt[rec * 5 + 2] = best;
                gantt[rec * 5 + 3] = start;
                gantt[rec * 5 + 4] = end;
                ++rec;
            }
        }
        free(free_at);
        int64_t *t = c_prev; c_prev = c_cur; c_cur = t;
    }
    int64_t cmax = 0;
    for (int32_t j = 0; j < n; ++j) if (c_prev[j] > cmax) cmax = c_prev[j];
    int64_t total_tardiness = 0;
    if (obj && obj->due)
        for (int32_t j = 0; j < n; ++j)
            if (c_prev[j] > obj->due[j]) total_tardiness += c_prev[j] - obj->due[j];
    free(c_prev); free(c_cur); free(order); free(pairs);
    return (obj && obj->due ? obj->wt * total_tardiness : 0) + cmax;
}

/* The makespan alone (no release or due times). */
int64_t orc_decode(int32_t n, int32_t S, const int32_t *M, const int32_t *p,
                   const int16_t *perm, int64_t *gantt)
{
    return orc_decode_obj(n, S, M, p, NULL, perm, gantt);
}

/* The paper's genotype (Section 4.1, genotype level; Section 3, P_jsm): a
 * string of n*S genes, gene i = the index (0-based) of the target machine of
 * job floor(i/S) at stage i mod S, on unrelated machines: p_u is [n][W],
 * W = M_0 + ... + M_{S-1}, the time of job j at stage s on machine m at
 * p_u[j*W + off_s + m], off_s = M_0 + ... + M_{s-1}.
 *
 * Sequencing (the paper leaves it unstated): every machine processes the
 * jobs assigned to it in order of arrival -- stage 1: release time R_j (0
 * without release times), later stages: completion at the previous stage
 * -- ties by job index; a job starts at max(machine free time, arrival).
 * This is the definition above with the machine fixed by the gene instead
 * of chosen as the earliest free one, and stage 1 in (R_j, j) order.
 *
 * Objective as orc_decode_obj.  Returns -1 if a gene is outside [0, M_s).
 * gantt as orc_decode_obj. */
int64_t orc_decode_assign(int32_t n, int32_t S, const int32_t *M, const int32_t *p_u,
                          const orc_objective *obj, const int16_t *genes, int64_t *gantt)
{
    for (int32_t j = 0; j < n; ++j)
        for (int32_t s = 0; s < S; ++s)
            if (genes[(int64_t)j * S + s] < 0 || genes[(int64_t)j * S + s] >= M[s]) return -1;
    int64_t W = 0;
    for (int32_t s = 0; s < S; ++s) W += M[s];
    int64_t *arrive = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    int64_t *done = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    orc_pair *pairs = (orc_pair *)malloc((size_t)n * sizeof(orc_pair));
    const int32_t *release = obj ? obj->release : NULL;
    for (int32_t j = 0; j < n; ++j) arrive[j] = release ? (int64_t)release[j] : 0;
    int64_t rec = 0, off = 0;
    for (int32_t s = 0; s < S; ++s) {
        for (int32_t j = 0; j < n; ++j) { pairs[j].c = arrive[j]; pairs[j].j = j; }
        qsort(pairs, (size_t)n, sizeof(orc_pair), orc_pair_cmp);
        int64_t *free_at = (int64_t *)calloc((size_t)M[s], sizeof(int64_t));
        for (int32_t k = 0; k < n; ++k) {
            const int32_t j = pairs[k].j;
            const int32_t m = genes[(int64_t)j * S + s];
            const int64_t start = free_at[m] > arrive[j] ? free_at[m] : arrive[j];
            const int64_t end = start + (int64_t)p_u[(int64_t)j * W + off + m];
            done[j] = end;
            free_at[m] = end;
            if (gantt) {
                gantt[rec * 5 + 0] = s;
                gantt[rec * 5 + 1] = j;
                gantt[rec * 5 + 2] = m;
                gantt[rec * 5 + 3] = start;
                gantt[rec * 5 + 4] = end;
                ++rec;
            }
        }
        free(free_at);
        off += M[s];
        int64_t *t = arrive; arrive = done; done = t;
    }
    int64_t cmax = 0;
    for (int32_t j = 0; j < n; ++j) if (arrive[j] > cmax) cmax = arrive[j];
    int64_t total_tardiness = 0;
    if (obj && obj->due)
        for (int32_t j = 0; j < n; ++j)
            if (arrive[j] > obj->due[j]) total_tardiness += arrive[j] - obj->due[j];
    free(arrive); free(done); free(pairs);
    return (obj && obj->due ? obj->wt * total_tardiness : 0) + cmax;
}

/* orc_decode_assign of every row of a population [N][ld] of genes. */
void orc_eval_population_assign(int32_t n, int32_t S, const int32_t *M, const int32_t *p_u,
                                const orc_objective *obj, const int16_t *pop, int64_t N, int64_t ld,
                                int64_t *out)
{
    for (int64_t i = 0; i < N; ++i)
        out[i] = orc_decode_assign(n, S, M, p_u, obj, pop + i * ld, NULL);
}

/* Objective of every row of a population [N][ld] (int16 genes); obj NULL:
 * the makespan. */
void orc_eval_population_obj(int32_t n, int32_t S, const int32_t *M, const int32_t *p,
                             const orc_objective *obj, const int16_t *pop, int64_t N, int64_t ld,
                             int64_t *out)
{
    for (int64_t i = 0; i < N; ++i)
        out[i] = orc_decode_obj(n, S, M, p, obj, pop + i * ld, NULL);
}

void orc_eval_population(int32_t n, int32_t S, const int32_t *M, const int32_t *p,
                         const int16_t *pop, int64_t N, int64_t ld, int64_t *out)
{
    orc_eval_population_obj(n, S, M, p, NULL, pop, N, ld, out);
}

/* Brute force over all n! orders (n <= 10): returns the minimum makespan and
 * writes the maximum to *worst.  Uses the lexicographic next-permutation walk. */
int64_t orc_bruteforce_obj(int32_t n, int32_t S, const int32_t *M, const int32_t *p,
                           const orc_objective *obj, int64_t *worst, int16_t *best_perm)
{
    int16_t perm[16];
    for (int32_t i = 0; i < n; ++i) perm[i] = (int16_t)i;
    int64_t best = -1, wst = -1;
    for (;;) {
        int64_t c = orc_decode_obj(n, S, M, p, obj, perm, NULL);
        if (best < 0 || c < best) {
            best = c;
            if (best_perm) memcpy(best_perm, perm, (size_t)n * sizeof(int16_t));
        }
        if (c > wst) wst = c;
        int32_t i = n - 2;
        while (i >= 0 && perm[i] >= perm[i + 1]) --i;
        if (i < 0) break;
        int32_t k = n - 1;
        while (perm[k] <= perm[i]) --k;
        int16_t t = perm[i]; perm[i] = perm[k]; perm[k] = t;
        for (int32_t a = i + 1, b = n - 1; a < b; ++a, --b) {
            t = perm[a]; perm[a] = perm[b]; perm[b] = t;
        }
    }
    if (worst) *worst = wst;
    return best;
}

int64_t orc_bruteforce(int32_t n, int32_t S, const int32_t *M, const int32_t *p,
                       int64_t *worst, int16_t *best_perm)
{
    return orc_bruteforce_obj(n, S, M, p, NULL, worst, best_perm);
}

/* ------------------------------------------------------------------ */
/* Genetic operators                                                    */
/* ------------------------------------------------------------------ */

/* Random initial chromosome (Section 4.1, "random initialization"): the
 * Fisher-Yates shuffle of the identity, i = n-1 down to 1, swapping a[i] with
 * a[uniform(i+1)], where the swap at position i uses draw number n-1-i. */
void orc_init_chromosome(uint64_t seed, uint32_t island, uint32_t cell, int32_t n,
                         int16_t *out)
{
    for (int32_t i = 0; i < n; ++i) out[i] = (int16_t)i;
    for (int32_t i = n - 1; i >= 1; --i) {
        uint32_t x = orc_draw(seed, ORC_PURPOSE_INIT, island, 0u, cell, (uint32_t)(n - 1 - i));
        int32_t j = (int32_t)orc_uniform(x, (uint32_t)(i + 1));
        int16_t t = out[i]; out[i] = out[j]; out[j] = t;
    }
}

/* Order crossover (Davis's OX): the child keeps p1's genes at positions
 * l..r (inclusive); the remaining positions, visited from r+1 onward and
 * wrapping to 0, receive the genes of p2 in the order met when scanning p2
 * from position r+1 onward (wrapping), skipping genes already in the child. */
void orc_order_crossover(int32_t n, const int16_t *p1, const int16_t *p2,
                         int32_t l, int32_t r, int16_t *child)
{
    unsigned char *taken = (unsigned char *)calloc((size_t)n, 1);
    for (int32_t k = l; k <= r; ++k) {
        child[k] = p1[k];
        taken[p1[k]] = 1;
    }
    int32_t pos = (r + 1) % n;
    for (int32_t t = 0; t < n; ++t) {
        int16_t g = p2[(r + 1 + t) % n];
        if (taken[g]) continue;
        child[pos] = g;
        taken[g] = 1;
        pos = (pos + 1) % n;
    }
    free(taken);
}

/* The five cells of the von Neumann neighbourhood of cell c on an R x Q torus:
 * slot 0 = the cell itself, 1 = north (row - 1), 2 = south (row + 1),
 * 3 = west (column - 1), 4 = east (column + 1), rows and columns mod R, Q. */
void orc_neighbours(int32_t rows, int32_t cols, int32_t c, int32_t out[5])
{
    int32_t r = c / cols, q = c % cols;
    out[0] = c;
    out[1] = ((r - 1 + rows) % rows) * cols + q;
    out[2] = ((r + 1) % rows) * cols + q;
    out[3] = r * cols + (q - 1 + cols) % cols;
    out[4] = r * cols + (q + 1) % cols;
}

/* GA parameters as plain numbers (the oracle's own representation). */
typedef struct {
    uint64_t seed;
    uint64_t cell_pc;      /* crossover threshold, Bernoulli fires iff x < pc */
    uint64_t cell_pm;      /* mutation threshold (one swap per child) */
    uint64_t pseudo_pc;    /* pseudo crossover threshold */
    int32_t cell_replace_le;   /* 0: replace iff child < cell; 1: iff child <= cell */
    int32_t pseudo_always;     /* 0: pair keeps the 2 best of {c1,c2,a,b}; 1: children replace parents */
    const orc_objective *obj;  /* the instance's objective (NULL: makespan); every "makespan"
                                  below is then this objective */
} orc_params;

/* One child of the cellular island for cell c (Section 4.2), given its ten
 * draws x[0..9]: two binary tournaments over the five neighbourhood slots
 * (draws 0,1 and 2,3; the lower makespan wins, the first-drawn on ties),
 * crossover with probability pc (draw 4; cut points from draws 5 and 6,
 * l = min, r = max), otherwise the child is a copy of the first parent;
 * then with probability pm (draw 7) one swap of the positions given by draws
 * 8 and 9.  The parents' makespans are those of the previous generation. */
void orc_cellular_child(int32_t n, int32_t rows, int32_t cols, int32_t c,
                        const uint32_t x[10], const orc_params *prm,
                        const int16_t *pop, int64_t ld, const int64_t *ms,
                        int16_t *child, int32_t *parents_out)
{
    int32_t nb[5];
    orc_neighbours(rows, cols, c, nb);
    int32_t a1 = nb[orc_uniform(x[0], 5u)], b1 = nb[orc_uniform(x[1], 5u)];
    int32_t par1 = (ms[b1] < ms[a1]) ? b1 : a1;
    int32_t a2 = nb[orc_uniform(x[2], 5u)], b2 = nb[orc_uniform(x[3], 5u)];
    int32_t par2 = (ms[b2] < ms[a2]) ? b2 : a2;
    if (parents_out) { parents_out[0] = par1; parents_out[1] = par2; }
    if (orc_bernoulli(x[4], prm->cell_pc)) {
        int32_t u = (int32_t)orc_uniform(x[5], (uint32_t)n);
        int32_t v = (int32_t)orc_uniform(x[6], (uint32_t)n);
        int32_t l = u < v ? u : v, r = u < v ? v : u;
        orc_order_crossover(n, pop + (int64_t)par1 * ld, pop + (int64_t)par2 * ld, l, r, child);
    } else {
        memcpy(child, pop + (int64_t)par1 * ld, (size_t)n * sizeof(int16_t));
    }
    if (orc_bernoulli(x[7], prm->cell_pm)) {
        int32_t i = (int32_t)orc_uniform(x[8], (uint32_t)n);
        int32_t j = (int32_t)orc_uniform(x[9], (uint32_t)n);
        int16_t t = child[i]; child[i] = child[j]; child[j] = t;
    }
}

/* One synchronous generation of a cellular island (Section 4.1-4.2): every
 * cell reads the previous generation (pop_in, ms_in) and writes the next
 * (pop_out, ms_out); the child replaces the cell iff its makespan is lower
 * (or not higher, with cell_replace_le).  Returns the number of children
 * decoded. */
/* Cells c0 .. c1-1 of one cellular generation (the cells are independent
 * within a generation: each reads only the previous generation). */
int64_t orc_cellular_generation_range(int32_t n, int32_t S, const int32_t *M, const int32_t *p,
                                      const orc_params *prm, uint32_t island, uint32_t generation,
                                      int32_t rows, int32_t cols, int64_t ld,
                                      const int16_t *pop_in, const int64_t *ms_in,
                                      int16_t *pop_out, int64_t *ms_out, int32_t c0, int32_t c1)
{
    int16_t *child = (int16_t *)malloc((size_t)n * sizeof(int16_t));
    for (int32_t c = c0; c < c1; ++c) {
        uint32_t x[10];
        for (uint32_t d = 0; d < 10u; ++d)
            x[d] = orc_draw(prm->seed, ORC_PURPOSE_CELLULAR, island, generation, (uint32_t)c, d);
        orc_cellular_child(n, rows, cols, c, x, prm, pop_in, ld, ms_in, child, NULL);
        int64_t mc = orc_decode_obj(n, S, M, p, prm->obj, child, NULL);
        int better = prm->cell_replace_le ? (mc <= ms_in[c]) : (mc < ms_in[c]);
        int16_t *dst = pop_out + (int64_t)c * ld;
        if (better) {
            memcpy(dst, child, (size_t)n * sizeof(int16_t));
            ms_out[c] = mc;
        } else {
            memcpy(dst, pop_in + (int64_t)c * ld, (size_t)n * sizeof(int16_t));
            ms_out[c] = ms_in[c];
        }
    }
    free(child);
    return c1 - c0;
}

int64_t orc_cellular_generation(int32_t n, int32_t S, const int32_t *M, const int32_t *p,
                                const orc_params *prm, uint32_t island, uint32_t generation,
                                int32_t rows, int32_t cols, int64_t ld,
                                const int16_t *pop_in, const int64_t *ms_in,
                                int16_t *pop_out, int64_t *ms_out)
{
    return orc_cellular_generation_range(n, S, M, p, prm, island, generation, rows, cols, ld, pop_in, ms_in,
                                         pop_out, ms_out, 0, rows * cols);
}

/* Complementary parents of the pseudo island (Section 4.1): a pair is a
 * random chromosome a and its complement, read for a job-order chromosome as
 * the reversed order b[i] = a[n-1-i].  Pair k occupies slots 2k and 2k+1 and
 * a is drawn with cell index 2k. */
void orc_init_pseudo_pair(uint64_t seed, uint32_t island, int32_t k, int32_t n,
                          int16_t *a, int16_t *b)
{
    orc_init_chromosome(seed, island, (uint32_t)(2 * k), n, a);
    for (int32_t i = 0; i < n; ++i) b[i] = a[n - 1 - i];
}

/* The two best members of a pseudo family given in role order
 * (c1, c2, a, b): ranked by (makespan, role), lowest first. */
void orc_family_best2(const int64_t fms[4], int32_t out[2])
{
    int32_t first = 0;
    for (int32_t t = 1; t < 4; ++t) if (fms[t] < fms[first]) first = t;
    int32_t second = -1;
    for (int32_t t = 0; t < 4; ++t) {
        if (t == first) continue;
        if (second < 0 || fms[t] < fms[second]) second = t;
    }
    out[0] = first;
    out[1] = second;
}

/* One generation of a pseudo island (Section 4.1-4.2): pair k (slots 2k,
 * 2k+1) crosses with probability pc (draw 0; cuts from draws 1 and 2):
 * c1 = OX(a, b), c2 = OX(b, a) on the same cuts.  With pseudo_always the
 * children replace the parents; otherwise the pair keeps the two best of
 * (c1, c2, a, b) ranked by (makespan, that role order), best in slot 2k.
 * Without crossover the pair is copied unchanged.  Returns the number of
 * children decoded. */
/* Pairs k0 .. k1-1 of one pseudo generation (pairs are independent). */
int64_t orc_pseudo_generation_range(int32_t n, int32_t S, const int32_t *M, const int32_t *p,
                                    const orc_params *prm, uint32_t island, uint32_t generation,
                                    int32_t size, int64_t ld,
                                    const int16_t *pop_in, const int64_t *ms_in,
                                    int16_t *pop_out, int64_t *ms_out, int32_t k0, int32_t k1)
{
    (void)size;
    int16_t *c1 = (int16_t *)malloc((size_t)n * sizeof(int16_t));
    int16_t *c2 = (int16_t *)malloc((size_t)n * sizeof(int16_t));
    int64_t decoded = 0;
    for (int32_t k = k0; k < k1; ++k) {
        const int16_t *a = pop_in + (int64_t)(2 * k) * ld;
        const int16_t *b = pop_in + (int64_t)(2 * k + 1) * ld;
        int16_t *oa = pop_out + (int64_t)(2 * k) * ld;
        int16_t *ob = pop_out + (int64_t)(2 * k + 1) * ld;
        uint32_t x0 = orc_draw(prm->seed, ORC_PURPOSE_PSEUDO, island, generation, (uint32_t)k, 0u);
        if (!orc_bernoulli(x0, prm->pseudo_pc)) {
            memcpy(oa, a, (size_t)n * sizeof(int16_t));
            memcpy(ob, b, (size_t)n * sizeof(int16_t));
            ms_out[2 * k] = ms_in[2 * k];
            ms_out[2 * k + 1] = ms_in[2 * k + 1];
            continue;
        }
        uint32_t x1 = orc_draw(prm->seed, ORC_PURPOSE_PSEUDO, island, generation, (uint32_t)k, 1u);
        uint32_t x2 = orc_draw(prm->seed, ORC_PURPOSE_PSEUDO, island, generation, (uint32_t)k, 2u);
        int32_t u = (int32_t)orc_uniform(x1, (uint32_t)n);
        int32_t v = (int32_t)orc_uniform(x2, (uint32_t)n);
        int32_t l = u < v ? u : v, r = u < v ? v : u;
        orc_order_crossover(n, a, b, l, r, c1);
        orc_order_crossover(n, b, a, l, r, c2);
        int64_t m1 = orc_decode_obj(n, S, M, p, prm->obj, c1, NULL);
        int64_t m2 = orc_decode_obj(n, S, M, p, prm->obj, c2, NULL);
        decoded += 2;
        if (prm->pseudo_always) {
            memcpy(oa, c1, (size_t)n * sizeof(int16_t));
            memcpy(ob, c2, (size_t)n * sizeof(int16_t));
            ms_out[2 * k] = m1;
            ms_out[2 * k + 1] = m2;
            continue;
        }
        /* the family in role order c1, c2, a, b */
        const int16_t *fam[4] = { c1, c2, a, b };
        int64_t fms[4] = { m1, m2, ms_in[2 * k], ms_in[2 * k + 1] };
        int32_t pick[2];
        orc_family_best2(fms, pick);
        int32_t first = pick[0], second = pick[1];
        /* pop_in and pop_out are distinct buffers (synchronous generations) */
        memcpy(oa, fam[first], (size_t)n * sizeof(int16_t));
        memcpy(ob, fam[second], (size_t)n * sizeof(int16_t));
        ms_out[2 * k] = fms[first];
        ms_out[2 * k + 1] = fms[second];
    }
    free(c1); free(c2);
    return decoded;
}

int64_t orc_pseudo_generation(int32_t n, int32_t S, const int32_t *M, const int32_t *p,
                              const orc_params *prm, uint32_t island, uint32_t generation,
                              int32_t size, int64_t ld,
                              const int16_t *pop_in, const int64_t *ms_in,
                              int16_t *pop_out, int64_t *ms_out)
{
    return orc_pseudo_generation_range(n, S, M, p, prm, island, generation, size, ld, pop_in, ms_in, pop_out,
                                       ms_out, 0, size / 2);
}

/* ------------------------------------------------------------------ */
/* Migration                                                            */
/* ------------------------------------------------------------------ */

typedef struct { int64_t ms; int32_t idx; } orc_rank;

static int orc_rank_cmp(const void *a, const void *b)
{
    const orc_rank *x = (const orc_rank *)a, *y = (const orc_rank *)b;
    if (x->ms < y->ms) return -1;
    if (x->ms > y->ms) return 1;
    return (x->idx < y->idx) ? -1 : (x->idx > y->idx);
}

/* Cell indices of an island sorted by (makespan, cell index) ascending:
 * the reading of the paper's sort of each island before migration
 * (Section 4.2-4.3): rank 0 is the best individual, rank N-1 the worst. */
void orc_rank_island(int32_t N, const int64_t *ms, int32_t *order)
{
    orc_rank *r = (orc_rank *)malloc((size_t)N * sizeof(orc_rank));
    for (int32_t i = 0; i < N; ++i) { r[i].ms = ms[i]; r[i].idx = i; }
    qsort(r, (size_t)N, sizeof(orc_rank), orc_rank_cmp);
    for (int32_t i = 0; i < N; ++i) order[i] = r[i].idx;
    free(r);
}

/* Ring migration: island i sends copies of its best k rows to island
 * (i+1) mod I, where the t-th best immigrant overwrites the destination's
 * rank N-1-t row (the worst first).  k = max(1, floor(num * min(N_i, N_dst)
 * / den)).  All ranks and rows are taken from a snapshot before any write.
 * pops[i] is [N_i][ld], ms[i] is [N_i]. */
void orc_migrate_ring(int32_t I, const int32_t *sizes, int64_t ld, int32_t n,
                      int16_t **pops, int64_t **ms, int64_t num, int64_t den)
{
    int32_t **order = (int32_t **)malloc((size_t)I * sizeof(int32_t *));
    int16_t **snap = (int16_t **)malloc((size_t)I * sizeof(int16_t *));
    int64_t **snap_ms = (int64_t **)malloc((size_t)I * sizeof(int64_t *));
    int32_t *kk = (int32_t *)malloc((size_t)I * sizeof(int32_t));
    for (int32_t i = 0; i < I; ++i) {
        order[i] = (int32_t *)malloc((size_t)sizes[i] * sizeof(int32_t));
        orc_rank_island(sizes[i], ms[i], order[i]);
    }
    for (int32_t i = 0; i < I; ++i) {
        int32_t dst = (i + 1) % I;
        int32_t nmin = sizes[i] < sizes[dst] ? sizes[i] : sizes[dst];
        int64_t k = (num * (int64_t)nmin) / den;
        if (k < 1) k = 1;
        kk[i] = (int32_t)k;
        snap[i] = (int16_t *)malloc((size_t)k * (size_t)n * sizeof(int16_t));
        snap_ms[i] = (int64_t *)malloc((size_t)k * sizeof(int64_t));
        for (int32_t t = 0; t < k; ++t) {
            int32_t src = order[i][t];
            memcpy(snap[i] + (int64_t)t * n, pops[i] + (int64_t)src * ld, (size_t)n * sizeof(int16_t));
            snap_ms[i][t] = ms[i][src];
        }
    }
    for (int32_t i = 0; i < I; ++i) {
        int32_t dst = (i + 1) % I;
        for (int32_t t = 0; t < kk[i]; ++t) {
            int32_t cell = order[dst][sizes[dst] - 1 - t];
            memcpy(pops[dst] + (int64_t)cell * ld, snap[i] + (int64_t)t * n, (size_t)n * sizeof(int16_t));
            ms[dst][cell] = snap_ms[i][t];
        }
    }
    for (int32_t i = 0; i < I; ++i) { free(order[i]); free(snap[i]); free(snap_ms[i]); }
    free(order); free(snap); free(snap_ms); free(kk);
}

/* Penetration migration between two islands A and B (Section 4.3,
 * Eq. (1)-(2)), read for makespans (lower is better): with best makespans
 * cA, cB, nothing moves if cA == cB.  Otherwise lo = min, hi = max,
 * beta = lo / hi and the move happens iff 1 - beta < theta, i.e.
 * (hi - lo) * theta_den < theta_num * hi; then alpha = 1 - beta and
 * floor(alpha * N) = floor((hi - lo) * N / hi) of the best rows of the
 * lower-makespan island overwrite as many of the worst rows of the other
 * (t-th best onto rank N-1-t), N = min(N_A, N_B).
 * Returns the signed count: > 0 for A -> B, < 0 for B -> A, 0 for none. */
int64_t orc_penetration_count(int64_t cA, int64_t cB, int32_t N,
                              int64_t theta_num, int64_t theta_den)
{
    if (cA == cB) return 0;
    int64_t lo = cA < cB ? cA : cB, hi = cA < cB ? cB : cA;
    if (!((hi - lo) * theta_den < theta_num * hi)) return 0;
    int64_t count = ((hi - lo) * (int64_t)N) / hi;
    return cA < cB ? count : -count;
}

int64_t orc_migrate_penetration(int32_t NA, int32_t NB, int64_t ld, int32_t n,
                                int16_t *popA, int64_t *msA, int16_t *popB, int64_t *msB,
                                int64_t theta_num, int64_t theta_den)
{
    int32_t *oa = (int32_t *)malloc((size_t)NA * sizeof(int32_t));
    int32_t *ob = (int32_t *)malloc((size_t)NB * sizeof(int32_t));
    orc_rank_island(NA, msA, oa);
    orc_rank_island(NB, msB, ob);
    int32_t N = NA < NB ? NA : NB;
    int64_t cnt = orc_penetration_count(msA[oa[0]], msB[ob[0]], N, theta_num, theta_den);
    int64_t k = cnt < 0 ? -cnt : cnt;
    int16_t *spop = cnt > 0 ? popA : popB;
    int64_t *sms = cnt > 0 ? msA : msB;
    int32_t *sord = cnt > 0 ? oa : ob;
    int16_t *dpop = cnt > 0 ? popB : popA;
    int64_t *dms = cnt > 0 ? msB : msA;
    int32_t *dord = cnt > 0 ? ob : oa;
    int32_t dN = cnt > 0 ? NB : NA;
    for (int64_t t = 0; t < k; ++t) {
        int32_t src = sord[t], dst = dord[dN - 1 - t];
        memcpy(dpop + (int64_t)dst * ld, spop + (int64_t)src * ld, (size_t)n * sizeof(int16_t));
        dms[dst] = sms[src];
    }
    free(oa); free(ob);
    return cnt;
}

/* ------------------------------------------------------------------ */
/* Surrogate-screened cellular generation                              */
/* ------------------------------------------------------------------ */

/* Each cell makes K candidate children, candidate k exactly as the cellular
 * child (tournaments, crossover, mutation) but with the draws of purpose
 * ORC_PURPOSE_SURROGATE + k.  The candidate with the lowest given score
 * (scores[c * K + k]; the lowest k on ties) is decoded exactly and replaces
 * the cell iff its makespan is lower (or not higher, with cell_replace_le).
 * The scores are an input (the network's predictions), so this checks the
 * screening around them.  chosen[c] receives the picked k.  Returns the
 * number of exact decodes. */
int64_t orc_screened_cellular_generation(int32_t n, int32_t S, const int32_t *M, const int32_t *p,
                                         const orc_params *prm, uint32_t island, uint32_t generation,
                                         int32_t rows, int32_t cols, int64_t ld,
                                         const int16_t *pop_in, const int64_t *ms_in,
                                         int16_t *pop_out, int64_t *ms_out,
                                         const float *scores, int32_t K, int32_t *chosen,
                                         int16_t *candidates /* [cells*K][n], may be NULL */)
{
    int32_t cells = rows * cols;
    int16_t *child = (int16_t *)malloc((size_t)n * sizeof(int16_t));
    int16_t *best = (int16_t *)malloc((size_t)n * sizeof(int16_t));
    for (int32_t c = 0; c < cells; ++c) {
        int32_t pick = 0;
        for (int32_t k = 0; k < K; ++k) {
            uint32_t x[10];
            for (uint32_t d = 0; d < 10u; ++d)
                x[d] = orc_draw(prm->seed, ORC_PURPOSE_SURROGATE + (uint32_t)k, island, generation, (uint32_t)c, d);
            orc_cellular_child(n, rows, cols, c, x, prm, pop_in, ld, ms_in, child, NULL);
            if (candidates) memcpy(candidates + ((int64_t)c * K + k) * n, child, (size_t)n * sizeof(int16_t));
            if (k == 0 || scores[(int64_t)c * K + k] < scores[(int64_t)c * K + pick]) {
                pick = k;
                memcpy(best, child, (size_t)n * sizeof(int16_t));
            }
        }
        if (chosen) chosen[c] = pick;
        int64_t mc = orc_decode_obj(n, S, M, p, prm->obj, best, NULL);
        int better = prm->cell_replace_le ? (mc <= ms_in[c]) : (mc < ms_in[c]);
        int16_t *dst = pop_out + (int64_t)c * ld;
        if (better) {
            memcpy(dst, best, (size_t)n * sizeof(int16_t));
            ms_out[c] = mc;
        } else {
            memcpy(dst, pop_in + (int64_t)c * ld, (size_t)n * sizeof(int16_t));
            ms_out[c] = ms_in[c];
        }
    }
    free(child);
    free(best);
    return cells;
}

/* Surrogate-screened pseudo generation.  Pair k (rows 2k, 2k+1 = a, b)
 * crosses with probability pc, decided by draw 0 of purpose
 * ORC_PURPOSE_PSEUDO as in the plain generation; a pair that does not cross
 * is copied unchanged.  A crossing pair has K candidate cut pairs: candidate
 * t takes its cuts from draws 1 and 2 of purpose ORC_PURPOSE_SURROGATE_PSEUDO
 * + t (uniform in [0, n), l = min, r = max) and makes c1 = OX(a, b) and
 * c2 = OX(b, a) on them, with the given scores scores[2 (k K + t)] and
 * scores[2 (k K + t) + 1].  The candidate whose better child scores lowest,
 * min(score c1, score c2), wins (the lowest t on ties); only its two
 * children are decoded exactly, and the pair is replaced from them as in the
 * plain generation.  chosen[k] = the winning t, or -1 for a pair that did
 * not cross.  candidates (may be NULL) receives every pair's candidate
 * children, crossing or not, as rows [pairs][K][2][n].  Returns the number
 * of exact decodes. */
int64_t orc_screened_pseudo_generation(int32_t n, int32_t S, const int32_t *M, const int32_t *p,
                                       const orc_params *prm, uint32_t island, uint32_t generation,
                                       int32_t size, int64_t ld,
                                       const int16_t *pop_in, const int64_t *ms_in,
                                       int16_t *pop_out, int64_t *ms_out,
                                       const float *scores, int32_t K, int32_t *chosen,
                                       int16_t *candidates)
{
    int16_t *c1 = (int16_t *)malloc((size_t)n * sizeof(int16_t));
    int16_t *c2 = (int16_t *)malloc((size_t)n * sizeof(int16_t));
    int16_t *b1 = (int16_t *)malloc((size_t)n * sizeof(int16_t));
    int16_t *b2 = (int16_t *)malloc((size_t)n * sizeof(int16_t));
    int64_t decoded = 0;
    for (int32_t k = 0; k < size / 2; ++k) {
        const int16_t *a = pop_in + (int64_t)(2 * k) * ld;
        const int16_t *b = pop_in + (int64_t)(2 * k + 1) * ld;
        int16_t *oa = pop_out + (int64_t)(2 * k) * ld;
        int16_t *ob = pop_out + (int64_t)(2 * k + 1) * ld;
        /* every candidate, and the winner by its better child's score */
        int32_t pick = 0;
        float pick_score = 0.0f;
        for (int32_t t = 0; t < K; ++t) {
            const uint32_t purpose = ORC_PURPOSE_SURROGATE_PSEUDO + (uint32_t)t;
            const int32_t u = (int32_t)orc_uniform(orc_draw(prm->seed, purpose, island, generation, (uint32_t)k, 1u),
                                                   (uint32_t)n);
            const int32_t v = (int32_t)orc_uniform(orc_draw(prm->seed, purpose, island, generation, (uint32_t)k, 2u),
                                                   (uint32_t)n);
            const int32_t l = u < v ? u : v, r = u < v ? v : u;
            orc_order_crossover(n, a, b, l, r, c1);
            orc_order_crossover(n, b, a, l, r, c2);
            if (candidates) {
                memcpy(candidates + (((int64_t)k * K + t) * 2) * n, c1, (size_t)n * sizeof(int16_t));
                memcpy(candidates + (((int64_t)k * K + t) * 2 + 1) * n, c2, (size_t)n * sizeof(int16_t));
            }
            const float s1 = scores[((int64_t)k * K + t) * 2], s2 = scores[((int64_t)k * K + t) * 2 + 1];
            const float sc = s2 < s1 ? s2 : s1;
            if (t == 0 || sc < pick_score) {
                pick = t;
                pick_score = sc;
                memcpy(b1, c1, (size_t)n * sizeof(int16_t));
                memcpy(b2, c2, (size_t)n * sizeof(int16_t));
            }
        }
        const uint32_t x0 = orc_draw(prm->seed, ORC_PURPOSE_PSEUDO, island, generation, (uint32_t)k, 0u);
        if (!orc_bernoulli(x0, prm->pseudo_pc)) {
            if (chosen) chosen[k] = -1;
            memcpy(oa, a, (size_t)n * sizeof(int16_t));
            memcpy(ob, b, (size_t)n * sizeof(int16_t));
            ms_out[2 * k] = ms_in[2 * k];
            ms_out[2 * k + 1] = ms_in[2 * k + 1];
            continue;
        }
        if (chosen) chosen[k] = pick;
        const int64_t m1 = orc_decode_obj(n, S, M, p, prm->obj, b1, NULL);
        const int64_t m2 = orc_decode_obj(n, S, M, p, prm->obj, b2, NULL);
        decoded += 2;
        if (prm->pseudo_always) {
            memcpy(oa, b1, (size_t)n * sizeof(int16_t));
            memcpy(ob, b2, (size_t)n * sizeof(int16_t));
            ms_out[2 * k] = m1;
            ms_out[2 * k + 1] = m2;
            continue;
        }
        const int16_t *fam[4] = { b1, b2, a, b };
        int64_t fms[4] = { m1, m2, ms_in[2 * k], ms_in[2 * k + 1] };
        int32_t best2[2];
        orc_family_best2(fms, best2);
        memcpy(oa, fam[best2[0]], (size_t)n * sizeof(int16_t));
        memcpy(ob, fam[best2[1]], (size_t)n * sizeof(int16_t));
        ms_out[2 * k] = fms[best2[0]];
        ms_out[2 * k + 1] = fms[best2[1]];
    }
    free(c1); free(c2); free(b1); free(b2);
    return decoded;
}

/* ------------------------------------------------------------------ */
/* GA on the paper's own genotype (Section 4.1, genotype level): a row of */
/* L = n * S genes, gene j * S + s = the machine of job j at stage s.     */
/* The paper names no operators for it; the readings below are this      */
/* library's (random initial machines, complementary pairs by reflection, */
/* two-point crossover, one-gene machine reassignment), with the draws    */
/* and the selection / replacement rules of the job-order GA above.       */
/* ------------------------------------------------------------------ */

/* Initial row: gene i = uniform(M_{i mod S}) with draw i of the stream
 * (seed, purpose 1, island, generation 0, cell). */
void orc_assign_init_row(uint64_t seed, uint32_t island, uint32_t cell, int32_t n, int32_t S, const int32_t *M,
                         int16_t *genes)
{
    for (int32_t i = 0; i < n * S; ++i)
        genes[i] = (int16_t)orc_uniform(orc_draw(seed, ORC_PURPOSE_INIT, island, 0u, cell, (uint32_t)i),
                                        (uint32_t)M[i % S]);
}

/* Complement of a machine index at stage s: M_s - 1 - m.  When M_s is a
 * power of two, 2^b, this is the bitwise complement of m's b-bit binary
 * code (the binary lower layer of the genotype); otherwise it is the same
 * reflection, which keeps the gene a valid machine. */
int32_t orc_assign_complement(int32_t m, int32_t M_s) { return M_s - 1 - m; }

/* Complementary pair k of a pseudo island: rows 2k, 2k + 1 = a and its
 * complement, gene by gene; a is drawn with cell 2k. */
void orc_assign_init_pair(uint64_t seed, uint32_t island, int32_t k, int32_t n, int32_t S, const int32_t *M,
                          int16_t *a, int16_t *b)
{
    orc_assign_init_row(seed, island, (uint32_t)(2 * k), n, S, M, a);
    for (int32_t i = 0; i < n * S; ++i) b[i] = (int16_t)orc_assign_complement(a[i], M[i % S]);
}

/* Two-point crossover of strings of L genes: the child takes p1's genes at
 * positions l..r and p2's everywhere else. */
void orc_two_point(int32_t L, const int16_t *p1, const int16_t *p2, int32_t l, int32_t r, int16_t *child)
{
    for (int32_t i = 0; i < L; ++i) child[i] = (i >= l && i <= r) ? p1[i] : p2[i];
}

/* Machine reassignment of gene i (stage s = i mod S): with u = uniform(x,
 * M_s - 1), the gene becomes u if u < old, else u + 1 -- a machine other
 * than the old one, uniformly; no change when M_s = 1. */
void orc_assign_reassign(int16_t *genes, int32_t i, int32_t M_s, uint32_t x)
{
    if (M_s < 2) return;
    const int32_t old = genes[i];
    const int32_t u = (int32_t)orc_uniform(x, (uint32_t)(M_s - 1));
    genes[i] = (int16_t)(u < old ? u : u + 1);
}

/* One child of cell c of a cellular island of assignment strings, given its
 * ten draws (purpose 2): the two binary tournaments of orc_cellular_child
 * (draws 0-3), two-point crossover with probability pc (draw 4; cut points
 * uniform in [0, L) from draws 5 and 6, l = min, r = max), else a copy of
 * the first parent; with probability pm (draw 7) the reassignment of gene
 * uniform(L) (draw 8) with draw 9. */
void orc_assign_cellular_child(int32_t n, int32_t S, const int32_t *M, int32_t rows, int32_t cols, int32_t c,
                               const uint32_t x[10], const orc_params *prm, const int16_t *pop, int64_t ld,
                               const int64_t *obj, int16_t *child)
{
    const int32_t L = n * S;
    int32_t nb[5];
    orc_neighbours(rows, cols, c, nb);
    int32_t a1 = nb[orc_uniform(x[0], 5u)], b1 = nb[orc_uniform(x[1], 5u)];
    int32_t par1 = (obj[b1] < obj[a1]) ? b1 : a1;
    int32_t a2 = nb[orc_uniform(x[2], 5u)], b2 = nb[orc_uniform(x[3], 5u)];
    int32_t par2 = (obj[b2] < obj[a2]) ? b2 : a2;
    if (orc_bernoulli(x[4], prm->cell_pc)) {
        int32_t u = (int32_t)orc_uniform(x[5], (uint32_t)L);
        int32_t v = (int32_t)orc_uniform(x[6], (uint32_t)L);
        orc_two_point(L, pop + (int64_t)par1 * ld, pop + (int64_t)par2 * ld, u < v ? u : v, u < v ? v : u, child);
    } else {
        memcpy(child, pop + (int64_t)par1 * ld, (size_t)L * sizeof(int16_t));
    }
    if (orc_bernoulli(x[7], prm->cell_pm)) {
        const int32_t i = (int32_t)orc_uniform(x[8], (uint32_t)L);
        orc_assign_reassign(child, i, M[i % S], x[9]);
    }
}

/* One synchronous cellular generation of assignment strings: every cell's
 * child (orc_assign_cellular_child) is evaluated (orc_decode_assign) and
 * replaces the cell iff better (flag: not worse).  Returns the cells done. */
int64_t orc_assign_cellular_generation(int32_t n, int32_t S, const int32_t *M, const int32_t *p_u,
                                       const orc_params *prm, uint32_t island, uint32_t generation, int32_t rows,
                                       int32_t cols, int64_t ld, const int16_t *pop_in, const int64_t *obj_in,
                                       int16_t *pop_out, int64_t *obj_out)
{
    const int32_t L = n * S, cells = rows * cols;
    int16_t *child = (int16_t *)malloc((size_t)L * sizeof(int16_t));
    for (int32_t c = 0; c < cells; ++c) {
        uint32_t x[10];
        for (uint32_t d = 0; d < 10u; ++d)
            x[d] = orc_draw(prm->seed, ORC_PURPOSE_CELLULAR, island, generation, (uint32_t)c, d);
        orc_assign_cellular_child(n, S, M, rows, cols, c, x, prm, pop_in, ld, obj_in, child);
        const int64_t mc = orc_decode_assign(n, S, M, p_u, prm->obj, child, NULL);
        const int better = prm->cell_replace_le ? (mc <= obj_in[c]) : (mc < obj_in[c]);
        int16_t *dst = pop_out + (int64_t)c * ld;
        if (better) {
            memcpy(dst, child, (size_t)L * sizeof(int16_t));
            obj_out[c] = mc;
        } else {
            memcpy(dst, pop_in + (int64_t)c * ld, (size_t)L * sizeof(int16_t));
            obj_out[c] = obj_in[c];
        }
    }
    free(child);
    return cells;
}

/* One pseudo generation of assignment strings (Section 4.1): pair k =
 * rows (2k, 2k+1) = (a, b) crosses with probability pseudo_pc (draw 0,
 * purpose 3; cut points uniform in [0, L) from draws 1-2): c1 = two-point
 * (a, b), c2 = two-point (b, a); the pair keeps the two best of (c1, c2, a,
 * b) ranked by (objective, that order), best first, or with pseudo_always
 * the children.  Pairs that do not cross are copied.  Returns the children
 * evaluated. */
int64_t orc_assign_pseudo_generation(int32_t n, int32_t S, const int32_t *M, const int32_t *p_u,
                                     const orc_params *prm, uint32_t island, uint32_t generation, int32_t size,
                                     int64_t ld, const int16_t *pop_in, const int64_t *obj_in, int16_t *pop_out,
                                     int64_t *obj_out)
{
    const int32_t L = n * S;
    int16_t *c1 = (int16_t *)malloc((size_t)L * sizeof(int16_t));
    int16_t *c2 = (int16_t *)malloc((size_t)L * sizeof(int16_t));
    int64_t decoded = 0;
    for (int32_t k = 0; k < size / 2; ++k) {
        const int16_t *a = pop_in + (int64_t)(2 * k) * ld, *b = pop_in + (int64_t)(2 * k + 1) * ld;
        int16_t *oa = pop_out + (int64_t)(2 * k) * ld, *ob = pop_out + (int64_t)(2 * k + 1) * ld;
        const uint32_t x0 = orc_draw(prm->seed, ORC_PURPOSE_PSEUDO, island, generation, (uint32_t)k, 0u);
        if (!orc_bernoulli(x0, prm->pseudo_pc)) {
            memcpy(oa, a, (size_t)L * sizeof(int16_t));
            memcpy(ob, b, (size_t)L * sizeof(int16_t));
            obj_out[2 * k] = obj_in[2 * k];
            obj_out[2 * k + 1] = obj_in[2 * k + 1];
            continue;
        }
        const int32_t u = (int32_t)orc_uniform(orc_draw(prm->seed, ORC_PURPOSE_PSEUDO, island, generation,
                                                        (uint32_t)k, 1u), (uint32_t)L);
        const int32_t v = (int32_t)orc_uniform(orc_draw(prm->seed, ORC_PURPOSE_PSEUDO, island, generation,
                                                        (uint32_t)k, 2u), (uint32_t)L);
        const int32_t l = u < v ? u : v, r = u < v ? v : u;
        orc_two_point(L, a, b, l, r, c1);
        orc_two_point(L, b, a, l, r, c2);
        const int64_t m1 = orc_decode_assign(n, S, M, p_u, prm->obj, c1, NULL);
        const int64_t m2 = orc_decode_assign(n, S, M, p_u, prm->obj, c2, NULL);
        decoded += 2;
        if (prm->pseudo_always) {
            memcpy(oa, c1, (size_t)L * sizeof(int16_t));
            memcpy(ob, c2, (size_t)L * sizeof(int16_t));
            obj_out[2 * k] = m1;
            obj_out[2 * k + 1] = m2;
            continue;
        }
        const int16_t *fam[4] = { c1, c2, a, b };
        int64_t fobj[4] = { m1, m2, obj_in[2 * k], obj_in[2 * k + 1] };
        int32_t pick[2];
        orc_family_best2(fobj, pick);
        memcpy(oa, fam[pick[0]], (size_t)L * sizeof(int16_t));
        memcpy(ob, fam[pick[1]], (size_t)L * sizeof(int16_t));
        obj_out[2 * k] = fobj[pick[0]];
        obj_out[2 * k + 1] = fobj[pick[1]];
    }
    free(c1); free(c2);
    return decoded;
}
