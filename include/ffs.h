/*
 * ffs.h -- C ABI of the GB300 library for the flexible flow shop (FFS) dual
 * island genetic algorithm of Luo & El Baz, "A Dual Heterogeneous Island
 * Genetic Algorithm for Solving Large Size Flexible Flow Shop Scheduling
 * Problems on Hybrid multi-core CPU and GPU Platforms" (arXiv:1903.10722).
 *
 * Every step of the hot path runs in this library's own CUDA kernels for
 * sm_103a.  Conventions shared by all calls:
 *   - Every call returns an ffs_status; FFS_OK is 0.  No call exits, aborts
 *     or traps; on failure ffs_last_error() (per host thread) says why.
 *   - Handles (ffs_instance, ffs_assign_instance, ffs_islands, ffs_batch,
 *     ffs_mlp) are opaque, owned by the library and released by their
 *     *_destroy call.
 *   - Host arrays given to *_create calls are copied; the caller keeps them.
 *   - "device" pointers must be CUDA device (or managed) memory of the
 *     current device; the call only enqueues work on `stream` and returns
 *     without waiting (stream-ordered, asynchronous) unless it says it
 *     synchronises.  `stream` is a cudaStream_t (NULL = legacy default).
 *   - Chromosomes are job orders: a row of n int16 genes, a permutation of
 *     0..n-1, rows `ld` genes apart (ld >= n, ld a multiple of 8, row base
 *     16-byte aligned) -- except for ffs_assign_eval, whose rows are the
 *     paper's machine-assignment strings (see there).
 *   - Makespans are int32.  A row holding a gene outside [0, n) gets
 *     makespan -1 (it is not decoded).
 */
#ifndef FFS_H
#define FFS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FFS_OK = 0,
    FFS_EINVAL = 1,        /* invalid argument (sizes, NULL, alignment, ranges) */
    FFS_ENOMEM = 2,        /* device or host allocation failed */
    FFS_ECUDA = 3,         /* a CUDA runtime call failed */
    FFS_EOVERFLOW = 4,     /* the instance's times do not fit the 32-bit keys */
    FFS_ETIMEOUT = 5,      /* a bounded device wait gave up */
    FFS_EDEVICE = 6,       /* a kernel reported an error word */
    FFS_EUNSUPPORTED = 7   /* valid input beyond this build's limits */
} ffs_status;

typedef struct ffs_instance ffs_instance;
typedef struct ffs_islands ffs_islands;
typedef void *ffs_stream;   /* cudaStream_t */

/* Message of the last failed call on this host thread ("" if none). */
const char *ffs_last_error(void);

/* ------------------------------------------------------------------------
 * Problem instance (Section 3): n jobs each pass stages 0..S-1 in order;
 * stage s has M_s identical parallel machines; job j takes proc_time[j][s]
 * time units at stage s on whichever machine it is given; no preemption.
 *
 * machines_per_stage: host int32[S], each >= 1.
 * proc_time: host int32[n][S] row-major (job-major), each in [1, 65535].
 * Limits: 1 <= n <= 32767 (int16 genes), 1 <= S <= 64, min(M_s, n) <= 32,
 * and sum of all proc_time below 2^(31 - ceil(log2(n + 1))) (the decoder's
 * 32-bit (time, job) keys; every completion time is at most that sum);
 * otherwise FFS_EINVAL / FFS_EUNSUPPORTED / FFS_EOVERFLOW.  Copies the
 * tables to the current device.  Synchronous.
 * ---------------------------------------------------------------------- */
int ffs_instance_create(int32_t n_jobs, int32_t n_stages, const int32_t *machines_per_stage,
                        const int32_t *proc_time, ffs_instance **out);

/* The same problem with the paper's objective (Section 3): job j may not
 * start its first operation before release[j], has due time due[j], and a
 * schedule costs  wt * sum_j max(0, C_j - due[j]) + C_max  (C_j = job j's
 * completion at the last stage); with Section 5 / Table 1, wt = 100.
 * release, due: host int32[n] (>= 0) or NULL (no release times / the
 * makespan alone; wt is then ignored).  Every "makespan" that the
 * evaluation and GA entry points below read or write is then this
 * objective.  Additional limits: max release + sum of proc_time within the
 * key bound above, and wt * n * (that bound) + (that bound) < 2^31 (the
 * objective is an int32), else FFS_EOVERFLOW; wt < 0: FFS_EINVAL.
 * Batches (ffs_batch_*) take the makespan alone. */
int ffs_instance_create_objective(int32_t n_jobs, int32_t n_stages, const int32_t *machines_per_stage,
                                  const int32_t *proc_time, const int32_t *release, const int32_t *due,
                                  int32_t wt, ffs_instance **out);
int ffs_instance_destroy(ffs_instance *inst);

/* ------------------------------------------------------------------------
 * The paper's own genotype (Section 4.1, genotype level; Section 3, P_jsm):
 * a string of n*S genes per row, gene j*S + s = the index (0-based) of the
 * machine that processes job j at stage s, on unrelated machines.
 *
 * ffs_assign_instance_create copies the instance: machines_per_stage[S]
 * (1..32), proc_time[n][W] int32 with W = sum_s M_s, the time of job j at
 * stage s on machine m at proc_time[j*W + M_0 + ... + M_{s-1} + m], every
 * time in [1, 65535]; release[n] and due[n] (host, nullable, >= 0) and WT as
 * in ffs_instance_create_objective.  FFS_EOVERFLOW when the latest possible
 * completion (max release + sum over jobs and stages of the slowest
 * machine) does not fit the key, or the objective bound does not fit int32.
 * Allocates library-owned device memory (the instance and a stream scratch
 * of up to 1 GiB); synchronous.
 *
 * ffs_assign_eval: objective[i] of row i of pop (device int16[N][ld], ld a
 * multiple of 8 and >= n*S; objective device int32[N]).  Sequencing, which
 * the paper leaves unstated: every machine processes the jobs assigned to it
 * in order of arrival -- stage 1: release time (0 without), later stages:
 * completion at the previous stage -- ties by job index; a job starts at
 * max(machine free time, arrival).  objective = C_max (+ WT * total
 * tardiness with due times); -1 for a row with a gene outside [0, M_s).
 * N = 0 is a no-op.  Asynchronous on `stream`; calls on one instance must
 * not overlap on the GPU (they share the stream scratch).
 * ---------------------------------------------------------------------- */
typedef struct ffs_assign_instance ffs_assign_instance;
int ffs_assign_instance_create(int32_t n_jobs, int32_t n_stages, const int32_t *machines_per_stage,
                               const int32_t *proc_time, const int32_t *release, const int32_t *due, int32_t wt,
                               ffs_assign_instance **out);
int ffs_assign_instance_destroy(ffs_assign_instance *inst);
int ffs_assign_eval(const ffs_assign_instance *inst, const int16_t *pop, int64_t N, int32_t ld, int32_t *objective,
                    ffs_stream stream);


/* ------------------------------------------------------------------------
 * Batched makespan evaluation (the decoder).  Each row is decoded by
 * stage-wise list scheduling: stage 0 takes the jobs in row order; every
 * later stage takes them in ascending (completion time at the previous
 * stage, job index) order; each job goes to the machine that is free
 * earliest (lowest index on ties) and starts at max(machine free time, its
 * completion at the previous stage).  makespan[i] = the last completion at
 * the last stage.  (Section 3 states the problem; the paper names only the
 * objective, this decoding rule is the library's reading.)
 *
 * pop: device int16[N][ld]; makespan: device int32[N].  N >= 0 (N = 0 is a
 * no-op).  Asynchronous on `stream`.
 * ---------------------------------------------------------------------- */
int ffs_population_eval(const ffs_instance *inst, const int16_t *pop, int64_t N, int32_t ld,
                        int32_t *makespan, ffs_stream stream);

/* Same, with an explicit launch shape: decode_chunk = jobs per round
 * (multiple of 8; >= n means one round per stage), block_threads
 * (multiple of 32, <= 512) and variant (0 library choice: stage pairs, the
 * heaps saved between rounds in tensor memory where that fits more threads
 * per SM; 1 one stage at a time, 2 stages in interleaved pairs, both with
 * the saved heaps in shared memory; 3 / 4 as 1 / 2 with the saved heaps in
 * tensor memory whenever the shape allows it (chunked decoding); 5 the
 * stage-parallel decoder: lane s of a group of S lanes runs stage s of one
 * chromosome, consuming the completions stage s - 1 emits one step earlier,
 * floor(32 / S) chromosomes per warp (S <= 32, else FFS_EUNSUPPORTED; chunk
 * and threads are ignored); FFS_EINVAL outside 0..5); 0 lets the library
 * choose: with chunk and threads 0 it takes the stage-parallel decoder where
 * a cost model fitted to GB300 measurements predicts it at most 0.7x the
 * time of one chromosome per lane (small launches of many-stage instances,
 * whose one-lane chains leave the GPU latency-bound).  Results do not
 * depend on the shape or variant. */
int ffs_population_eval_tuned(const ffs_instance *inst, const int16_t *pop, int64_t N, int32_t ld,
                              int32_t *makespan, int32_t decode_chunk, int32_t block_threads,
                              int32_t variant, ffs_stream stream);

/* The launch shape the library uses for a decoding kernel (kernel 0: the
 * batched decoder, 1: the fused cellular generation, 2: the fused decode
 * launch of a dual-island generation) given requested decode_chunk /
 * block_threads (0 = choose) and decoder variant (as in
 * ffs_population_eval_tuned): jobs per round, threads per block, resident
 * blocks per SM, dynamic shared bytes per block and the tensor-memory
 * columns each block allocates for saved heaps (0: none).  Host pointers;
 * any may be NULL.  Synchronous, launches nothing. */
int ffs_decode_plan(const ffs_instance *inst, int32_t kernel, int32_t decode_chunk, int32_t block_threads,
                    int32_t variant, int32_t *chunk, int32_t *threads, int32_t *blocks_per_sm,
                    int64_t *smem_bytes, int32_t *tmem_cols);

/* Same, with host (pageable or pinned) pop and makespan: copies pop in,
 * decodes and copies the makespans out on `stream`, then synchronises the
 * stream.  Uses a library-owned device buffer grown on demand. */
int ffs_population_eval_host(const ffs_instance *inst, const int16_t *pop, int64_t N, int32_t ld,
                             int32_t *makespan, ffs_stream stream);

/* ------------------------------------------------------------------------
 * Counter-based randomness: Philox4x32-10 (Salmon et al., SC 2011).  Draw
 * d of the stream (seed, purpose, island, generation, cell) is word d mod 4
 * of Philox applied to the counter (d / 4, cell, generation,
 * island | purpose << 24) under the key (low, high halves of seed).
 * Purposes: 1 initial population, 2 cellular generation, 3 pseudo
 * generation, 14 surrogate weight initialisation, 15 surrogate training
 * batches, 16 + k surrogate candidate k.
 * out: device uint32[n_cells][n_draws], row c holding cell cell0 + c.
 * ---------------------------------------------------------------------- */
#define FFS_PURPOSE_INIT 1
#define FFS_PURPOSE_CELLULAR 2
#define FFS_PURPOSE_PSEUDO 3
#define FFS_PURPOSE_MLP_INIT 14
#define FFS_PURPOSE_TRAIN_SAMPLE 15
#define FFS_PURPOSE_SURROGATE 16   /* + candidate index */
int ffs_philox_draws(uint64_t seed, uint32_t purpose, uint32_t island, uint32_t generation,
                     uint32_t cell0, int32_t n_cells, int32_t n_draws, uint32_t *out,
                     ffs_stream stream);

/* ------------------------------------------------------------------------
 * GA parameters.  Probabilities are thresholds t in [0, 2^32]: an event
 * fires iff its draw x < t (t = floor(p * 2^32)).  Defaults (Section 5):
 * cellular crossover 1.00 and mutation 0.05, pseudo crossover 0.75,
 * penetration threshold theta = 1, ring migration of 2% every 50
 * generations.
 * ---------------------------------------------------------------------- */
#define FFS_MIG_NONE 0
#define FFS_MIG_RING 1
#define FFS_MIG_PENETRATION 2

typedef struct {
    uint64_t seed;            /* Philox key */
    uint64_t cell_pc;         /* cellular crossover threshold */
    uint64_t cell_pm;         /* cellular mutation threshold (one swap per child) */
    uint64_t pseudo_pc;       /* pseudo crossover threshold */
    int32_t cell_replace_le;  /* 0: child replaces cell iff strictly better; 1: iff not worse */
    int32_t pseudo_always;    /* 0: pair keeps the 2 best of {c1, c2, a, b}; 1: children replace parents */
    int32_t migration_mode;   /* FFS_MIG_* used by ffs_island_step every migration_gap generations */
    int32_t migration_gap;    /* 0 = never inside ffs_island_step */
    int64_t ring_num, ring_den;    /* ring: k = max(1, floor(ring_num * N / ring_den)), k <= N/2 */
    int64_t theta_num, theta_den;  /* penetration threshold theta = num / den, in [0, 1] */
    int32_t decode_chunk;     /* decoder chunk (jobs per round, multiple of 8); 0 = library choice */
    int32_t block_threads;    /* threads per block for the decoder; 0 = library choice */
    int32_t decode_variant;   /* as in ffs_population_eval_tuned: 0 = library choice, 1 = one stage at a
                                 time, 2 = stages in interleaved pairs, 3 / 4 = as 1 / 2 with saved heaps
                                 in tensor memory (batches: 3 / 4 decode as 1 / 2) */
} ffs_params;

/* Fill *p with the defaults above (seed 7). */
void ffs_params_default(ffs_params *p);

/* ------------------------------------------------------------------------
 * Stateless generation steps on caller buffers (all device pointers).
 *
 * ffs_population_init: random initial rows (Section 4.1).  kind 0
 * (cellular): row c is the Fisher-Yates shuffle of the identity using
 * draws (seed, purpose 1, island, generation 0, cell c): for i = n-1 .. 1
 * swap genes i and uniform(i+1) with draw n-1-i, where uniform(k) of draw
 * x = (x * k) >> 32.  kind 1 (pseudo, N even): rows 2k, 2k+1 are a and its
 * complement, read as the reversed order, a drawn with cell 2k.  Padding
 * genes n..ld-1 are set to 0.  Makespans are not computed.
 *
 * ffs_cellular_step: one synchronous generation of a cellular island on an
 * rows x cols torus (Sections 4.1-4.2): every cell draws ten numbers
 * (purpose 2): two binary tournaments over its von Neumann neighbourhood
 * [itself, north, south, west, east] (draws 0-1 and 2-3; lower makespan
 * wins, the first drawn on ties), order crossover of the two winners with
 * probability cell_pc (draw 4, cut points from draws 5-6) or else a copy of
 * the first winner, one swap mutation with probability cell_pm (draw 7,
 * positions from draws 8-9), decoding, and replacement of the cell iff the
 * child is better.  Reads pop_in/ms_in, writes pop_out/ms_out (distinct
 * buffers of rows*cols rows).
 *
 * ffs_pseudo_step: one generation of a pseudo island of `size` rows (even)
 * (Sections 4.1-4.2): pair k = rows (2k, 2k+1) crosses with probability
 * pseudo_pc (draw 0, purpose 3; cut points from draws 1-2): c1 = OX(a, b),
 * c2 = OX(b, a); the pair keeps the two best of (c1, c2, a, b) ranked by
 * (makespan, that order), best first, or with pseudo_always the children.
 * Pairs that do not cross are copied.  scratch: device memory of
 * ffs_pseudo_scratch_bytes(size, ld) bytes, 256-byte aligned, owned by the
 * caller; its contents on entry do not matter.
 * ---------------------------------------------------------------------- */
int ffs_population_init(const ffs_instance *inst, uint64_t seed, uint32_t island, int32_t kind,
                        int64_t N, int32_t ld, int16_t *pop, ffs_stream stream);
int ffs_cellular_step(const ffs_instance *inst, const ffs_params *prm, uint32_t island,
                      uint32_t generation, int32_t rows, int32_t cols, int32_t ld,
                      const int16_t *pop_in, const int32_t *ms_in, int16_t *pop_out,
                      int32_t *ms_out, ffs_stream stream);
int64_t ffs_pseudo_scratch_bytes(int32_t size, int32_t ld);
int ffs_pseudo_step(const ffs_instance *inst, const ffs_params *prm, uint32_t island,
                    uint32_t generation, int32_t size, int32_t ld, const int16_t *pop_in,
                    const int32_t *ms_in, int16_t *pop_out, int32_t *ms_out, void *scratch,
                    ffs_stream stream);

/* ------------------------------------------------------------------------
 * ffs_pseudo_step without caller scratch.  The paper has no counterpart:
 * this is for callers that cannot allocate device memory (code running where
 * cudaMalloc is not allowed or must not block, or inside a framework that
 * owns every allocation).  It is ffs_pseudo_step with its scratch in a fixed
 * array of FFS_NOALLOC_SCRATCH_BYTES compiled into the library (a
 * file-scope __device__ array: each GPU that loads the library holds it
 * until the process exits).  The caller still passes inputs and outputs.
 *   - Sizes whose scratch (ffs_pseudo_scratch_bytes(size, ld)) exceeds the
 *     array are rejected with FFS_EUNSUPPORTED, e.g. size 4096 with ld 480
 *     fits, size 16384 with ld 504 does not.
 *   - It calls no cudaMalloc / cudaFree and no allocating library routine.
 *   - The first call in a CUDA context (per device, and again in the new
 *     primary context after cudaDeviceReset) looks up the array's device
 *     address (cudaGetSymbolAddress) with that device current; make that
 *     first call before any stream capture.  The address is cached per
 *     context (keyed on the driver's context ID).
 *   - Every call on a device shares the one array and leaves its contents
 *     behind; the slot counter is cleared on the stream at the start of each
 *     call.  Calls that overlap on the GPU (different streams, or
 *     concurrent graph branches) race on the array and give wrong results.
 * ---------------------------------------------------------------------- */
#define FFS_NOALLOC_SCRATCH_BYTES (4u << 20)
int ffs_pseudo_step_noalloc(const ffs_instance *inst, const ffs_params *prm, uint32_t island,
                            uint32_t generation, int32_t size, int32_t ld, const int16_t *pop_in,
                            const int32_t *ms_in, int16_t *pop_out, int32_t *ms_out, ffs_stream stream);

/* ------------------------------------------------------------------------
 * The GA on the paper's genotype (Section 4.1, genotype level).  The paper
 * names no operators for the machine-assignment string; the library's
 * (L = n * S genes per row):
 *   ffs_assign_population_init: kind 0, row r: gene i = uniform(M_{i mod S})
 *     with draw i of (seed, purpose 1, island, generation 0, cell r); kind 1
 *     (N even): rows 2k, 2k + 1 = a (drawn with cell 2k) and its
 *     complement, gene i -> M_s - 1 - a_i (the bitwise complement of the
 *     binary lower layer when M_s is a power of two; the same reflection
 *     keeps the gene a valid machine otherwise).  Padding genes are 0.
 *   ffs_assign_cellular_step: one synchronous generation of a rows x cols
 *     torus of assignment strings, the tournaments, draws and replacement
 *     of ffs_cellular_step (purpose 2) with two-point crossover (draw 4;
 *     cut points uniform in [0, L) from draws 5-6, l = min, r = max; the
 *     child takes the first winner's genes l..r and the second's elsewhere,
 *     or is a copy of the first winner) and machine reassignment (draw 7;
 *     gene uniform(L) from draw 8 moves to machine u or u + 1, u =
 *     uniform(M_s - 1) from draw 9, whichever is not its old machine).
 *   ffs_assign_pseudo_step: pair k crosses with probability pseudo_pc (draw
 *     0, purpose 3; cut points from draws 1-2): c1 = two-point(a, b), c2 =
 *     two-point(b, a); replacement as in ffs_pseudo_step.
 * Objectives (obj_in / obj_out, device int32) are those of ffs_assign_eval.
 * scratch: device memory of ffs_assign_step_scratch_bytes(N, ld) bytes
 * (N = the island's rows), 256-byte aligned, caller-owned; its contents on
 * entry do not matter.  Asynchronous; calls on one instance must not
 * overlap on the GPU (they share the evaluator's scratch). */
int ffs_assign_population_init(const ffs_assign_instance *inst, uint64_t seed, uint32_t island, int32_t kind,
                               int64_t N, int32_t ld, int16_t *pop, ffs_stream stream);
int64_t ffs_assign_step_scratch_bytes(int64_t N, int32_t ld);
int ffs_assign_cellular_step(const ffs_assign_instance *inst, const ffs_params *prm, uint32_t island,
                             uint32_t generation, int32_t rows, int32_t cols, int32_t ld, const int16_t *pop_in,
                             const int32_t *obj_in, int16_t *pop_out, int32_t *obj_out, void *scratch,
                             ffs_stream stream);
int ffs_assign_pseudo_step(const ffs_assign_instance *inst, const ffs_params *prm, uint32_t island,
                           uint32_t generation, int32_t size, int32_t ld, const int16_t *pop_in,
                           const int32_t *obj_in, int16_t *pop_out, int32_t *obj_out, void *scratch,
                           ffs_stream stream);

/* ------------------------------------------------------------------------
 * Islands: the dual-island GA state on the device (Section 4.1, Fig. 2).
 * Islands are kept in ring order [cellular 0, pseudo 0, cellular 1,
 * pseudo 1, ...]; island i uses Philox island id i.  Each cellular island is
 * a rows x cols torus, each pseudo island has pseudo_size rows (even).
 * ffs_islands_create allocates library-owned device memory, initialises
 * every island (ffs_population_init) and decodes it; generation = 0.
 * Device memory: two row buffers and two makespan buffers per island
 * (2 N ld 2 + 2 N 4 bytes), the rank order and ranking keys (12 N bytes),
 * the pseudo scratch (ffs_pseudo_scratch_bytes of the largest pseudo
 * island, for up to 16 pseudo islands at once) and, when both kinds are
 * present with at most 16 islands of each, the cellular children of one
 * generation (cells x ld x 2 bytes per cellular island).
 * ---------------------------------------------------------------------- */
int ffs_islands_create(const ffs_instance *inst, const ffs_params *prm, int32_t n_cellular,
                       int32_t rows, int32_t cols, int32_t n_pseudo, int32_t pseudo_size,
                       ffs_stream stream, ffs_islands **out);
int ffs_islands_destroy(ffs_islands *isl);

/* Number of islands, row stride, generation count; sizes (may be NULL)
 * receives n_islands int32 and kinds (may be NULL) 0 = cellular, 1 = pseudo. */
int ffs_islands_info(const ffs_islands *isl, int32_t *n_islands, int32_t *ld,
                     int64_t *generation, int32_t *sizes, int32_t *kinds);

/* Run n_generations synchronous generations of every island (island = -1)
 * or of one island; generation numbers continue from the handle's count.
 * After each generation g with migration_gap > 0 and g % migration_gap == 0,
 * runs ffs_migrate(migration_mode) (only when all islands are stepped).
 * The generation loop is replayed from a CUDA graph.  Asynchronous. */
int ffs_island_step(ffs_islands *isl, int32_t island, int32_t n_generations, ffs_stream stream);

/* Migration (Section 4.3).  Islands are ranked by (makespan, row index).
 * FFS_MIG_RING: island i sends copies of its k best rows to island
 * (i+1) mod I, the t-th best overwriting the destination's t-th worst,
 * k = max(1, floor(ring_num * min(N_i, N_dst) / ring_den)), all ranks
 * taken before any write.
 * FFS_MIG_PENETRATION (Eq. (1)-(2), for makespans): for each pair
 * (cellular q, pseudo q) with best makespans cA != cB, lo = min, hi = max:
 * if (hi - lo) * theta_den < theta_num * hi, the lower island's
 * floor((hi - lo) * N / hi) best rows overwrite the other's worst
 * (N = min of the two sizes).  Asynchronous. */
int ffs_migrate(ffs_islands *isl, int32_t mode, ffs_stream stream);

/* Copy island `island`'s current rows (into pop, row stride ld_out >= n;
 * ld_out equal to the handle's row stride, ffs_islands_info's ld, makes it
 * one contiguous copy that includes the padding genes) and makespans out,
 * or in (ffs_islands_set).  Pointers may be host or
 * device memory (copies use cudaMemcpyDefault); either may be NULL to skip.
 * Asynchronous on `stream` (pageable host memory makes the copy
 * synchronous with respect to the host, as CUDA does). */
int ffs_islands_get(const ffs_islands *isl, int32_t island, int16_t *pop, int32_t ld_out,
                    int32_t *makespan, ffs_stream stream);
int ffs_islands_set(ffs_islands *isl, int32_t island, const int16_t *pop, int32_t ld_in,
                    const int32_t *makespan, ffs_stream stream);
/* The same for every island in one call: the islands' rows back to back in
 * ring order (island i from row sum_{k<i} size_k), makespans likewise. */
int ffs_islands_get_all(const ffs_islands *isl, int16_t *pop, int32_t ld_out, int32_t *makespan,
                        ffs_stream stream);
int ffs_islands_set_all(ffs_islands *isl, const int16_t *pop, int32_t ld_in, const int32_t *makespan,
                        ffs_stream stream);

/* Best makespan over all islands and where it is (lowest island, then
 * lowest row on ties).  Synchronises `stream`.  Outputs are host pointers. */
int ffs_islands_best(const ffs_islands *isl, int32_t *best_makespan, int32_t *best_island,
                     int32_t *best_row, ffs_stream stream);

/* Number of exact decodes (children evaluated) since creation; synchronises. */
int ffs_islands_decoded(const ffs_islands *isl, int64_t *count, ffs_stream stream);

/* Per-island metrics (no counterpart in the paper).  A record is
 * FFS_STAT_WORDS int64 values for one island at one generation:
 *   [0] generation, [1] best makespan (-1 if no row is valid), [2] worst,
 *   [3] sum of the valid makespans (mean = [3] / [4]), [4] valid rows,
 *   [5] best makespan any metrics pass has seen since creation (-1: none),
 *   [6] migrations the island has received (ring or penetration events
 *   that delivered rows to it), [7] rows received by migration.
 * Makespans are the instance's objective when it has one.
 * ffs_islands_stats: the current generation's record of every island into
 * out[n_islands][FFS_STAT_WORDS] (host); synchronises `stream`.
 * ffs_islands_record_stats: from now on, one record per island at the end
 * of every generation (after migration), kept on the device in a ring of
 * `capacity` generations (0 switches recording off and frees it); the
 * current generation is recorded at once.  The records are written by a
 * kernel inside the captured generation graphs (one small launch per
 * generation); switching re-captures them.  All islands must be at the
 * same generation.  Synchronises `stream`.
 * ffs_islands_stats_history: *count = the records kept, the oldest kept
 * generation first (at most `capacity`); with out != NULL also copies them
 * to out[*count][n_islands][FFS_STAT_WORDS] (host; max_records >= *count,
 * else FFS_EINVAL).  Synchronises `stream`.
 * The best-so-far value and the migration counters travel in checkpoints. */
#define FFS_STAT_WORDS 8
int ffs_islands_stats(ffs_islands *isl, int64_t *out, ffs_stream stream);
int ffs_islands_record_stats(ffs_islands *isl, int32_t capacity, ffs_stream stream);
int ffs_islands_stats_history(const ffs_islands *isl, int64_t *out, int32_t max_records, int32_t *count,
                              ffs_stream stream);

/* ------------------------------------------------------------------------
 * Batch: many instances of uneven size, each evolving one cellular island
 * on a rows x cols torus (the island step of Sections 4.1-4.2 per instance;
 * instance i uses Philox island id i).  One generation of every instance is
 * one persistent kernel launch (blocks take (instance, tile) work units,
 * heaviest instances first, from a device counter), replayed from a CUDA
 * graph.
 *
 * ffs_batch_create: count instances given back to back: n_jobs[count],
 * n_stages[count], machines = the count M arrays concatenated,
 * proc_time = the count [n_i][S_i] tables concatenated (host memory; same
 * limits as ffs_instance_create).  Allocates library-owned device memory,
 * initialises every island and decodes it; synchronous.
 * ffs_batch_step: n_generations generations of every instance; async.
 * ffs_batch_autotune: times every launch shape (threads per block x decode
 * chunk x decoder variant) that fits, `repeats` timed runs each (a shape's
 * time is its fastest run), on generations that do not advance the state,
 * keeps the fastest shape and reports
 * it; synchronous.
 * ffs_batch_info: instance count, generations done, launch shape and the
 * decoder variant in use (1 / 2: one stage / stage pairs, saved heaps in
 * shared memory; 3 / 4: the same with saved heaps in tensor memory).
 * ffs_batch_get / ffs_batch_set: rows and makespans of one instance out /
 * in (host or device pointers, cudaMemcpyDefault; either may be NULL).
 * ffs_batch_best: best makespan of every instance into best[count] (host),
 * synchronous.
 * ffs_batch_checkpoint_bytes / _save / _load: the whole batch state (every
 * instance's rows and makespans, the generation count, the decode count and
 * the GA parameters) to or from a host blob of ffs_batch_checkpoint_bytes
 * bytes; both synchronise `stream`.  The blob carries its length and a
 * checksum of its contents (FNV-1a over 64-bit words).  Load reads no byte
 * past that length (`size` may be larger) and accepts only a complete,
 * unaltered blob whose sections fill its length exactly, of a batch of the
 * same instances and torus (FFS_EINVAL otherwise, nothing written); the
 * launch shape in use is kept.  Generations after a load draw the same
 * Philox streams as the uninterrupted run, so the results are identical.
 * ffs_batch_dry_run: kind 0 runs one generation's launches (breeding and
 * decoding) without advancing: the current rows, makespans, generation and
 * decode counts are unchanged, only the next generation's buffers are
 * written (as ffs_batch_autotune does); kind 1 runs the decoding launch
 * alone on the children of the last breeding launch (for timing it; run
 * kind 0 first).  Asynchronous.
 * ffs_batch_check: FFS_EDEVICE if any launch so far met a work unit whose
 * decode layout would exceed the shared memory or TMEM columns the launch
 * was sized for (that unit was skipped, its cells left as they were; the
 * kernel never accesses memory out of range), else FFS_OK; synchronises
 * `stream`.  The flag stays set for the batch's lifetime.
 * ---------------------------------------------------------------------- */
typedef struct ffs_batch ffs_batch;
int ffs_batch_create(int32_t count, const int32_t *n_jobs, const int32_t *n_stages, const int32_t *machines,
                     const int32_t *proc_time, const ffs_params *prm, int32_t rows, int32_t cols,
                     ffs_stream stream, ffs_batch **out);
int ffs_batch_destroy(ffs_batch *b);
int ffs_batch_step(ffs_batch *b, int32_t n_generations, ffs_stream stream);
int ffs_batch_autotune(ffs_batch *b, int32_t repeats, ffs_stream stream, int32_t *threads_out,
                       int32_t *chunk_out, float *best_ms);
int ffs_batch_info(const ffs_batch *b, int32_t *count, int64_t *generation, int32_t *threads,
                   int32_t *chunk, int32_t *blocks_per_sm, int32_t *variant);
int ffs_batch_get(const ffs_batch *b, int32_t instance, int16_t *pop, int32_t ld_out, int32_t *makespan,
                  ffs_stream stream);
int ffs_batch_set(ffs_batch *b, int32_t instance, const int16_t *pop, int32_t ld_in, const int32_t *makespan,
                  ffs_stream stream);
int ffs_batch_best(const ffs_batch *b, int32_t *best, ffs_stream stream);
int64_t ffs_batch_checkpoint_bytes(const ffs_batch *b);
int ffs_batch_checkpoint_save(const ffs_batch *b, void *host, int64_t capacity, ffs_stream stream);
int ffs_batch_checkpoint_load(ffs_batch *b, const void *host, int64_t size, ffs_stream stream);
int ffs_batch_decoded(const ffs_batch *b, int64_t *count, ffs_stream stream);
int ffs_batch_check(const ffs_batch *b, ffs_stream stream);
int ffs_batch_dry_run(ffs_batch *b, int32_t kind, ffs_stream stream);

/* ------------------------------------------------------------------------
 * Surrogate network (the paper has no surrogate: this is the library's
 * learned pre-screen of oversampled offspring, whose exact makespans still
 * come only from the decoder).
 *
 * ffs_gemm_bf16: D[M][N] (FP32, row stride ldd, 16-byte aligned) =
 * A[M][K] * B[N][K]^T with A, B BF16 (uint16 bit patterns), K-major rows
 * (strides lda, ldb in elements, multiples of 8, 16-byte aligned bases);
 * N a multiple of 64; rows of A past M and columns past K read as zero.
 * Runs on the 5th-generation tensor cores (TMA -> shared memory ->
 * tcgen05.mma -> tensor memory).  err: device int32 that a kernel sets to a
 * non-zero code if one of its bounded waits gave up.  Asynchronous.
 *
 * ffs_mlp: y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3 with BF16 weights and
 * activations and FP32 accumulation.  in_dim <= 4096; h1, h2 multiples of
 * 64 in [64, 1024]; batches up to max_batch (a multiple of 128).
 *   set_params/get take host FP32 arrays W1[h1][in_dim], b1[h1],
 *   W2[h2][h1], b2[h2], w3[h2], b3; get returns the parameters (which = 0),
 *   the last training step's gradients (1), or Adam's first (2) or second
 *   (3) moment estimates; both synchronise the device.  set_params resets
 *   Adam (moments 0, step count 0); ffs_mlp_adam_steps reports the count.
 *   ffs_mlp_init: He-uniform initialisation (limit sqrt(6 / fan_in)) drawn
 *   from Philox: W1[o][i] = lim1 * u(seed, purpose 14, island 1, cell o,
 *   draw i), W2 likewise with island 2 and fan_in h1, w3[j] = (lim3 * u(seed,
 *   14, 3, cell 0, draw j)) * 0.1, biases 0, where u(x) = ((x >> 8) - 2^23) /
 *   2^23 of the draw x and each product is rounded once to FP32; resets
 *   Adam.  Asynchronous on `stream`.
 *   ffs_mlp_state_bytes / ffs_mlp_save / ffs_mlp_load: parameters, Adam
 *   moments and step count to or from a host blob (a 40-byte header, then
 *   n_params FP32 parameters, first moments and second moments in the
 *   library's order); load accepts only a blob of a network of the same
 *   sizes.  Both synchronise `stream`.
 *   forward: x device BF16 [B][ldx] (ldx >= in_dim, multiple of 8), y
 *   device FP32 [B].  train_step: one Adam step (beta 0.9/0.999, eps 1e-8)
 *   on the mean squared error to target (device FP32 [B]); B a multiple of
 *   128; loss (device FP32, may be NULL) receives the batch MSE.
 *   ffs_mlp_check synchronises and returns FFS_ETIMEOUT if a tensor-core
 *   wait gave up since the last check.
 * ---------------------------------------------------------------------- */
typedef struct ffs_mlp ffs_mlp;
int ffs_gemm_bf16(const uint16_t *A, int32_t lda, const uint16_t *B, int32_t ldb, float *D, int32_t ldd,
                  int32_t M, int32_t N, int32_t K, int32_t *err, ffs_stream stream);
int ffs_mlp_create(int32_t in_dim, int32_t h1, int32_t h2, int32_t max_batch, ffs_mlp **out);
int ffs_mlp_destroy(ffs_mlp *mlp);
int ffs_mlp_input_width(const ffs_mlp *mlp);
int ffs_mlp_set_params(ffs_mlp *mlp, const float *W1, const float *b1, const float *W2, const float *b2,
                       const float *w3, float b3);
int ffs_mlp_get(const ffs_mlp *mlp, int32_t which, float *W1, float *b1, float *W2, float *b2, float *w3,
                float *b3);
int ffs_mlp_init(ffs_mlp *mlp, uint64_t seed, ffs_stream stream);
int ffs_mlp_adam_steps(const ffs_mlp *mlp, int64_t *steps);
int64_t ffs_mlp_state_bytes(const ffs_mlp *mlp);
int ffs_mlp_save(const ffs_mlp *mlp, void *host, int64_t capacity, ffs_stream stream);
int ffs_mlp_load(ffs_mlp *mlp, const void *host, int64_t size, ffs_stream stream);
int ffs_mlp_forward(ffs_mlp *mlp, const uint16_t *x, int32_t ldx, int32_t B, float *y, ffs_stream stream);
int ffs_mlp_train_step(ffs_mlp *mlp, const uint16_t *x, int32_t ldx, const float *target, int32_t B, float lr,
                       float *loss, ffs_stream stream);
int ffs_mlp_check(ffs_mlp *mlp, ffs_stream stream);

/* ------------------------------------------------------------------------
 * Surrogate-screened cellular islands.  After ffs_islands_attach_surrogate,
 * every generation of every cellular island: each cell makes `candidates`
 * children (candidate k exactly like the cellular child of
 * ffs_cellular_step, with Philox purpose 16 + k); the network scores them
 * (features: x[j] = position of job j / (n - 1) for j < n, zero up to
 * in_dim - 40, then 40 instance-summary values); only the lowest-scored
 * candidate (lowest k on ties) is decoded exactly and replaces the cell iff
 * better.  During the first warmup_generations every score is 0 (so
 * candidate 0 is taken).  Every exact (child, makespan) pair goes to a
 * device ring buffer.  After every generation G (counted from 1) with G %
 * train_every == 0, a training round of train_steps Adam steps on batches of
 * train_batch pairs, drawn uniformly (Philox purpose 15) from the pairs of
 * generations 1..G (the newest ring_capacity - cells pairs), with the
 * targets standardised by generation G's makespans, (makespan - mean) / std
 * (std at least 1): the screen needs only the ranking of a cell's
 * candidates.  With overlap = 1 (the default) the round runs beside the
 * whole of generation G + 1, which scores its candidates with the network
 * as it stood when G + 1 began (a copy of the weights taken then: trained
 * through the round after generation G - 1), and ends with the generation
 * (ring_capacity must then hold two generations' pairs); with overlap = 0
 * it runs beside G + 1's candidate building only and ends before G + 1's
 * candidates are scored.
 * With screen_pseudo = 0 the pseudo islands run the plain generation.  With
 * screen_pseudo = 1 a pair that crosses (the plain generation's decision,
 * draw 0 of its pseudo stream) has `candidates` candidate cut pairs,
 * candidate t with its cuts from draws 1 and 2 of Philox purpose 32 + t and
 * the children c1 = OX(a, b), c2 = OX(b, a); the network scores every
 * candidate child (of every pair, crossing or not), the candidate whose
 * better child scores lowest wins (the lowest t on ties), its two children
 * are decoded exactly and replace the pair as in the plain generation
 * (family best-2, or always); no pseudo pair enters the ring buffer.  The
 * pseudo islands then step together (at most 64 of them), and the network
 * must also have max_batch >= pseudo pairs x candidates x 2.  The network
 * must have in_dim >= n + 40 and max_batch >= cellular cells x candidates;
 * it is used, not owned;
 * ring_capacity must be at least cells + train_batch.  Generations are
 * replayed from CUDA graphs (captured on first use; four forms: before /
 * after the warm-up, with / without a training round).
 * ffs_islands_surrogate_last copies the last generation's scores
 * [cells x candidates] and picks [cells] (cellular islands in ring order),
 * the last training loss (mean squared error on the standardised targets),
 * the last generation's candidate rows (candidates [cells x
 * candidates][ld_out], may be NULL), and reports the pairs produced so far.
 * ---------------------------------------------------------------------- */
typedef struct {
    int32_t candidates;          /* children per cell, 1..16 (8) */
    int32_t train_every;         /* generations between training rounds (1; 0 = never) */
    int32_t train_steps;         /* Adam steps per round (2) */
    int32_t train_batch;         /* pairs per step, multiple of 128 (1024) */
    int32_t ring_capacity;       /* pairs kept (131072) */
    int32_t warmup_generations;  /* generations scored 0 while the ring fills (5) */
    float lr;                    /* Adam learning rate (1e-3) */
    int32_t overlap;             /* 1: the training round runs beside the whole screen (1) */
    int32_t screen_pseudo;       /* 1: the pseudo islands' pairs are screened too (0) */
} ffs_surrogate_params;
void ffs_surrogate_params_default(ffs_surrogate_params *p);
int ffs_islands_attach_surrogate(ffs_islands *isl, ffs_mlp *mlp, const ffs_surrogate_params *sp,
                                 ffs_stream stream);
int ffs_islands_surrogate_last(const ffs_islands *isl, float *scores, int32_t *chosen, float *loss,
                               int64_t *pairs, int16_t *candidates, int32_t ld_out, ffs_stream stream);
/* With screen_pseudo: the last generation's pseudo candidate children's
 * scores [pairs x candidates x 2] (pairs of the pseudo islands in island
 * order, then candidate, then child), the picks [pairs] (-1: the pair did
 * not cross) and the candidate children [pairs x candidates x 2][ld_out]
 * (may be NULL). */
int ffs_islands_surrogate_last_pseudo(const ffs_islands *isl, float *scores, int32_t *chosen, int16_t *candidates,
                                      int32_t ld_out, ffs_stream stream);

/* ------------------------------------------------------------------------
 * The checked build (no counterpart in the paper).  The library built with
 * -DFFS_DEBUG_CHECKS (libffs_gb300_debug.so) checks, on the device, the
 * index at each of the GA's indexing sites (tournament parents, crossover
 * cuts and writes, migration rows, the surrogate's ring slots and picks,
 * reassigned machine genes) and, after every generation of islands or of a
 * batch, that every row is a permutation of [0, n) with a makespan >= 0.
 * A failing check skips the access it guards and leaves its code in a
 * device error word (the first failure wins): 1 row not a permutation,
 * 2 tournament parent, 3 crossover cut, 4 crossover write, 5 migration row,
 * 6 ring slot, 7 surrogate pick, 8 machine gene.
 * ffs_debug_checks: *enabled = 1 in the checked build, 0 otherwise.
 * ffs_debug_check_error: synchronises `stream` and returns the error word in
 * *code (0: no check failed; always 0 in the normal build), clearing it when
 * reset != 0.
 * ---------------------------------------------------------------------- */
int ffs_debug_checks(int32_t *enabled);
int ffs_debug_check_error(int32_t *code, int32_t reset, ffs_stream stream);

/* ------------------------------------------------------------------------
 * Measurement and self-tests (no counterpart in the paper).
 * ffs_measure_int_rate: lane operations per second of one 32-bit
 * operation kind with 8 independent chains per thread at full occupancy;
 * best of 3 runs; synchronous.  kind: 0 min/max, 1 three-input logic,
 * 2 add, 3 multiply-add, 4 fp32 min/max on finite non-negative bit
 * patterns, 5 packed 16-bit min/max, 6 three-input min/max, 7 add-then-max,
 * 8 min/max and multiply-add alternating, 9 integer and fp32 min/max
 * alternating; FFS_EINVAL outside 0..9.
 * ffs_selftest_wait_timeout: a kernel waits on an mbarrier that nothing
 * completes, with the same bounded wait the tensor-core kernels use
 * (limit_ns <= 2 s); returns FFS_ETIMEOUT with *status = 1 when the wait gave
 * up as it must, FFS_OK with *status = 0 if the phase completed.
 * ---------------------------------------------------------------------- */
int ffs_measure_int_rate(int32_t kind, double *lane_ops_per_s, float *ms, ffs_stream stream);
int ffs_selftest_wait_timeout(int64_t limit_ns, int32_t *status, ffs_stream stream);

/* Checkpoint support: set the generation count of every island (the
 * populations come back with ffs_islands_set); the next generation then
 * draws the same Philox streams as an uninterrupted run.  Synchronous. */
int ffs_islands_set_generation(ffs_islands *isl, int64_t generation);

/* Checkpoint / resume of the whole islands state to or from a host blob of
 * ffs_checkpoint_bytes(isl) bytes: every island's current rows and
 * makespans and generation count, the decode count, the GA parameters, and
 * with a surrogate attached its ring buffer (filled slots and counters),
 * training-round count and the network's parameters, Adam moments and step
 * count.  Save and load synchronise `stream`.  The blob carries its length
 * and a checksum of its contents (FNV-1a over 64-bit words); load reads no
 * byte past that length (`size` may be larger), refuses a truncated or
 * altered blob, one whose sections do not fill its length exactly, and GA
 * parameters outside ffs_islands_create's limits (FFS_EINVAL, nothing
 * written), and checks that it
 * comes from a handle of the same instance (a fingerprint of n, S, M, p and
 * the objective's tables), islands, row stride and surrogate shape (attach
 * the surrogate before loading), else FFS_EINVAL with nothing written; the
 * launch shape in use is kept.  Generations after a load are identical to
 * those of the uninterrupted run. */
int64_t ffs_checkpoint_bytes(const ffs_islands *isl);
int ffs_checkpoint_save(const ffs_islands *isl, void *host, int64_t capacity, ffs_stream stream);
int ffs_checkpoint_load(ffs_islands *isl, const void *host, int64_t size, ffs_stream stream);

/* Launch one generation's kernels (kind 0: the cellular islands alone,
 * 1: the pseudo islands alone, 2: all islands -- the breeding launch, the
 * fused decode launch of all cellular and pseudo children, pseudo replace --
 * exactly as ffs_island_step does, migration and generation advance
 * excepted), without advancing the state: only the next-generation buffers
 * are rewritten (for timing and profiling).  kind 3: the fused decode launch
 * alone, over the children the last kind-2 run (or generation) bred -- call
 * it after kind 2 to time that launch by itself; FFS_EINVAL for handles
 * whose generations do not use the fused launch.  Not with a surrogate
 * attached.  Asynchronous. */
int ffs_islands_dry_run(ffs_islands *isl, int32_t kind, ffs_stream stream);
int ffs_islands_params(const ffs_islands *isl, ffs_params *out);

/* Time one generation of every island at every launch shape and decoder
 * variant that fits, `repeats` timed runs each (a shape's time is its
 * fastest run), on generations that do not advance the state, keep the
 * fastest shape and report it (ffs_islands_params returns the parameters in
 * use); synchronous. */
int ffs_islands_autotune(ffs_islands *isl, int32_t repeats, ffs_stream stream, int32_t *threads_out,
                         int32_t *chunk_out, float *best_ms);

#ifdef __cplusplus
}
#endif
#endif /* FFS_H */
