// ffs_internal.cuh -- host-side internals shared by the library's .cu files.
#pragma once

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "../../include/ffs.h"
#include "ffs_device.cuh"

namespace fgpu {

// An NVTX range for the scope (a profiler shows the library's calls and the
// phases of a generation; free when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// FFS_EAGER=1 in the environment: generations run launch by launch instead
// of being replayed from captured CUDA graphs, so that each phase's NVTX
// range covers its own kernels in a profiler's timeline.
bool eager_generations();

// Thread-local error message; returns the status for one-line returns.
int set_error(int status, const char *fmt, ...);
void clear_error();

#define FFS_CUDA_TRY(expr)                                                                   \
    do {                                                                                     \
        cudaError_t e_ = (expr);                                                             \
        if (e_ != cudaSuccess)                                                               \
            return ::fgpu::set_error(FFS_ECUDA, "%s failed: %s (%s:%d)", #expr,                \
                                    cudaGetErrorString(e_), __FILE__, __LINE__);             \
    } while (0)

// Launch plan of a decoding kernel.
struct Plan {
    DecodeLayout L;
    int T = 0;            // threads per block
    size_t smem = 0;      // dynamic shared bytes
    int blocks_per_sm = 0;
    int smem_words_fixed = 0;  // table + stage descriptors + warp state
};

// Shared-memory word offsets inside a decoding block.
struct SmemMap {
    int tab;       // processing-time table, then the objective's release / due tables
    int stage;     // [2S]: M_s, heap offset
    int warp;      // warp state, (T/32) * S * 2 words
    int bits;      // per-warp crossover mark, (T/32) * bits_per_warp words
    int region;    // per-thread interleaved region
};

__host__ __device__ inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Words of the shared uint16 processing-time table (S rows of
// table_row_halves(n) entries), rounded to 16 bytes.
__host__ __device__ inline int table_words(int n, int S) { return round_up(S * table_row_halves(n) / 2, 4); }

// Words of the objective's tables (release and due times of job j at entry
// j + 1 of two uint32 arrays, entry 0 = 0), or 0 for the makespan alone.
__host__ __device__ inline int objective_words(int n) { return 2 * round_up(n + 1, 4); }

// Per-warp shared words for the order crossover's mark of the segment genes:
// one byte per gene (a plain store to set, a byte load to test), rounded to
// 16 bytes.
__host__ __device__ inline int mark_words(int n) { return round_up(n, 16) / 4; }

__host__ __device__ inline SmemMap smem_map(int n, int S, int T, int bits_per_warp = 0, int obj_words = 0)
{
    SmemMap m;
    m.tab = 0;
    m.stage = table_words(n, S) + obj_words;
    m.warp = m.stage + round_up(2 * S, 4);
    m.bits = m.warp + round_up((T / 32) * S * 2, 4);
    m.region = m.bits + round_up((T / 32) * bits_per_warp, 4);
    return m;
}

}  // namespace fgpu

struct ffs_instance {
    int n = 0, S = 0, SH = 0, device = 0;
    int64_t total_p = 0;
    std::vector<int32_t> host_M;     // machines per stage as given
    std::vector<int32_t> host_p;     // [n][S] processing times as given
    std::vector<int32_t> M_eff;      // min(M_s, n)
    std::vector<int32_t> heap_off;   // prefix sums of M_eff
    int heap_words = 0;
    uint32_t *d_tab = nullptr;       // uint16 [S][table_row_halves(n)] times, as words; then the
                                     // objective's release and due tables (obj_words)
    int obj_words = 0;               // objective_words(n) with release or due times, else 0
    int has_rel = 0, has_due = 0;
    int32_t wt = 0;                  // WT of the objective (0 without due times)
    std::vector<int32_t> host_R, host_D;
    int32_t *d_stage = nullptr;      // [2S]: M_eff, heap_off
    int tab_words = 0;
    int num_sms = 0;
    // launch plans already chosen: (kernel, chunk request, threads request, extra words)
    struct PlanKey { const void *kernel; int B_req, T_req, bits_per_warp, variant; };
    mutable std::vector<std::pair<PlanKey, fgpu::Plan>> plan_cache;
    // buffers of ffs_population_eval_host
    int16_t *d_host_pop = nullptr;
    int32_t *d_host_ms = nullptr;
    size_t host_cap = 0;
};

namespace fgpu {

// FNV-1a (64-bit) fingerprint of an instance as given (n, S, M, p, release,
// due, WT): a checkpoint records it so that it is only loaded into a handle
// of the same problem.
inline uint64_t instance_fingerprint(const ffs_instance *I, uint64_t h = 1469598103934665603ull)
{
    auto mix = [&h](int64_t v) {
        for (int b = 0; b < 8; ++b) {
            h ^= (uint64_t)((v >> (8 * b)) & 0xFF);
            h *= 1099511628211ull;
        }
    };
    mix(I->n);
    mix(I->S);
    for (int32_t v : I->host_M) mix(v);
    for (int32_t v : I->host_p) mix(v);
    mix((int64_t)I->host_R.size());
    for (int32_t v : I->host_R) mix(v);
    mix((int64_t)I->host_D.size());
    for (int32_t v : I->host_D) mix(v);
    mix(I->wt);
    return h;
}

// Failure injection for tests (host side, no device fault): with
// FFS_INJECT_ALLOC_FAILURE=k in the environment, the k-th device allocation
// of a network's buffers in the process (counting from 1) fails as an
// out-of-memory allocation would.  Unset: never.
bool injected_alloc_failure();

// Checksum of a checkpoint blob: FNV-1a over its 64-bit words (blobs are
// multiples of 16 bytes), the word at byte offset `skip` (the checksum's own
// field) taken as zero.
inline uint64_t blob_checksum(const char *p, int64_t bytes, int64_t skip)
{
    uint64_t h = 14695981039346656037ull;
    for (int64_t o = 0; o + 8 <= bytes; o += 8) {
        uint64_t w = 0;
        if (o != skip) memcpy(&w, p + o, 8);
        h ^= w;
        h *= 1099511628211ull;
    }
    return h;
}

// Bounds-checked writer / reader of a host checkpoint blob.
struct BlobWriter {
    char *p;
    int64_t cap, off = 0;
    char *take(int64_t bytes) {
        if (off + bytes > cap) return nullptr;
        char *q = p + off;
        off += bytes;
        return q;
    }
};
struct BlobReader {
    const char *p;
    int64_t size, off = 0;
    const char *take(int64_t bytes) {
        if (bytes < 0 || off + bytes > size) return nullptr;
        const char *q = p + off;
        off += bytes;
        return q;
    }
};

// Choose (B, T) for a decoding kernel, honouring requests (0 = choose).
// bits_per_warp: shared words per warp the kernel needs besides decoding
// (the crossover bitmask).  kernel: for the occupancy query.
// variant: 0 = library choice (stage pairs, saved heaps in TMEM where that
// raises the resident threads), 1 = one stage at a time, 2 = stages in
// interleaved pairs, 3 / 4 = as 1 / 2 with saved heaps in TMEM wherever the
// shape allows it (chunked decoding).
constexpr int kMaxVariant = 4;
// Variant 5: the stage-parallel decoder (ffs_lanes.cuh), for decode launches
// that accept it; not one of the launch shapes the autotuners sweep.
constexpr int kVariantLanes = 5;
int plan_decode(const ffs_instance *inst, const void *kernel, int B_req, int T_req, int bits_per_warp,
                Plan *out, int variant = 0);
inline int pairs_of(int variant) { return (variant == 1 || variant == 3) ? 0 : 1; }
inline int tmem_of(int variant) { return variant == 0 ? 1 : variant >= 3 ? 2 : 0; }

// Threads per block for a decoding launch of `units` rows when the caller
// asked for none (T_req = 0): with fewer than 512 rows per SM the planner's
// widest block would leave most SMs idle, so the block gets about
// rows / SMs threads (a multiple of 32, at least 32), which spreads the
// latency-bound decodes over every SM.  Otherwise 0 (the planner chooses).
inline int spread_threads(const ffs_instance *inst, int64_t units, int T_req);

// Grid size for N items (persistent, grid-stride).
inline int grid_for(const ffs_instance *inst, const Plan &p, int64_t N)
{
    int64_t need = (N + p.T - 1) / p.T;
    int64_t cap = (int64_t)inst->num_sms * (p.blocks_per_sm > 0 ? p.blocks_per_sm : 1);
    int64_t g = need < cap ? need : cap;
    return (int)(g < 1 ? 1 : g);
}

// Kernel-side view of where a GA step reads and writes.
struct IslandRef {
    const int16_t *pop_in;
    const int32_t *ms_in;
    int16_t *pop_out;
    int32_t *ms_out;
    int16_t *pop[2];
    int32_t *ms[2];
    const int32_t *dev_cur;   // non-null: in = [cur], out = [cur ^ 1]
    const int32_t *dev_gen;   // non-null: generation = *dev_gen + 1
    uint32_t generation;
    uint32_t island;
};

__device__ __forceinline__ void resolve(const IslandRef &r, const int16_t *&pin, const int32_t *&min_,
                                        int16_t *&pout, int32_t *&mout, uint32_t &gen)
{
    if (r.dev_cur) {
        const int c = *r.dev_cur;
        pin = r.pop[c];
        min_ = r.ms[c];
        pout = r.pop[c ^ 1];
        mout = r.ms[c ^ 1];
        gen = (uint32_t)(*r.dev_gen) + 1u;
    } else {
        pin = r.pop_in;
        min_ = r.ms_in;
        pout = r.pop_out;
        mout = r.ms_out;
        gen = r.generation;
    }
}

// Up to kMaxBatch islands of one kind stepped by one launch (same instance,
// same size); lanes of a warp may belong to different islands.
constexpr int kMaxBatch = 16;
struct IslandBatch {
    IslandRef ref[kMaxBatch];
    int count;
};

struct GaScalars {
    uint64_t seed, cell_pc, cell_pm, pseudo_pc;
    int32_t replace_le, pseudo_always;
    int32_t variant;   // decoder variant (plan_decode)
};

inline GaScalars scalars_of(const ffs_params *p)
{
    GaScalars g;
    g.seed = p->seed;
    g.cell_pc = p->cell_pc;
    g.cell_pm = p->cell_pm;
    g.pseudo_pc = p->pseudo_pc;
    g.replace_le = p->cell_replace_le;
    g.pseudo_always = p->pseudo_always;
    g.variant = p->decode_variant;
    return g;
}

// Launchers (defined in the .cu files).
// Launch plan of a stage-parallel decoding kernel (ffs_lanes.cuh): the heap
// size compiled for, chromosomes per warp, threads per block, dynamic shared
// bytes (table, stage array, each warp's staged rows) and blocks.
struct LanesPlan {
    int MM = 1, C = 1, T = 128, blocks = 1;
    size_t smem = 0;
};
bool lanes_decode_pays(const ffs_instance *inst, int64_t N, int variant);
int plan_lanes(const ffs_instance *inst, int64_t N, int ld, LanesPlan *out);

int launch_eval(const ffs_instance *inst, const int16_t *pop, int64_t N, int ld, int32_t *out,
                const int32_t *count_dev, int B_req, int T_req, unsigned long long *decoded,
                cudaStream_t st, int variant = 0);
int launch_init(const ffs_instance *inst, uint64_t seed, uint32_t island, int kind, int64_t N, int ld,
                int16_t *pop, cudaStream_t st);
int launch_cellular(const ffs_instance *inst, const GaScalars &g, const IslandBatch &batch, int rows,
                    int cols, int ld, int B_req, int T_req, unsigned long long *decoded,
                    cudaStream_t st);
int launch_pseudo(const ffs_instance *inst, const GaScalars &g, const IslandBatch &batch, int size,
                  int ld, void *scratch, int B_req, int T_req, unsigned long long *decoded,
                  cudaStream_t st);
// scratch for `islands` pseudo islands of `size` rows each
int64_t pseudo_scratch_bytes(int size, int ld, int islands = 1);
const void *cellular_kernel();
const void *eval_kernel();
const void *step_decode_kernel();

int validate_rows(const void *p, int ld, int n);

// Surrogate screening (ffs_surrogate.cu).
int launch_sur_candidates(const ffs_instance *inst, const GaScalars &g, const IslandBatch &batch, int rows, int cols,
                          int ld, int K, int16_t *cand, void *X, int xw, cudaStream_t st);
// Every candidate child of screened pseudo pairs ([pairs][K][2] rows of
// cand) and, with X non-null, their scoring input rows of xw values.
int launch_sur_pseudo_candidates(const ffs_instance *inst, const GaScalars &g, const IslandBatch &batch, int size,
                                 int ld, int K, int16_t *cand, void *X, int xw, cudaStream_t st);
int launch_sur_select(const ffs_instance *inst, const GaScalars &g, const IslandBatch &batch, int rows, int cols,
                      int ld, int K, const int16_t *cand, const float *scores, int32_t *chosen, int16_t *ring_rows,
                      int32_t *ring_ms, long long ring_cap, const long long *ctr, int B_req, int T_req,
                      unsigned long long *decoded, cudaStream_t st);
int launch_sur_gather(const int16_t *ring_rows, const int32_t *ring_ms, long long ring_cap, int recent,
                      long long *ctr, int ld, uint64_t seed, int B, int batches, float *targets,
                      float *norm, int n, int P, const float *inst_feat, int nfeat, void *X, int ldx,
                      cudaStream_t st);
int launch_sur_tick(long long *ctr, int which, long long add, cudaStream_t st);
int launch_fill_f32(float *p, int64_t n, float v, cudaStream_t st);
int mlp_in_dim(const ffs_mlp *m);
int mlp_max_batch(const ffs_mlp *m);
int64_t mlp_state_bytes(const ffs_mlp *m);
int mlp_save(const ffs_mlp *m, void *host, cudaStream_t st);                   // synchronises
int mlp_load(ffs_mlp *m, const void *host, int64_t size, cudaStream_t st);     // synchronises
int mlp_check_state(const ffs_mlp *m, const void *host, int64_t size);        // mlp_load's checks alone
// The scoring copy: allocate it (idempotent) and take it (stream-ordered);
// mlp_forward_folded reads it when asked to (with activations of its own;
// max_ctas > 0 caps the CTAs of its persistent GEMMs).
int mlp_enable_copy(ffs_mlp *m);
int mlp_take_copy(ffs_mlp *m, cudaStream_t st);
// Forward of rows whose network input is xpos[j] for j < kpos, zero for
// kpos <= j < P, the vector feat at [P, P + nfeat) and zero beyond: the
// constant block is folded into layer 1's bias (mlp_fold_bias, launched
// before it in stream order with the same weights), layer 1 contracts over
// the kpos leading columns (xpos rows of ldxpos BF16 values).  The weights
// read are the scoring copy's (use_copy) or the network's own.
int mlp_fold_bias(ffs_mlp *m, bool use_copy, int P, const float *feat, int nfeat, cudaStream_t st);
int mlp_forward_folded(ffs_mlp *m, bool use_copy, const void *xpos, int ldxpos, int kpos, int P, const float *feat,
                       int nfeat, int B, float *y, int max_ctas, cudaStream_t st);

inline int spread_threads(const ffs_instance *inst, int64_t units, int T_req)
{
    if (T_req > 0 || units <= 0 || inst->num_sms <= 0) return T_req;
    const int64_t per_sm = (units + inst->num_sms - 1) / inst->num_sms;
    if (per_sm >= 512) return 0;
    return (int)((per_sm + 31) / 32 * 32);
}

}  // namespace fgpu
