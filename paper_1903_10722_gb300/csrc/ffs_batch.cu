// ffs_batch.cu -- many FFS instances of uneven size, each with one cellular
// island, evolved together: one persistent launch per generation, replayed
// from a CUDA graph, with the launch shape chosen by a timing autotuner.
//
// A generation is two launches.  k_batch_breed builds every instance's
// children (8 cells per warp, many warps: the crossover waits on the
// parents' loads) into per-instance child rows and copies each cell to its
// output row.  k_batch_cellular then decodes: work is split into units
// (instance, tile of `threads` cells), ordered heaviest first (decode cost ~
// n * sum_s (2 M_s + 6)); blocks of the persistent grid take the next unit
// from a device counter, stage that instance's processing-time table into
// shared memory, decode the tile's children and write each child that is
// better over its cell's copy.  Shared memory is sized for the largest
// instance.
#include <algorithm>
#include <cstddef>
#include <cstring>
#include <numeric>
#include <vector>

#include "ffs_internal.cuh"
#include "ffs_ga_device.cuh"

namespace fgpu {

struct BatchInst {
    int32_t n, S, SH, heap_words;
    uint32_t mulSH;
    int32_t ld;
    const uint32_t *tab;
    const int32_t *stage;
    int16_t *pop[2];
    int32_t *ms[2];
    int16_t *child;   // [cells][ld]: this generation's children
};

struct BatchShape {
    int B;          // jobs per round requested (instances with n <= B run in one round)
    int max_n, max_S, max_tw;
    int pairs;      // decoder variant: stages in interleaved pairs
    int tmem_cols;  // TMEM columns per block for saved heaps (0: none)
    int tmem_group_cols;  // columns per warp of a lane quarter
};

constexpr int kBatchCellsPerWarp = 8;

__device__ __forceinline__ IslandRef batch_ref(const BatchInst &I, const int32_t *cur, const int32_t *gen, int i)
{
    IslandRef ref;
    memset(&ref, 0, sizeof(ref));
    ref.pop[0] = I.pop[0];
    ref.pop[1] = I.pop[1];
    ref.ms[0] = I.ms[0];
    ref.ms[1] = I.ms[1];
    ref.dev_cur = cur;
    ref.dev_gen = gen;
    ref.island = (uint32_t)i;
    return ref;
}

// The breeding half of a generation of every instance: warp gw takes cells
// [8 q, 8 q + 8) of instance i (gw = i * warps_per_inst + q), lane l < 8 one
// cell: draws, tournaments, order crossover and swap into the instance's
// child row, the cell copied to its output row.  wbits: the warp's
// crossover mark, mark_words(max_n) words.
__global__ void __launch_bounds__(256, 4) k_batch_breed(const BatchInst *__restrict__ insts, int count, GaScalars g,
                                                     const int32_t *cur, const int32_t *gen, int rows, int cols,
                                                     int warps_per_inst, int mark_words_max)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * (blockDim.x >> 5) + warp;
    const int i = gw / warps_per_inst;
    if (i >= count) return;   // whole warps leave together
    const int cells = rows * cols;
    const int base = (gw - i * warps_per_inst) * kBatchCellsPerWarp;
    const BatchInst &I = insts[i];
    const int c = base + lane;
    const bool valid = lane < kBatchCellsPerWarp && c < cells;
    const int cq = valid ? c : base;
    cellular_warp_breed(batch_ref(I, cur, gen, i), g, I.n, cq, valid, rows, cols, I.ld, smem + warp * mark_words_max,
                        I.child + (int64_t)cq * I.ld);
}

__global__ void __launch_bounds__(512) k_batch_cellular(const BatchInst *__restrict__ insts, const int2 *__restrict__ units,
                                                        int n_units, int *counter, GaScalars g, const int32_t *cur,
                                                        const int32_t *gen, int rows, int cols, BatchShape shape,
                                                        unsigned long long *decoded, unsigned long long decoded_add,
                                                        int *err)
{
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ int s_unit;
    __shared__ int s_skip;
    __shared__ DecodeLayout s_L;
    __shared__ uint32_t s_tbase;
    const int T = blockDim.x;
    const SmemMap map = smem_map(shape.max_n, shape.max_S, T, 0);   // the crossover ran in k_batch_breed
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpStageState *wst = reinterpret_cast<WarpStageState *>(smem + map.warp) + warp * shape.max_S;
    int32_t *st = reinterpret_cast<int32_t *>(smem + map.stage);
    const uint16_t *tab = reinterpret_cast<const uint16_t *>(smem + map.tab);
    const int cells = rows * cols;
    if (decoded && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(decoded, decoded_add);
    // TMEM for saved heaps, held for the whole launch; freed after the loop
    if (shape.tmem_cols) {
        if (warp == 0) tc::tmem_alloc(&s_tbase, (uint32_t)shape.tmem_cols);
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
    }
    for (;;) {
        __syncthreads();  // the previous unit is done with shared memory
        if (threadIdx.x == 0) s_unit = atomicAdd(counter, 1);
        __syncthreads();
        const int u = s_unit;
        if (u >= n_units) break;
        const int2 un = units[u];
        const BatchInst &I = insts[un.x];
        const int n = I.n, S = I.S;
        stage_table(smem + map.tab, I.tab, table_words(n, S));
        for (int i = threadIdx.x; i < 2 * S; i += T) st[i] = I.stage[i];
        __syncthreads();   // the table and the stage array are complete in shared memory
        if (threadIdx.x == 0) {
            DecodeLayout &L = s_L;
            L.n = n;
            L.S = S;
            L.SH = I.SH;
            L.mulSH = I.mulSH;
            L.single = shape.B >= n ? 1 : 0;
            L.B = L.single ? round_up(n, 8) : shape.B;
            L.pairs = shape.pairs;
            L.M = st;
            L.heap_off = st + S;
            // this instance's stages whose heaps fit the warp's TMEM columns,
            // from the stage array in shared memory (complete since the
            // barrier above)
            const int32_t *gst = st;
            int ns = 0;
            if (!L.single && shape.tmem_cols)
                while (ns < S && gst[S + ns] + gst[ns] <= shape.tmem_group_cols) ++ns;
            L.tmem_cols = (uint32_t)shape.tmem_cols;
            L.tmem_group_cols = shape.tmem_group_cols;
            L.tmem_stages = ns;
            L.tmem_split = ns < S ? gst[S + ns] : I.heap_words;
            L.tmem_addr = s_tbase;
            L.obj_words = 0;   // batches decode the makespan
            L.has_rel = L.has_due = 0;
            L.wt = 0u;
            L.rel_sa = L.due_sa = 0u;
            L.heap_words = L.single ? 0 : I.heap_words - L.tmem_split;
            L.thread_words = L.heap_words + L.B + 4;
            // the unit's layout must stay inside what the launch was sized
            // for (shared words per thread, TMEM columns per warp); a unit
            // that does not is skipped and reported, never run out of range
            const bool fits = n <= shape.max_n && S <= shape.max_S && L.thread_words <= shape.max_tw &&
                              (ns == 0 || gst[S + ns - 1] + gst[ns - 1] <= shape.tmem_group_cols);
            s_skip = fits ? 0 : 1;
            if (!fits) atomicOr(err, 1);
        }
        __syncthreads();
        if (s_skip) continue;   // block-uniform; the loop head synchronises again
        const DecodeLayout &L = s_L;
        uint32_t *region = thread_region(smem + map.region, L.thread_words);
        const IslandRef ref = batch_ref(I, cur, gen, un.x);
        const int end = min(un.y + T, cells);
        for (int base = un.y + warp * 32; base < end; base += T) {
            const int c = base + lane;
            const bool valid = c < end;
            const int cq = valid ? c : end - 1;
            cellular_warp_decode_child(L, g, ref, cq, valid, I.ld, I.child + (int64_t)cq * I.ld, region, T, tab, wst);
        }
    }
    if (shape.tmem_cols) {
        tc::tmem_wait_st();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (warp == 0) tc::tmem_dealloc(s_tbase, (uint32_t)shape.tmem_cols);
    }
}

// The FFS_DEBUG_CHECKS build's validity pass over every instance's current
// rows (blockIdx.y = instance, one warp per row): warp_check_row.
__global__ void __launch_bounds__(128) k_check_batch(const BatchInst *insts, int count, const int32_t *cur,
                                                     int cells, int words_max)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const int warp = threadIdx.x >> 5;
    for (int i = blockIdx.y; i < count; i += gridDim.y) {
        const BatchInst &I = insts[i];
        for (int r = blockIdx.x * 4 + warp; r < cells; r += gridDim.x * 4)
            warp_check_row(I.pop[cur[0]] + (int64_t)r * I.ld, I.n, I.ms[cur[0]][r], smem + warp * words_max);
    }
}

__global__ void k_batch_advance(int32_t *cur, int32_t *gen)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        cur[0] ^= 1;
        gen[0] += 1;
    }
}

}  // namespace fgpu

using namespace fgpu;

struct ffs_batch {
    int count = 0, rows = 0, cols = 0;
    ffs_params prm{};
    std::vector<ffs_instance *> insts;
    std::vector<BatchInst> hinst;
    std::vector<double> cost;
    BatchInst *d_inst = nullptr;
    int2 *d_units = nullptr;
    int n_units = 0;
    int *d_counter = nullptr;
    int32_t *d_cur = nullptr, *d_gen = nullptr;
    unsigned long long *d_decoded = nullptr;
    int *d_err = nullptr;   // set by a unit whose layout exceeds the launch shape
    int host_cur = 0;
    long long host_gen = 0;
    int T = 0, B = 0, blocks_per_sm = 0;
    int max_n = 0;
    size_t smem = 0;
    BatchShape shape{};
    int num_sms = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    std::vector<void *> allocs;
};

namespace fgpu {

static void batch_free(ffs_batch *b)
{
    if (!b) return;
    if (b->graph) cudaGraphExecDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    for (void *p : b->allocs) cudaFree(p);
    for (ffs_instance *I : b->insts) ffs_instance_destroy(I);
    delete b;
}

// Shape (threads per block T, chunk B): feasibility and occupancy.  The
// decoder variant decides pairs and the TMEM option (as for a single
// instance): saved heaps in shared memory only, or the prefix of each
// instance's stages that fits the warp's TMEM column group, with `tb` blocks
// per SM sharing the 512 columns (shared memory padded so that no further
// block becomes resident).  Kept: most resident threads, then the TMEM
// preference of the variant.
static int batch_shape(ffs_batch *b, int T, int B, BatchShape *shape, size_t *smem, int *blocks)
{
    const int pref = tmem_of(b->prm.decode_variant);
    BatchShape best{};
    size_t best_bytes = 0;
    int best_nb = 0;
    long best_score = -1;
    for (int tb : {0, 1, 2, 4}) {
        if (tb && pref == 0) continue;
        BatchShape s{};
        s.B = B;
        s.pairs = pairs_of(b->prm.decode_variant);
        const int groups = (T / 32 + 3) / 4;
        s.tmem_cols = tb ? 512 / tb : 0;
        s.tmem_group_cols = tb ? s.tmem_cols / groups : 0;
        bool any_tmem = false;
        for (size_t i = 0; i < b->hinst.size(); ++i) {
            const BatchInst &I = b->hinst[i];
            s.max_n = std::max(s.max_n, I.n);
            s.max_S = std::max(s.max_S, I.S);
            const bool single = B >= I.n;
            int split = 0;
            if (tb && !single) {
                const ffs_instance *inst = b->insts[i];
                for (int st = 0; st < I.S && split + inst->M_eff[st] <= s.tmem_group_cols; ++st) split += inst->M_eff[st];
                any_tmem = any_tmem || split > 0;
            }
            const int tw = (single ? 0 : I.heap_words - split) + (single ? round_up(I.n, 8) : B) + 4;
            s.max_tw = std::max(s.max_tw, tw);
        }
        if (tb && !any_tmem) continue;
        const SmemMap m = smem_map(s.max_n, s.max_S, T, 0);
        size_t bytes = (size_t)(m.region + s.max_tw * T) * 4u;
        if (bytes > 232448) continue;
        auto occ = [&](size_t by) {
            int nb = 0;
            if (cudaFuncSetAttribute(k_batch_cellular, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)by) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_cellular, T, by) != cudaSuccess) {
                (void)cudaGetLastError();
                return 0;
            }
            return nb;
        };
        int nb = occ(bytes);
        while (tb && nb > tb && bytes + 4096 <= 232448) {
            bytes += 4096;
            nb = occ(bytes);
        }
        if (nb < 1 || (tb && nb != tb)) continue;
        const long score = (long)nb * T * 4 + (tb ? (pref == 2 ? 2 : -2) : 0);
        if (score > best_score) {
            best_score = score;
            best = s;
            best_bytes = bytes;
            best_nb = nb;
        }
    }
    if (best_score < 0) return FFS_EUNSUPPORTED;
    *shape = best;
    *smem = best_bytes;
    *blocks = best_nb;
    return FFS_OK;
}

// Work units (instance, first cell) for tiles of T cells, heaviest first.
static int batch_units(ffs_batch *b, int T, cudaStream_t st)
{
    const int cells = b->rows * b->cols;
    const int tiles = (cells + T - 1) / T;
    std::vector<int> order(b->count);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return b->cost[x] > b->cost[y]; });
    std::vector<int2> units;
    units.reserve((size_t)b->count * tiles);
    for (int i : order)
        for (int t = 0; t < tiles; ++t) units.push_back(make_int2(i, t * T));
    b->n_units = (int)units.size();
    FFS_CUDA_TRY(cudaMemcpyAsync(b->d_units, units.data(), units.size() * sizeof(int2), cudaMemcpyHostToDevice, st));
    FFS_CUDA_TRY(cudaStreamSynchronize(st));
    return FFS_OK;
}

static int batch_set_shape(ffs_batch *b, int T, int B, cudaStream_t st)
{
    BatchShape s;
    size_t smem;
    int nb;
    if (batch_shape(b, T, B, &s, &smem, &nb)) return set_error(FFS_EUNSUPPORTED, "batch shape T=%d B=%d does not fit", T, B);
    b->T = T;
    b->B = B;
    b->shape = s;
    b->smem = smem;
    b->blocks_per_sm = nb;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return batch_units(b, T, st);
}

// One generation's launches: the breeding launch, the counter reset and the
// persistent decode launch (breed = false: the decode launch alone, on the
// children of the last breeding launch); advance = false leaves the
// generation state untouched (autotuning, timing).
static int batch_generation(ffs_batch *b, bool advance, unsigned long long *decoded, cudaStream_t st,
                            bool breed = true)
{
    FFS_CUDA_TRY(cudaMemsetAsync(b->d_counter, 0, sizeof(int), st));
    if (breed) {
        NvtxRange r("ffs batch breed");
        const int cells = b->rows * b->cols;
        const int wpi = (cells + kBatchCellsPerWarp - 1) / kBatchCellsPerWarp;
        const int mw = mark_words(b->max_n);
        int Tb = 256;
        while (Tb > 32 && (size_t)(Tb / 32) * mw * 4 > 232448) Tb >>= 1;
        const size_t smem = (size_t)(Tb / 32) * mw * 4;
        if (smem > 232448) return set_error(FFS_EUNSUPPORTED, "crossover mark of n = %d too large", b->max_n);
        const long long warps = (long long)wpi * b->count;
        FFS_CUDA_TRY(cudaFuncSetAttribute(k_batch_breed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_batch_breed<<<(unsigned)((warps * 32 + Tb - 1) / Tb), Tb, smem, st>>>(
            b->d_inst, b->count, scalars_of(&b->prm), b->d_cur, b->d_gen, b->rows, b->cols, wpi, mw);
        FFS_CUDA_TRY(cudaGetLastError());
    }
    NvtxRange r("ffs batch decode + replace");
    FFS_CUDA_TRY(cudaFuncSetAttribute(k_batch_cellular, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->smem));
    int grid = b->num_sms * b->blocks_per_sm;
    if (grid > b->n_units) grid = b->n_units;
    k_batch_cellular<<<grid, b->T, b->smem, st>>>(b->d_inst, b->d_units, b->n_units, b->d_counter, scalars_of(&b->prm),
                                                   b->d_cur, b->d_gen, b->rows, b->cols, b->shape, decoded,
                                                   (unsigned long long)b->count * b->rows * b->cols, b->d_err);
    FFS_CUDA_TRY(cudaGetLastError());
    if (advance) {
        k_batch_advance<<<1, 32, 0, st>>>(b->d_cur, b->d_gen);
        FFS_CUDA_TRY(cudaGetLastError());
#ifdef FFS_DEBUG_CHECKS
        const int cells = b->rows * b->cols, words = (b->max_n + 31) >> 5;
        k_check_batch<<<dim3(std::min((cells + 3) / 4, 1024), std::min(b->count, 65535)), 128, 4 * words * 4, st>>>(
            b->d_inst, b->count, b->d_cur, cells, words);
        FFS_CUDA_TRY(cudaGetLastError());
#endif
    }
    return FFS_OK;
}

}  // namespace fgpu

extern "C" {

int ffs_batch_create(int32_t count, const int32_t *n_jobs, const int32_t *n_stages, const int32_t *machines,
                     const int32_t *proc_time, const ffs_params *prm, int32_t rows, int32_t cols, ffs_stream stream,
                     ffs_batch **out)
{
    clear_error();
    if (!out || !n_jobs || !n_stages || !machines || !proc_time || !prm) return set_error(FFS_EINVAL, "NULL argument");
    *out = nullptr;
    if (count < 1 || count > (1 << 20)) return set_error(FFS_EINVAL, "count %d", count);
    if (rows < 1 || cols < 1 || (int64_t)rows * cols > (1 << 24)) return set_error(FFS_EINVAL, "bad torus %dx%d", rows, cols);
    cudaStream_t st = (cudaStream_t)stream;
    ffs_batch *b = new ffs_batch();
    b->count = count;
    b->rows = rows;
    b->cols = cols;
    b->prm = *prm;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
    auto alloc = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) { (void)cudaGetLastError(); return nullptr; }
        b->allocs.push_back(p);
        return p;
    };
    const int cells = rows * cols;
    int64_t moff = 0, poff = 0;
    for (int i = 0; i < count; ++i) {
        ffs_instance *I = nullptr;
        int rc = ffs_instance_create(n_jobs[i], n_stages[i], machines + moff, proc_time + poff, &I);
        if (rc) {
            std::string msg = std::string("instance ") + std::to_string(i) + ": " + ffs_last_error();
            batch_free(b);
            return set_error(rc, "%s", msg.c_str());
        }
        b->insts.push_back(I);
        double c = 0;
        for (int s = 0; s < I->S; ++s) c += (double)I->n * (2.0 * I->M_eff[s] + 6.0);
        b->cost.push_back(c);
        BatchInst h;
        memset(&h, 0, sizeof(h));
        h.n = I->n;
        h.S = I->S;
        h.SH = I->SH;
        h.mulSH = 1u << I->SH;
        h.heap_words = I->heap_words;
        h.ld = round_up(I->n, 8);
        h.tab = I->d_tab;
        h.stage = I->d_stage;
        for (int k = 0; k < 2; ++k) {
            h.pop[k] = (int16_t *)alloc((size_t)cells * h.ld * 2);
            h.ms[k] = (int32_t *)alloc((size_t)cells * 4);
            if (!h.pop[k] || !h.ms[k]) {
                batch_free(b);
                return set_error(FFS_ENOMEM, "populations of instance %d", i);
            }
        }
        h.child = (int16_t *)alloc((size_t)cells * h.ld * 2);
        if (!h.child) {
            batch_free(b);
            return set_error(FFS_ENOMEM, "child rows of instance %d", i);
        }
        b->max_n = std::max(b->max_n, h.n);
        b->hinst.push_back(h);
        moff += n_stages[i];
        poff += (int64_t)n_jobs[i] * n_stages[i];
    }
    b->d_inst = (BatchInst *)alloc(sizeof(BatchInst) * count);
    b->d_units = (int2 *)alloc(sizeof(int2) * (size_t)count * cells);   // enough for tiles of >= 1 cell
    b->d_counter = (int *)alloc(sizeof(int));
    b->d_cur = (int32_t *)alloc(4);
    b->d_gen = (int32_t *)alloc(4);
    b->d_decoded = (unsigned long long *)alloc(8);
    b->d_err = (int *)alloc(4);
    if (!b->d_inst || !b->d_units || !b->d_counter || !b->d_cur || !b->d_gen || !b->d_decoded || !b->d_err) {
        batch_free(b);
        return set_error(FFS_ENOMEM, "batch state");
    }
    int rc = FFS_OK;
    if (cudaMemcpyAsync(b->d_inst, b->hinst.data(), sizeof(BatchInst) * count, cudaMemcpyHostToDevice, st) ||
        cudaMemsetAsync(b->d_cur, 0, 4, st) || cudaMemsetAsync(b->d_gen, 0, 4, st) ||
        cudaMemsetAsync(b->d_decoded, 0, 8, st) || cudaMemsetAsync(b->d_err, 0, 4, st))
        rc = set_error(FFS_ECUDA, "batch state initialisation");
    for (int i = 0; i < count && !rc; ++i) {
        rc = launch_init(b->insts[i], prm->seed, (uint32_t)i, 0, cells, b->hinst[i].ld, b->hinst[i].pop[0], st);
        if (!rc)
            rc = launch_eval(b->insts[i], b->hinst[i].pop[0], cells, b->hinst[i].ld, b->hinst[i].ms[0], nullptr, 0, 0,
                             nullptr, st);
    }
    // default shape: the largest tile that fits with chunk 32 (or the requested one)
    if (!rc) {
        const int Breq = prm->decode_chunk > 0 ? prm->decode_chunk : 32;
        const int Ts[4] = {256, 128, 64, 32};
        rc = FFS_EUNSUPPORTED;
        if (prm->block_threads > 0) {
            if (prm->block_threads % 32 == 0 && prm->block_threads <= 512)
                rc = batch_set_shape(b, prm->block_threads, Breq, st);
        } else {
            for (int t = 0; t < 4 && rc; ++t) rc = batch_set_shape(b, Ts[t], Breq, st);
        }
        if (rc) rc = set_error(FFS_EUNSUPPORTED, "no batch launch shape fits shared memory");
    }
    if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = set_error(FFS_ECUDA, "batch initialisation failed");
    if (rc) {
        batch_free(b);
        return rc;
    }
    *out = b;
    return FFS_OK;
}

int ffs_batch_destroy(ffs_batch *b)
{
    batch_free(b);
    return FFS_OK;
}

int ffs_batch_step(ffs_batch *b, int32_t n_generations, ffs_stream stream)
{
    clear_error();
    if (!b) return set_error(FFS_EINVAL, "NULL batch");
    if (n_generations < 0) return set_error(FFS_EINVAL, "n_generations %d < 0", n_generations);
    if (n_generations == 0) return FFS_OK;
    NvtxRange call("ffs_batch_step");
    if (eager_generations()) {
        for (int g = 0; g < n_generations; ++g) {
            NvtxRange gen("ffs batch generation");
            int rc = batch_generation(b, true, b->d_decoded, (cudaStream_t)stream);
            if (rc) return rc;
            b->host_cur ^= 1;
            b->host_gen += 1;
        }
        return FFS_OK;
    }
    if (!b->graph) {
        if (!b->cap_stream) FFS_CUDA_TRY(cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking));
        cudaGraph_t graph = nullptr;
        FFS_CUDA_TRY(cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeRelaxed));
        int rc = batch_generation(b, true, b->d_decoded, b->cap_stream);
        cudaError_t e = cudaStreamEndCapture(b->cap_stream, &graph);
        if (rc) {
            if (graph) cudaGraphDestroy(graph);
            return rc;
        }
        if (e != cudaSuccess) return set_error(FFS_ECUDA, "graph capture: %s", cudaGetErrorString(e));
        e = cudaGraphInstantiate(&b->graph, graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            b->graph = nullptr;
            return set_error(FFS_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
        }
    }
    for (int g = 0; g < n_generations; ++g) {
        FFS_CUDA_TRY(cudaGraphLaunch(b->graph, (cudaStream_t)stream));
        b->host_cur ^= 1;
        b->host_gen += 1;
    }
    return FFS_OK;
}

int ffs_batch_autotune(ffs_batch *b, int32_t repeats, ffs_stream stream, int32_t *threads_out, int32_t *chunk_out,
                       float *best_ms)
{
    clear_error();
    NvtxRange call("ffs_batch_autotune");
    if (!b) return set_error(FFS_EINVAL, "NULL batch");
    if (repeats < 1) repeats = 1;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    FFS_CUDA_TRY(cudaEventCreate(&e0));
    FFS_CUDA_TRY(cudaEventCreate(&e1));
    float best = -1.0f;
    int bestT = b->T, bestB = b->B, bestV = b->prm.decode_variant;
    const int Ts[7] = {64, 128, 256, 320, 384, 448, 512};
    const int Bs[9] = {8, 16, 32, 48, 64, 96, 104, 112, 128};
    int rc = FFS_OK;
    for (int vi = 1; vi <= kMaxVariant && !rc; ++vi)
    for (int ti = 0; ti < 7 && !rc; ++ti) {
        for (int bi = 0; bi < 9 && !rc; ++bi) {
            BatchShape s;
            size_t smem;
            int nb;
            b->prm.decode_variant = vi;
            if (batch_shape(b, Ts[ti], Bs[bi], &s, &smem, &nb)) continue;
            if ((rc = batch_set_shape(b, Ts[ti], Bs[bi], st))) break;
            // writes the next-generation buffers only; the state does not advance
            if ((rc = batch_generation(b, false, nullptr, st))) break;
            float fastest = -1.0f;   // the fastest of the timed runs: the least disturbed
            for (int r = 0; r < repeats && !rc; ++r) {
                cudaEventRecord(e0, st);
                rc = batch_generation(b, false, nullptr, st);
                cudaEventRecord(e1, st);
                if (cudaEventSynchronize(e1) != cudaSuccess) rc = set_error(FFS_ECUDA, "autotune timing");
                float ms = 0.0f;
                cudaEventElapsedTime(&ms, e0, e1);
                if (fastest < 0.0f || ms < fastest) fastest = ms;
            }
            const float avg = fastest;
            if (!rc && (best < 0.0f || avg < best)) {
                best = avg;
                bestT = Ts[ti];
                bestB = Bs[bi];
                bestV = vi;
            }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc) return rc;
    b->prm.decode_variant = bestV;
    if ((rc = batch_set_shape(b, bestT, bestB, st))) return rc;
    if (threads_out) *threads_out = bestT;
    if (chunk_out) *chunk_out = bestB;
    if (best_ms) *best_ms = best;
    return FFS_OK;
}

int ffs_batch_info(const ffs_batch *b, int32_t *count, int64_t *generation, int32_t *threads, int32_t *chunk,
                   int32_t *blocks_per_sm, int32_t *variant)
{
    clear_error();
    if (!b) return set_error(FFS_EINVAL, "NULL batch");
    if (variant) *variant = (b->shape.pairs ? 2 : 1) + (b->shape.tmem_cols ? 2 : 0);
    if (count) *count = b->count;
    if (generation) *generation = b->host_gen;
    if (threads) *threads = b->T;
    if (chunk) *chunk = b->B;
    if (blocks_per_sm) *blocks_per_sm = b->blocks_per_sm;
    return FFS_OK;
}

int ffs_batch_get(const ffs_batch *b, int32_t instance, int16_t *pop, int32_t ld_out, int32_t *ms, ffs_stream stream)
{
    clear_error();
    if (!b) return set_error(FFS_EINVAL, "NULL batch");
    if (instance < 0 || instance >= b->count) return set_error(FFS_EINVAL, "instance %d", instance);
    const BatchInst &h = b->hinst[instance];
    const int cells = b->rows * b->cols;
    cudaStream_t st = (cudaStream_t)stream;
    if (pop) {
        if (ld_out < h.n) return set_error(FFS_EINVAL, "ld_out %d < n %d", ld_out, h.n);
        FFS_CUDA_TRY(cudaMemcpy2DAsync(pop, (size_t)ld_out * 2, h.pop[b->host_cur], (size_t)h.ld * 2, (size_t)h.n * 2,
                                       cells, cudaMemcpyDefault, st));
    }
    if (ms) FFS_CUDA_TRY(cudaMemcpyAsync(ms, h.ms[b->host_cur], (size_t)cells * 4, cudaMemcpyDefault, st));
    return FFS_OK;
}

int ffs_batch_best(const ffs_batch *b, int32_t *best, ffs_stream stream)
{
    clear_error();
    if (!b || !best) return set_error(FFS_EINVAL, "NULL argument");
    const int cells = b->rows * b->cols;
    std::vector<int32_t> h((size_t)cells);
    cudaStream_t st = (cudaStream_t)stream;
    for (int i = 0; i < b->count; ++i) {
        FFS_CUDA_TRY(cudaMemcpyAsync(h.data(), b->hinst[i].ms[b->host_cur], (size_t)cells * 4, cudaMemcpyDeviceToHost, st));
        FFS_CUDA_TRY(cudaStreamSynchronize(st));
        int32_t m = -1;
        for (int32_t v : h)
            if (v >= 0 && (m < 0 || v < m)) m = v;
        best[i] = m;
    }
    return FFS_OK;
}

int ffs_batch_decoded(const ffs_batch *b, int64_t *count, ffs_stream stream)
{
    clear_error();
    if (!b || !count) return set_error(FFS_EINVAL, "NULL argument");
    unsigned long long v = 0;
    FFS_CUDA_TRY(cudaMemcpyAsync(&v, b->d_decoded, 8, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    FFS_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    *count = (int64_t)v;
    return FFS_OK;
}

int ffs_batch_dry_run(ffs_batch *b, int32_t kind, ffs_stream stream)
{
    clear_error();
    if (!b) return set_error(FFS_EINVAL, "NULL batch");
    if (kind != 0 && kind != 1) return set_error(FFS_EINVAL, "dry-run kind %d", kind);
    return batch_generation(b, false, nullptr, (cudaStream_t)stream, kind == 0);
}

int ffs_batch_check(const ffs_batch *b, ffs_stream stream)
{
    clear_error();
    if (!b) return set_error(FFS_EINVAL, "NULL batch");
    int v = 0;
    FFS_CUDA_TRY(cudaMemcpyAsync(&v, b->d_err, 4, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    FFS_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    if (v) return set_error(FFS_EDEVICE, "a batch work unit's layout exceeded the launch shape and was skipped");
    return FFS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Rows in, and checkpoint / resume of a batch.  Blob (host memory), every
// section padded to 16 bytes: BatchBlobHeader, then per instance its
// current rows [cells][ld_i] int16 and makespans [cells] int32.
// ---------------------------------------------------------------------------
namespace fgpu {

struct BatchBlobHeader {
    uint32_t magic, version;
    int32_t count, rows, cols, pad;
    uint64_t fingerprint;
    int64_t generation, decoded;
    int64_t bytes;       // the blob's length
    uint64_t checksum;   // blob_checksum of the whole blob, this field taken as zero
    ffs_params prm;
};
constexpr uint32_t kBatchBlobMagic = 0x42534646u, kBatchBlobVersion = 2;

static int64_t b16(int64_t b) { return (b + 15) / 16 * 16; }

static uint64_t batch_fingerprint(const ffs_batch *b)
{
    uint64_t h = 1469598103934665603ull;
    for (const ffs_instance *I : b->insts) h = instance_fingerprint(I, h);
    return h;
}

static int64_t batch_blob_bytes(const ffs_batch *b)
{
    const int64_t cells = (int64_t)b->rows * b->cols;
    int64_t s = b16(sizeof(BatchBlobHeader));
    for (const BatchInst &h : b->hinst) s += b16(cells * h.ld * 2) + b16(cells * 4);
    return s;
}

}  // namespace fgpu

extern "C" {

int ffs_batch_set(ffs_batch *b, int32_t instance, const int16_t *pop, int32_t ld_in, const int32_t *ms,
                  ffs_stream stream)
{
    clear_error();
    if (!b) return set_error(FFS_EINVAL, "NULL batch");
    if (instance < 0 || instance >= b->count) return set_error(FFS_EINVAL, "instance %d", instance);
    const BatchInst &h = b->hinst[instance];
    const int cells = b->rows * b->cols;
    cudaStream_t st = (cudaStream_t)stream;
    if (pop) {
        if (ld_in < h.n) return set_error(FFS_EINVAL, "ld_in %d < n %d", ld_in, h.n);
        FFS_CUDA_TRY(cudaMemcpy2DAsync(h.pop[b->host_cur], (size_t)h.ld * 2, pop, (size_t)ld_in * 2, (size_t)h.n * 2,
                                       cells, cudaMemcpyDefault, st));
    }
    if (ms) FFS_CUDA_TRY(cudaMemcpyAsync(h.ms[b->host_cur], ms, (size_t)cells * 4, cudaMemcpyDefault, st));
    return FFS_OK;
}

int64_t ffs_batch_checkpoint_bytes(const ffs_batch *b) { return b ? batch_blob_bytes(b) : -1; }

int ffs_batch_checkpoint_save(const ffs_batch *b, void *host, int64_t capacity, ffs_stream stream)
{
    clear_error();
    if (!b || !host) return set_error(FFS_EINVAL, "NULL argument");
    const int64_t need = batch_blob_bytes(b);
    if (capacity < need) return set_error(FFS_EINVAL, "capacity %lld < %lld bytes", (long long)capacity, (long long)need);
    cudaStream_t st = (cudaStream_t)stream;
    BlobWriter w{static_cast<char *>(host), capacity};
    BatchBlobHeader hd;
    memset(&hd, 0, sizeof(hd));
    hd.magic = kBatchBlobMagic;
    hd.version = kBatchBlobVersion;
    hd.count = b->count;
    hd.rows = b->rows;
    hd.cols = b->cols;
    hd.fingerprint = batch_fingerprint(b);
    hd.generation = b->host_gen;
    hd.bytes = need;
    hd.prm = b->prm;
    unsigned long long dec = 0;
    FFS_CUDA_TRY(cudaMemcpyAsync(&dec, b->d_decoded, 8, cudaMemcpyDeviceToHost, st));
    FFS_CUDA_TRY(cudaStreamSynchronize(st));
    hd.decoded = (int64_t)dec;
    memcpy(w.take(b16(sizeof(hd))), &hd, sizeof(hd));
    const int64_t cells = (int64_t)b->rows * b->cols;
    for (const BatchInst &h : b->hinst) {
        char *rows = w.take(b16(cells * h.ld * 2));
        char *ms = w.take(b16(cells * 4));
        FFS_CUDA_TRY(cudaMemcpyAsync(rows, h.pop[b->host_cur], (size_t)cells * h.ld * 2, cudaMemcpyDefault, st));
        FFS_CUDA_TRY(cudaMemcpyAsync(ms, h.ms[b->host_cur], (size_t)cells * 4, cudaMemcpyDefault, st));
    }
    FFS_CUDA_TRY(cudaStreamSynchronize(st));
    const uint64_t ck = blob_checksum(static_cast<const char *>(host), need, offsetof(BatchBlobHeader, checksum));
    memcpy(static_cast<char *>(host) + offsetof(BatchBlobHeader, checksum), &ck, 8);
    return FFS_OK;
}

int ffs_batch_checkpoint_load(ffs_batch *b, const void *host, int64_t size, ffs_stream stream)
{
    clear_error();
    if (!b || !host) return set_error(FFS_EINVAL, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    BlobReader r{static_cast<const char *>(host), size};
    const char *hp = r.take(b16(sizeof(BatchBlobHeader)));
    if (!hp) return set_error(FFS_EINVAL, "checkpoint truncated (header)");
    BatchBlobHeader hd;
    memcpy(&hd, hp, sizeof(hd));
    if (hd.magic != kBatchBlobMagic || hd.version != kBatchBlobVersion)
        return set_error(FFS_EINVAL, "not a batch checkpoint of this version");
    if (hd.bytes < (int64_t)sizeof(hd) || hd.bytes > size || hd.bytes % 16)
        return set_error(FFS_EINVAL, "checkpoint truncated (%lld of %lld bytes)", (long long)size, (long long)hd.bytes);
    if (blob_checksum(static_cast<const char *>(host), hd.bytes, offsetof(BatchBlobHeader, checksum)) != hd.checksum)
        return set_error(FFS_EINVAL, "checkpoint corrupted (checksum differs)");
    r.size = hd.bytes;   // only what the checksum covers is read
    if (hd.count != b->count || hd.rows != b->rows || hd.cols != b->cols)
        return set_error(FFS_EINVAL, "checkpoint of %d instances on %dx%d tori; this batch: %d on %dx%d", hd.count,
                         hd.rows, hd.cols, b->count, b->rows, b->cols);
    if (hd.fingerprint != batch_fingerprint(b)) return set_error(FFS_EINVAL, "checkpoint of other instances");
    if (hd.generation < 0 || hd.generation > 0x7FFFFFFF)
        return set_error(FFS_EINVAL, "generation %lld", (long long)hd.generation);
    const int64_t cells = (int64_t)b->rows * b->cols;
    std::vector<const char *> rows(b->count), mss(b->count);
    for (int i = 0; i < b->count; ++i) {
        rows[i] = r.take(b16(cells * b->hinst[i].ld * 2));
        mss[i] = r.take(b16(cells * 4));
        if (!rows[i] || !mss[i]) return set_error(FFS_EINVAL, "checkpoint truncated (instance %d)", i);
    }
    if (r.off != hd.bytes)
        return set_error(FFS_EINVAL, "checkpoint of %lld bytes, its sections %lld", (long long)hd.bytes, (long long)r.off);
    for (int i = 0; i < b->count; ++i) {
        const BatchInst &h = b->hinst[i];
        FFS_CUDA_TRY(cudaMemcpyAsync(h.pop[b->host_cur], rows[i], (size_t)cells * h.ld * 2, cudaMemcpyDefault, st));
        FFS_CUDA_TRY(cudaMemcpyAsync(h.ms[b->host_cur], mss[i], (size_t)cells * 4, cudaMemcpyDefault, st));
    }
    const int32_t g32 = (int32_t)hd.generation;
    FFS_CUDA_TRY(cudaMemcpyAsync(b->d_gen, &g32, 4, cudaMemcpyHostToDevice, st));
    const unsigned long long dec = (unsigned long long)hd.decoded;
    FFS_CUDA_TRY(cudaMemcpyAsync(b->d_decoded, &dec, 8, cudaMemcpyHostToDevice, st));
    FFS_CUDA_TRY(cudaStreamSynchronize(st));
    b->host_gen = hd.generation;
    // the GA parameters come back; the launch shape stays the one in use
    const ffs_params keep = b->prm;
    b->prm = hd.prm;
    b->prm.decode_chunk = keep.decode_chunk;
    b->prm.block_threads = keep.block_threads;
    b->prm.decode_variant = keep.decode_variant;
    if (b->graph) {
        cudaGraphExecDestroy(b->graph);
        b->graph = nullptr;
    }
    return FFS_OK;
}

}  // extern "C"
