// ffs_ga.cu -- GA generations on the GPU: the fused cellular generation
// (cellular-only islands), the pseudo island (complementary pairs), the
// generation of both kinds in two launches (k_breed_dual: every child built;
// k_step_decode: every child decoded and the cells replaced), migration
// (chunked ranking, ring and penetration copies), and the islands handle
// that replays one generation of every island from a CUDA graph.
#include <algorithm>
#include <cstddef>
#include <cmath>
#include <cstring>
#include <vector>

#include "ffs_internal.cuh"
#include "ffs_ga_device.cuh"

namespace fgpu {

// ---------------------------------------------------------------------------
// One generation of a cellular island, fused (see cellular_warp_cells).
// One thread per cell; islands of a batch are laid end to end.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_cellular(DecodeLayout L, const uint32_t *__restrict__ tab_g,
                                                  const int32_t *__restrict__ stage_g, GaScalars g,
                                                  const __grid_constant__ IslandBatch batch, int rows,
                                                  int cols, int ld,
                                                  unsigned long long *decoded)
{
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ DecodeLayout s_L;
    const int T = blockDim.x;
    const int bits_per_warp = mark_words(L.n);   // crossover mark: one byte per gene
    const SmemMap map = smem_map(L.n, L.S, T, bits_per_warp, L.obj_words);
    stage_table(smem + map.tab, tab_g, table_words(L.n, L.S) + L.obj_words);
    int32_t *st = reinterpret_cast<int32_t *>(smem + map.stage);
    for (int i = threadIdx.x; i < 2 * L.S; i += T) st[i] = stage_g[i];
    if (threadIdx.x == 0) {
        s_L = L;
        s_L.M = st;
        s_L.heap_off = st + L.S;
        const uint32_t objt = tc::smem_u32(smem + map.tab + table_words(L.n, L.S));
        s_L.rel_sa = L.has_rel ? objt : 0u;
        s_L.due_sa = L.has_due ? objt + (uint32_t)L.obj_words * 2u : 0u;
    }
    __syncthreads();
    DecodeLayout &Ls = s_L;
    decode_tmem_begin(Ls);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpStageState *wst = reinterpret_cast<WarpStageState *>(smem + map.warp) + warp * L.S;
    uint32_t *wbits = smem + map.bits + warp * bits_per_warp;
    uint32_t *region = thread_region(smem + map.region, Ls.thread_words);
    const uint16_t *tab = reinterpret_cast<const uint16_t *>(smem + map.tab);

    const int cells = rows * cols;
    const int total = cells * batch.count;
    if (decoded && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(decoded, (unsigned long long)total);

    for (int base = blockIdx.x * T + warp * 32; base < total; base += gridDim.x * T) {
        const int gc = base + lane;
        const bool valid = gc < total;
        const int bi = (valid ? gc : total - 1) / cells;
        const int c = (valid ? gc : total - 1) - bi * cells;
        cellular_warp_cells(Ls, g, batch.ref[bi], c, valid, rows, cols, ld, wbits, region, T, tab, wst);
    }
    decode_tmem_end(Ls);
}

const void *cellular_kernel() { return (const void *)k_cellular; }

int launch_cellular(const ffs_instance *inst, const GaScalars &g, const IslandBatch &batch, int rows, int cols,
                    int ld, int B_req, int T_req, unsigned long long *decoded, cudaStream_t st)
{
    Plan p;
    const int bits_per_warp = mark_words(inst->n);
    const int T_sp = spread_threads(inst, (int64_t)rows * cols * batch.count, T_req);
    int rc = plan_decode(inst, (const void *)k_cellular, B_req, T_sp, bits_per_warp, &p, g.variant);
    if (rc && T_sp != T_req) rc = plan_decode(inst, (const void *)k_cellular, B_req, T_req, bits_per_warp, &p, g.variant);
    if (rc) return rc;
    FFS_CUDA_TRY(cudaFuncSetAttribute(k_cellular, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
    const int grid = grid_for(inst, p, (int64_t)rows * cols * batch.count);
    k_cellular<<<grid, p.T, p.smem, st>>>(p.L, inst->d_tab, inst->d_stage, g, batch, rows, cols, ld, decoded);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

// ---------------------------------------------------------------------------
// Pseudo island.  Scratch layout (each part 256-byte aligned):
//   children int16[size][ld] | child_ms int32[size] | pair_slot int32[size/2] | count int32
// ---------------------------------------------------------------------------
static inline size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

int64_t pseudo_scratch_bytes(int size, int ld, int islands)
{
    const size_t rows = (size_t)size * islands;
    return (int64_t)(a256(rows * ld * 2) + a256(rows * 4) + a256((rows / 2 + 1) * 4) + 256);
}

struct PseudoScratch {
    int16_t *children;
    int32_t *child_ms;
    int32_t *pair_slot;
    int32_t *count;   // children this generation
    int32_t *work;    // next warp work unit of the fused decode launch (count + 1)
};

static PseudoScratch carve(void *base, int size, int ld, int islands)
{
    const size_t rows = (size_t)size * islands;
    char *p = static_cast<char *>(base);
    PseudoScratch s;
    s.children = reinterpret_cast<int16_t *>(p);
    p += a256(rows * ld * 2);
    s.child_ms = reinterpret_cast<int32_t *>(p);
    p += a256(rows * 4);
    s.pair_slot = reinterpret_cast<int32_t *>(p);
    p += a256((rows / 2 + 1) * 4);
    s.count = reinterpret_cast<int32_t *>(p);
    s.work = s.count + 1;
    return s;
}

// Pairs per warp of k_pseudo_breed / k_pseudo_replace, and cells per warp
// of the cellular breeding: the warp builds (copies) its rows one after the other,
// so few rows per warp and many warps hide the memory latency of each.
constexpr int kPairsPerWarp = 4;
constexpr int kCellsPerWarp = 8;

// Lane l < kPairsPerWarp of a warp takes one pair: crossover decision,
// compacted child slots; the warp then builds the two children of each
// crossing pair cooperatively.
__device__ __forceinline__ void pseudo_breed_warp(const GaScalars &g, const IslandBatch &batch, int size, int n, int ld,
                                                  const PseudoScratch &s, int gw, uint32_t *bits)
{
    const int pairs = size / 2;
    const int total = pairs * batch.count;
    const int lane = threadIdx.x & 31;
    if (gw * kPairsPerWarp >= total) return;   // whole warps leave together
    const int gp = gw * kPairsPerWarp + lane;
    const bool mine = lane < kPairsPerWarp && gp < total;
    const int gq = mine ? gp : gw * kPairsPerWarp;
    const int bi = gq / pairs;
    const int k = gq - bi * pairs;
    const IslandRef &ref = batch.ref[bi];
    const int16_t *pin;
    const int32_t *msin;
    int16_t *pout;
    int32_t *msout;
    uint32_t gen;
    resolve(ref, pin, msin, pout, msout, gen);
    bool cross = false;
    U4 d{0, 0, 0, 0};
    if (mine) {
        d = draw_block(g.seed, kPurposePseudo, ref.island, gen, (uint32_t)k, 0u);
        cross = fires(d.x, g.pseudo_pc);
    }
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, cross);
    int base = 0;
    if (lane == 0 && mask) base = atomicAdd(s.count, 2 * __popc(mask));
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    const int slot = base + 2 * __popc(mask & ((1u << lane) - 1u));
    if (mine) s.pair_slot[gp] = cross ? slot : -1;
    const int u = (int)uniform_below(d.y, (uint32_t)n), v = (int)uniform_below(d.z, (uint32_t)n);
    const int16_t *a = pin + (int64_t)(2 * k) * ld;
    const int16_t *b = a + ld;
    ChildJob job;
    job.active = cross;
    job.cross = true;
    job.l = min(u, v);
    job.r = max(u, v);
    job.p1 = a;
    job.p2 = b;
    job.child = s.children + (int64_t)slot * ld;
    warp_build_children(job, n, ld, bits);
    job.p1 = b;
    job.p2 = a;
    job.child = s.children + (int64_t)(slot + 1) * ld;
    warp_build_children(job, n, ld, bits);
}

__global__ void k_pseudo_breed(GaScalars g, const __grid_constant__ IslandBatch batch, int size, int n, int ld,
                               PseudoScratch s)
{
    extern __shared__ uint32_t bits_smem[];
    pseudo_breed_warp(g, batch, size, n, ld, s, (blockIdx.x * blockDim.x + threadIdx.x) >> 5,
                      bits_smem + (threadIdx.x >> 5) * mark_words(n));
}

// Lane l < kPairsPerWarp of a warp takes one pair: it keeps the two best of
// (c1, c2, a, b), or the children, or itself when it did not cross.
__global__ void k_pseudo_replace(GaScalars g, const __grid_constant__ IslandBatch batch, int size, int ld,
                                 PseudoScratch s)
{
    const int pairs = size / 2;
    const int total = pairs * batch.count;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw * kPairsPerWarp >= total) return;   // whole warps leave together
    const int gp = gw * kPairsPerWarp + lane;
    const bool valid = lane < kPairsPerWarp && gp < total;
    const int gq = valid ? gp : gw * kPairsPerWarp;
    const int bi = gq / pairs, k = gq - bi * pairs;
    const int16_t *pin;
    const int32_t *msin;
    int16_t *pout;
    int32_t *msout;
    uint32_t gen;
    resolve(batch.ref[bi], pin, msin, pout, msout, gen);
    const int16_t *a = pin + (int64_t)(2 * k) * ld;
    const int16_t *b = a + ld;
    const int slot = s.pair_slot[gq];
    const int16_t *src[2];
    int32_t m[2];
    if (slot < 0) {
        src[0] = a; src[1] = b;
        m[0] = msin[2 * k]; m[1] = msin[2 * k + 1];
    } else {
        const int16_t *c1 = s.children + (int64_t)slot * ld, *c2 = c1 + ld;
        const int32_t fm[4] = {s.child_ms[slot], s.child_ms[slot + 1], msin[2 * k], msin[2 * k + 1]};
        int first = 0, second = 1;
        if (!g.pseudo_always) {
            for (int t = 1; t < 4; ++t)
                if ((uint32_t)fm[t] < (uint32_t)fm[first]) first = t;
            second = -1;
            for (int t = 0; t < 4; ++t) {
                if (t == first) continue;
                if (second < 0 || (uint32_t)fm[t] < (uint32_t)fm[second]) second = t;
            }
        }
        auto pick = [&](int t) { return t == 0 ? c1 : t == 1 ? c2 : t == 2 ? a : b; };
        src[0] = pick(first);
        src[1] = pick(second);
        m[0] = fm[first];
        m[1] = fm[second];
    }
    if (valid) {
        msout[2 * k] = m[0];
        msout[2 * k + 1] = m[1];
    }
    warp_copy_row_pairs(valid, src[0], pout + (int64_t)(2 * k) * ld, src[1], pout + (int64_t)(2 * k + 1) * ld, ld);
}

// The breeding half of a cellular generation for every cell of a batch of
// cellular islands (children into the output rows), kCellsPerWarp cells per
// warp, at high occupancy: its order crossover waits on memory, which many
// warps hide.
// children: child rows of the batch's cells (cell c of island bi at row
// bi * rows * cols + c), the cells copied to their output rows.
__device__ __forceinline__ void cellular_breed_warp(const GaScalars &g, const IslandBatch &batch, int rows, int cols,
                                                    int n, int ld, int gw, uint32_t *wbits, int16_t *children)
{
    const int lane = threadIdx.x & 31;
    const int cells = rows * cols, total = cells * batch.count;
    const int base = gw * kCellsPerWarp;
    if (base >= total) return;   // whole warps leave together
    const int gc = base + lane;
    const bool valid = lane < kCellsPerWarp && gc < total;
    const int gq = valid ? gc : base;
    const int bi = gq / cells, c = gq - bi * cells;
    cellular_warp_breed(batch.ref[bi], g, n, c, valid, rows, cols, ld, wbits, children + (int64_t)gq * ld);
}

// Both breeding halves of a dual generation in one launch: `cell_blocks`
// blocks breed the cellular cells, the others (launched first) the pseudo
// pairs; the two kinds of warps share the SMs and hide each other's memory
// latency.
__global__ void __launch_bounds__(256, 4) k_breed_dual(GaScalars g, const __grid_constant__ IslandBatch cb, int rows,
                                                    int cols, const __grid_constant__ IslandBatch pb, int psize,
                                                    int n, int ld, PseudoScratch s, int cell_blocks,
                                                    int16_t *cell_children)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const int warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
    uint32_t *wbits = smem + warp * mark_words(n);
    // the pseudo blocks first (0.3 % faster than the cellular ones first)
    const int P = gridDim.x - cell_blocks;
    if ((int)blockIdx.x >= P)
        cellular_breed_warp(g, cb, rows, cols, n, ld, (blockIdx.x - P) * wpb + warp, wbits, cell_children);
    else
        pseudo_breed_warp(g, pb, psize, n, ld, s, blockIdx.x * wpb + warp, wbits);
}

// Blocks of T threads for kPairsPerWarp pairs per warp.
static int pair_blocks(int pairs, int T)
{
    const long long warps = (pairs + kPairsPerWarp - 1) / kPairsPerWarp;
    return (int)((warps * 32 + T - 1) / T);
}

int launch_pseudo(const ffs_instance *inst, const GaScalars &g, const IslandBatch &batch, int size, int ld,
                  void *scratch, int B_req, int T_req, unsigned long long *decoded, cudaStream_t st)
{
    const int pairs = size / 2 * batch.count;
    if (pairs <= 0) return FFS_OK;
    PseudoScratch s = carve(scratch, size, ld, batch.count);
    FFS_CUDA_TRY(cudaMemsetAsync(s.count, 0, 2 * sizeof(int32_t), st));
    const int words = mark_words(inst->n);
    const int T = 128;
    const size_t smem = (size_t)(T / 32) * words * 4;
    if (smem > 232448) return set_error(FFS_EUNSUPPORTED, "crossover mark too large");
    FFS_CUDA_TRY(cudaFuncSetAttribute(k_pseudo_breed, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_pseudo_breed<<<pair_blocks(pairs, T), T, smem, st>>>(g, batch, size, inst->n, ld, s);
    FFS_CUDA_TRY(cudaGetLastError());
    int rc = launch_eval(inst, s.children, 2 * (int64_t)pairs, ld, s.child_ms, s.count, B_req, T_req, decoded, st,
                         g.variant);
    if (rc) return rc;
    k_pseudo_replace<<<pair_blocks(pairs, 128), 128, 0, st>>>(g, batch, size, ld, s);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

// Screened pseudo pairs (after the scoring of their candidates): lane
// l < kPairsPerWarp of a warp takes one pair.  The crossover decision is the
// plain generation's (draw 0, purpose kPurposePseudo); a crossing pair takes
// the candidate whose better child scores lowest, min(scores[2 (q K + t)],
// scores[2 (q K + t) + 1]) (the lowest t on ties), and its two children go
// to the compacted child slots that the decode and replacement launches of
// the plain generation then read.  chosen[q] = the pick, or -1.
__global__ void k_sur_pseudo_pick(GaScalars g, const __grid_constant__ IslandBatch batch, int size, int ld, int K,
                                  const int16_t *cand, const float *scores, int32_t *chosen, PseudoScratch s)
{
    const int pairs = size / 2;
    const int total = pairs * batch.count;
    const int lane = threadIdx.x & 31;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (gw * kPairsPerWarp >= total) return;   // whole warps leave together
    const int gp = gw * kPairsPerWarp + lane;
    const bool mine = lane < kPairsPerWarp && gp < total;
    const int gq = mine ? gp : gw * kPairsPerWarp;
    const int bi = gq / pairs, k = gq - bi * pairs;
    const int16_t *pin;
    const int32_t *msin;
    int16_t *pout;
    int32_t *msout;
    uint32_t gen;
    resolve(batch.ref[bi], pin, msin, pout, msout, gen);
    bool cross = false;
    int pick = 0;
    if (mine) {
        const U4 d = draw_block(g.seed, kPurposePseudo, batch.ref[bi].island, gen, (uint32_t)k, 0u);
        cross = fires(d.x, g.pseudo_pc);
        const float *sc = scores + (int64_t)gq * K * 2;
        float best = 0.0f;
        for (int t = 0; t < K; ++t) {
            const float s1 = sc[2 * t], s2 = sc[2 * t + 1];
            const float v = s2 < s1 ? s2 : s1;
            if (t == 0 || v < best) {
                best = v;
                pick = t;
            }
        }
        if (!FFS_DCHECK(pick >= 0 && pick < K, kCheckPick)) pick = 0;
        chosen[gq] = cross ? pick : -1;
    }
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, cross);
    int base = 0;
    if (lane == 0 && mask) base = atomicAdd(s.count, 2 * __popc(mask));
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    const int slot = base + 2 * __popc(mask & ((1u << lane) - 1u));
    if (mine) s.pair_slot[gp] = cross ? slot : -1;
    const int16_t *c1 = cand + ((int64_t)gq * K + pick) * 2 * ld;
    warp_copy_row_pairs(cross, c1, s.children + (int64_t)slot * ld, c1 + ld, s.children + (int64_t)(slot + 1) * ld,
                        ld);
}

// The rest of a screened pseudo generation once its candidates are scored:
// the picks into the child slots, their exact decode and the plain
// generation's replacement.
int launch_pseudo_screened(const ffs_instance *inst, const GaScalars &g, const IslandBatch &batch, int size, int ld,
                           int K, const int16_t *cand, const float *scores, int32_t *chosen, void *scratch, int B_req,
                           int T_req, unsigned long long *decoded, cudaStream_t st)
{
    const int pairs = size / 2 * batch.count;
    if (pairs <= 0) return FFS_OK;
    PseudoScratch s = carve(scratch, size, ld, batch.count);
    FFS_CUDA_TRY(cudaMemsetAsync(s.count, 0, 2 * sizeof(int32_t), st));
    k_sur_pseudo_pick<<<pair_blocks(pairs, 128), 128, 0, st>>>(g, batch, size, ld, K, cand, scores, chosen, s);
    FFS_CUDA_TRY(cudaGetLastError());
    int rc = launch_eval(inst, s.children, 2 * (int64_t)pairs, ld, s.child_ms, s.count, B_req, T_req, decoded, st,
                         g.variant);
    if (rc) return rc;
    k_pseudo_replace<<<pair_blocks(pairs, 128), 128, 0, st>>>(g, batch, size, ld, s);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

// ---------------------------------------------------------------------------
// One launch for the decoding work of a generation: the children of all
// cellular islands (bred by k_breed_dual into the output rows; decoded
// here, then replace-if-better) and the pseudo islands' compacted children.
// Warps take 32-unit work items from a device counter (cellular items first:
// they also replace and copy rows, and the heavier items go first), so the
// two kinds share one launch and its last wave instead of each leaving a
// partly idle wave.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_step_decode(DecodeLayout L, const uint32_t *__restrict__ tab_g,
                                                     const int32_t *__restrict__ stage_g, GaScalars g,
                                                     const __grid_constant__ IslandBatch cb, int rows, int cols, int ld,
                                                     PseudoScratch ps, const int16_t *cell_children,
                                                     unsigned long long *decoded)
{
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ DecodeLayout s_L;
    const int T = blockDim.x;
    const SmemMap map = smem_map(L.n, L.S, T, 0, L.obj_words);   // the crossover ran in k_breed_dual
    stage_table(smem + map.tab, tab_g, table_words(L.n, L.S) + L.obj_words);
    int32_t *st = reinterpret_cast<int32_t *>(smem + map.stage);
    for (int i = threadIdx.x; i < 2 * L.S; i += T) st[i] = stage_g[i];
    if (threadIdx.x == 0) {
        s_L = L;
        s_L.M = st;
        s_L.heap_off = st + L.S;
        const uint32_t objt = tc::smem_u32(smem + map.tab + table_words(L.n, L.S));
        s_L.rel_sa = L.has_rel ? objt : 0u;
        s_L.due_sa = L.has_due ? objt + (uint32_t)L.obj_words * 2u : 0u;
    }
    __syncthreads();
    DecodeLayout &Ls = s_L;
    decode_tmem_begin(Ls);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpStageState *wst = reinterpret_cast<WarpStageState *>(smem + map.warp) + warp * L.S;
    uint32_t *region = thread_region(smem + map.region, Ls.thread_words);
    const uint16_t *tab = reinterpret_cast<const uint16_t *>(smem + map.tab);
    const int cells = rows * cols;
    const int C = cells * cb.count, C32 = (C + 31) & ~31;
    const int P = *ps.count;
    const int witems = C32 / 32 + (P + 31) / 32;
    if (decoded && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(decoded, (unsigned long long)(C + P));
    for (;;) {
        int wu = 0;
        if (lane == 0) wu = atomicAdd(ps.work, 1);
        wu = __shfl_sync(0xFFFFFFFFu, wu, 0);
        if (wu >= witems) break;
        const int u0 = wu * 32;
        if (u0 < C32) {
            const int gc = u0 + lane;
            const bool valid = gc < C;
            const int gq = valid ? gc : C - 1;
            const int bi = gq / cells, c = gq - bi * cells;
            cellular_warp_decode_child(Ls, g, cb.ref[bi], c, valid, ld, cell_children + (int64_t)gq * ld, region, T,
                                       tab, wst);
        } else {
            const int k = u0 - C32 + lane;
            const bool valid = k < P;
            const int kk = valid ? k : P - 1;
            const int32_t ms = decode_chromosome(Ls, ps.children + (int64_t)kk * ld, region, T, tab, wst);
            if (valid) ps.child_ms[k] = ms;
        }
    }
    decode_tmem_end(Ls);
}

const void *step_decode_kernel() { return (const void *)k_step_decode; }

// A whole generation of the cellular batch `cb` and the pseudo batch `pb`
// (same torus for cb, same size for pb): pseudo breed, the fused decode
// launch, pseudo replace.
// decode_only: the decode launch alone, over the children that the last
// breeding launch left in the scratch (its work counter reset first); it
// rewrites the same next-generation rows, so it serves to time that launch.
static int launch_step_fused(const ffs_instance *inst, const GaScalars &g, const IslandBatch &cb, int rows, int cols,
                             const IslandBatch &pb, int psize, int ld, void *scratch, int16_t *cell_children,
                             int B_req, int T_req, unsigned long long *decoded, cudaStream_t st,
                             bool decode_only = false)
{
    PseudoScratch s = carve(scratch, psize, ld, pb.count);
    if (decode_only) {
        FFS_CUDA_TRY(cudaMemsetAsync(s.work, 0, sizeof(int32_t), st));
    } else {
        // cellular and pseudo breeding in one launch
        FFS_CUDA_TRY(cudaMemsetAsync(s.count, 0, 2 * sizeof(int32_t), st));   // count and work
        const int T = 256;
        const size_t smem = (size_t)(T / 32) * mark_words(inst->n) * 4;
        if (smem > 232448) return set_error(FFS_EUNSUPPORTED, "crossover mark too large");
        const int cell_warps = (rows * cols * cb.count + kCellsPerWarp - 1) / kCellsPerWarp;
        const int cell_blocks = (cell_warps + T / 32 - 1) / (T / 32);
        const int pseudo_blocks = pair_blocks(psize / 2 * pb.count, T);
        FFS_CUDA_TRY(cudaFuncSetAttribute(k_breed_dual, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        k_breed_dual<<<cell_blocks + pseudo_blocks, T, smem, st>>>(g, cb, rows, cols, pb, psize, inst->n, ld, s,
                                                                   cell_blocks, cell_children);
        FFS_CUDA_TRY(cudaGetLastError());
    }
    int rc;
    Plan p;
    const int T_sp = spread_threads(inst, (int64_t)rows * cols * cb.count + (int64_t)psize * pb.count, T_req);
    rc = plan_decode(inst, (const void *)k_step_decode, B_req, T_sp, 0, &p, g.variant);
    if (rc && T_sp != T_req) rc = plan_decode(inst, (const void *)k_step_decode, B_req, T_req, 0, &p, g.variant);
    if (rc) return rc;
    FFS_CUDA_TRY(cudaFuncSetAttribute(k_step_decode, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
    const int64_t units = (int64_t)rows * cols * cb.count + (int64_t)psize * pb.count;
    const int grid = grid_for(inst, p, units);
    k_step_decode<<<grid, p.T, p.smem, st>>>(p.L, inst->d_tab, inst->d_stage, g, cb, rows, cols, ld, s, cell_children,
                                             decoded);
    FFS_CUDA_TRY(cudaGetLastError());
    if (decode_only) return FFS_OK;
    const int pairs = psize / 2 * pb.count;
    k_pseudo_replace<<<pair_blocks(pairs, 128), 128, 0, st>>>(g, pb, psize, ld, s);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

// ---------------------------------------------------------------------------
// Migration.  Islands are ranked by (makespan, row): blocks sort chunks of
// 2048 keys (bitonic network in registers, shuffles and shared memory), then
// every key's rank in its island is its position in its chunk plus the keys
// below it in the island's other chunks (binary search); rows are then
// copied warp by warp.
// ---------------------------------------------------------------------------
struct IslandDesc {
    int16_t *pop[2];
    int32_t *ms[2];
    int32_t *order;    // [N] rows sorted by (makespan, row)
    int32_t N;
    int32_t kind;
    int32_t k_ring;    // rows sent to the next island by ring migration
    int32_t ring_off;  // prefix sum of k_ring
    int32_t row_off;   // the island's keys in the ranking scratch (prefix sum of N, each rounded up to even)
};

constexpr int kMaxMigrationRows = 16384;

// Migration runs iff gate is NULL, or the completed generation count
// gate[0] is a positive multiple of gap.
__device__ __forceinline__ bool migration_due(const int32_t *gate, int gap)
{
    if (!gate) return true;
    const int g = gate[0];
    return gap > 0 && g > 0 && (g % gap) == 0;
}

// Keys are (makespan << 32 | row), unique within an island.  A chunk of
// kRankChunk keys is sorted by one block of kRankChunk / 8 threads; a thread
// holds 8 consecutive keys e = 8 t + r in registers.  In shared memory key e
// sits at slot e + e / 8 (one pad slot per 8), so a thread's 8 keys load and
// store without bank conflicts.
constexpr int kRankChunk = 2048;
constexpr int kRankThreads = kRankChunk / 8;
__device__ __forceinline__ int rank_slot(int e) { return e + (e >> 3); }

// One compare-exchange step of distance J < 8 inside a thread's registers.
template <int J>
__device__ __forceinline__ void rank_reg_step(unsigned long long (&x)[8], int e0, int k)
{
#pragma unroll
    for (int r = 0; r < 8; ++r) {
        if ((r & J) == 0) {
            const unsigned long long a = x[r], b = x[r | J];
            const bool sw = (a > b) == (((e0 + r) & k) == 0);
            x[r] = sw ? b : a;
            x[r | J] = sw ? a : b;
        }
    }
}

// Block (chunk, island): sort keys [chunk * kRankChunk, ...) of the island
// into the scratch.  For each merge size k of the bitonic network the steps
// of distance j >= 256 run in shared memory, 8 <= j < 256 across the warp by
// shuffles (the partner of key 8 t + r is key 8 (t ^ j / 8) + r), j < 8 in
// registers.  Missing keys are padded with ~0 (they sort last).
__global__ void __launch_bounds__(kRankThreads) k_rank_chunks(const IslandDesc *desc, const int32_t *cur,
                                                              const int32_t *gate, int gap,
                                                              unsigned long long *scratch)
{
    if (!migration_due(gate, gap)) return;
    __shared__ unsigned long long keys[kRankChunk + kRankChunk / 8];
    const IslandDesc d = desc[blockIdx.y];
    const int c0 = blockIdx.x * kRankChunk;
    if (c0 >= d.N) return;   // the whole block
    const int len = min(kRankChunk, d.N - c0);
    const int32_t *ms = cur[blockIdx.y] ? d.ms[1] : d.ms[0];
    {
        uint32_t v[8];   // all loads in flight before the stores
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int e = threadIdx.x + i * kRankThreads;
            v[i] = e < len ? (uint32_t)ms[c0 + e] : 0u;
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int e = threadIdx.x + i * kRankThreads;
            keys[rank_slot(e)] = e < len ? ((unsigned long long)v[i] << 32) | (uint32_t)(c0 + e) : ~0ull;
        }
    }
    __syncthreads();
    const int t = threadIdx.x, e0 = 8 * t;
    for (int k = 2; k <= kRankChunk; k <<= 1) {
        int j = k >> 1;
        for (; j >= 256; j >>= 1) {
            for (int e = threadIdx.x; e < kRankChunk; e += blockDim.x) {
                const int o = e ^ j;
                if (o > e) {
                    const unsigned long long x = keys[rank_slot(e)], y = keys[rank_slot(o)];
                    if ((x > y) == ((e & k) == 0)) {
                        keys[rank_slot(e)] = y;
                        keys[rank_slot(o)] = x;
                    }
                }
            }
            __syncthreads();
        }
        unsigned long long x[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) x[r] = keys[rank_slot(e0 + r)];
        for (; j >= 8; j >>= 1) {
            const int lm = j >> 3;
            const bool lower = (t & lm) == 0;
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const unsigned long long y = __shfl_xor_sync(0xFFFFFFFFu, x[r], lm);
                const bool keep_min = lower == (((e0 + r) & k) == 0);
                x[r] = keep_min ? (x[r] < y ? x[r] : y) : (x[r] < y ? y : x[r]);
            }
        }
        if (j >= 4) rank_reg_step<4>(x, e0, k);
        if (j >= 2) rank_reg_step<2>(x, e0, k);
        rank_reg_step<1>(x, e0, k);
#pragma unroll
        for (int r = 0; r < 8; ++r) keys[rank_slot(e0 + r)] = x[r];
        __syncthreads();
    }
    unsigned long long *out = scratch + d.row_off + c0;
    for (int e = threadIdx.x; e < len; e += blockDim.x) out[e] = keys[rank_slot(e)];
}

// Block (1024 keys, island): the island's sorted chunks are staged in shared
// memory; a thread takes one key.  Its rank in the island = its position in
// its chunk + its lower bound in each other chunk, the lower bounds found by
// binary searches run side by side (independent shared loads).
// order[rank] = row; keys are unique, so the ranks are a permutation.
constexpr int kRankMergeThreads = 1024;
constexpr int kRankMaxChunks = kMaxMigrationRows / kRankChunk;

__global__ void __launch_bounds__(kRankMergeThreads) k_rank_merge(const IslandDesc *desc, const int32_t *gate, int gap,
                                                                  const unsigned long long *scratch)
{
    if (!migration_due(gate, gap)) return;
    extern __shared__ unsigned long long isl_keys[];
    const IslandDesc &d = desc[blockIdx.y];
    if (blockIdx.x * kRankMergeThreads >= d.N) return;   // the whole block
    // row_off is even, so the island's keys start on a 16-byte boundary:
    // 16-byte asynchronous copies, all in flight at once
    const unsigned long long *base = scratch + d.row_off;
    const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(isl_keys);
    for (int q = threadIdx.x; q < (d.N >> 1); q += blockDim.x)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sbase + 16u * (uint32_t)q), "l"(base + 2 * q)
                     : "memory");
    if ((d.N & 1) && threadIdx.x == 0) isl_keys[d.N - 1] = base[d.N - 1];
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    const int e = blockIdx.x * kRankMergeThreads + threadIdx.x;
    if (e >= d.N) return;
    const unsigned long long key = isl_keys[e];
    const int c = e / kRankChunk;
    int lo[kRankMaxChunks], hi[kRankMaxChunks];
#pragma unroll
    for (int c2 = 0; c2 < kRankMaxChunks; ++c2) {
        const int a0 = c2 * kRankChunk;
        lo[c2] = 0;
        hi[c2] = (c2 != c && a0 < d.N) ? min(kRankChunk, d.N - a0) : 0;
    }
    // a range of at most 2048 keys is empty after 12 halvings
#pragma unroll 1
    for (int step = 0; step < 12; ++step) {
#pragma unroll
        for (int c2 = 0; c2 < kRankMaxChunks; ++c2) {
            if (lo[c2] < hi[c2]) {
                const int mid = (lo[c2] + hi[c2]) >> 1;
                if (isl_keys[c2 * kRankChunk + mid] < key) lo[c2] = mid + 1;
                else hi[c2] = mid;
            }
        }
    }
    int rank = e - c * kRankChunk;
#pragma unroll
    for (int c2 = 0; c2 < kRankMaxChunks; ++c2) rank += lo[c2];
    d.order[rank] = (int32_t)(key & 0xFFFFFFFFu);
}

// One warp per migrated row: island i's t-th best onto island (i+1)'s t-th worst.
__global__ void k_ring_copy(const IslandDesc *desc, int I, const int32_t *cur, int ld, int total_rows,
                            const int32_t *gate, int gap, unsigned long long *mig)
{
    if (!migration_due(gate, gap)) return;
    const int lane = threadIdx.x & 31;
    // migrations received: island j takes the rows its ring predecessor sends
    if (blockIdx.x == 0 && (int)threadIdx.x < I) {
        const int j = threadIdx.x, i = (j + I - 1) % I;
        const int sent = desc[i].k_ring;
        mig[2 * j] += 1ull;
        mig[2 * j + 1] += (unsigned long long)sent;
    }
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total_rows; w += (gridDim.x * blockDim.x) >> 5) {
        int i = 0;
        while (i + 1 < I && desc[i + 1].ring_off <= w) ++i;
        const int t = w - desc[i].ring_off;
        const int j = (i + 1) % I;
        const IslandDesc &s = desc[i], &dd = desc[j];
        const int src = s.order[t], dst = dd.order[dd.N - 1 - t];
        if (!FFS_DCHECK(src >= 0 && src < s.N && dst >= 0 && dst < dd.N, kCheckMigrationRow)) continue;
        const int4 *from = reinterpret_cast<const int4 *>(s.pop[cur[i]] + (int64_t)src * ld);
        int4 *to = reinterpret_cast<int4 *>(dd.pop[cur[j]] + (int64_t)dst * ld);
        for (int k = lane; k < (ld >> 3); k += 32) to[k] = from[k];
        if (lane == 0) dd.ms[cur[j]][dst] = s.ms[cur[i]][src];
    }
}

// Penetration (Eq. (1)-(2) for makespans): one thread per pair (2q, 2q+1)
// decides the signed count; then one warp per candidate row copies.
__global__ void k_penetration(const IslandDesc *desc, int pairs, const int32_t *cur, long long theta_num,
                              long long theta_den, int32_t *counts, const int32_t *gate, int gap,
                              unsigned long long *mig)
{
    if (!migration_due(gate, gap)) return;
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= pairs) return;
    const IslandDesc &A = desc[2 * q], &B = desc[2 * q + 1];
    const long long cA = (uint32_t)A.ms[cur[2 * q]][A.order[0]];
    const long long cB = (uint32_t)B.ms[cur[2 * q + 1]][B.order[0]];
    long long cnt = 0;
    if (cA != cB) {
        const long long lo = cA < cB ? cA : cB, hi = cA < cB ? cB : cA;
        const long long N = A.N < B.N ? A.N : B.N;
        if ((hi - lo) * theta_den < theta_num * hi) cnt = ((hi - lo) * N) / hi;
        if (cA > cB) cnt = -cnt;
    }
    counts[q] = (int32_t)cnt;
    if (cnt != 0) {   // migrations received by the pair's other island
        const int di = cnt > 0 ? 2 * q + 1 : 2 * q;
        mig[2 * di] += 1ull;
        mig[2 * di + 1] += (unsigned long long)(cnt > 0 ? cnt : -cnt);
    }
}

__global__ void k_penetration_copy(const IslandDesc *desc, int pairs, const int32_t *cur, int ld,
                                   const int32_t *counts, int rows_per_pair, const int32_t *gate, int gap)
{
    if (!migration_due(gate, gap)) return;
    const int lane = threadIdx.x & 31;
    const int total = pairs * rows_per_pair;
    for (int w = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; w < total; w += (gridDim.x * blockDim.x) >> 5) {
        const int q = w / rows_per_pair, t = w - q * rows_per_pair;
        const int c = counts[q];
        const int k = c < 0 ? -c : c;
        if (t >= k) continue;
        const int si = c > 0 ? 2 * q : 2 * q + 1, di = c > 0 ? 2 * q + 1 : 2 * q;
        const IslandDesc &s = desc[si], &dd = desc[di];
        const int src = s.order[t], dst = dd.order[dd.N - 1 - t];
        if (!FFS_DCHECK(src >= 0 && src < s.N && dst >= 0 && dst < dd.N, kCheckMigrationRow)) continue;
        const int4 *from = reinterpret_cast<const int4 *>(s.pop[cur[si]] + (int64_t)src * ld);
        int4 *to = reinterpret_cast<int4 *>(dd.pop[cur[di]] + (int64_t)dst * ld);
        for (int kk = lane; kk < (ld >> 3); kk += 32) to[kk] = from[kk];
        if (lane == 0) dd.ms[cur[di]][dst] = s.ms[cur[si]][src];
    }
}

// Per-island metrics of the current generation, one block per island: the
// best, worst and sum of the valid makespans (a row with -1 is not
// counted), the valid rows, the best makespan any pass has seen so far
// (best_so_far[i], updated here) and the migrations the island has
// received (events, rows).  Record r of island i goes to
// out[((gen[i] % cap) * I + i) * kStatWords].
constexpr int kStatWords = 8;

__global__ void __launch_bounds__(256) k_island_stats(const IslandDesc *desc, int I, const int32_t *cur,
                                                     const int32_t *gen, int32_t *best_so_far,
                                                     const unsigned long long *mig, long long *out, int cap)
{
    __shared__ int s_lo[8], s_hi[8], s_cnt[8];
    __shared__ long long s_sum[8];
    const int i = blockIdx.x;
    const IslandDesc &D = desc[i];
    const int32_t *ms = D.ms[cur[i]];
    int lo = 0x7FFFFFFF, hi = -1, cnt = 0;
    long long sum = 0;
    for (int r = threadIdx.x; r < D.N; r += blockDim.x) {
        const int v = ms[r];
        if (v >= 0) {
            lo = min(lo, v);
            hi = max(hi, v);
            sum += v;
            ++cnt;
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xFFFFFFFFu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xFFFFFFFFu, hi, o));
        cnt += __shfl_xor_sync(0xFFFFFFFFu, cnt, o);
        sum += __shfl_xor_sync(0xFFFFFFFFu, sum, o);
    }
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_lo[warp] = lo;
        s_hi[warp] = hi;
        s_cnt[warp] = cnt;
        s_sum[warp] = sum;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            lo = min(lo, s_lo[w]);
            hi = max(hi, s_hi[w]);
            cnt += s_cnt[w];
            sum += s_sum[w];
        }
        const int bsf = cnt > 0 ? min(best_so_far[i], lo) : best_so_far[i];
        best_so_far[i] = bsf;
        long long *rec = out + ((long long)(gen[i] % cap) * I + i) * kStatWords;
        rec[0] = gen[i];
        rec[1] = cnt > 0 ? lo : -1;
        rec[2] = hi;
        rec[3] = sum;
        rec[4] = cnt;
        rec[5] = bsf == 0x7FFFFFFF ? -1 : bsf;
        rec[6] = (long long)mig[2 * i];
        rec[7] = (long long)mig[2 * i + 1];
    }
}

// The FFS_DEBUG_CHECKS build's validity pass over every island's current
// rows (blockIdx.y = island, one warp per row): warp_check_row.
__global__ void __launch_bounds__(128) k_check_islands(const IslandDesc *desc, const int32_t *cur, int n, int ld)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const int i = blockIdx.y, warp = threadIdx.x >> 5;
    const int words = (n + 31) >> 5;
    const IslandDesc &D = desc[i];
    for (int r = blockIdx.x * 4 + warp; r < D.N; r += gridDim.x * 4)
        warp_check_row(D.pop[cur[i]] + (int64_t)r * ld, n, D.ms[cur[i]][r], smem + warp * words);
}

// Advance the generation counter and flip the buffers of islands [i0, i1).
__global__ void k_advance(int32_t *cur, int32_t *gen, int i0, int i1)
{
    const int i = i0 + blockIdx.x * blockDim.x + threadIdx.x;
    if (i < i1) {
        cur[i] ^= 1;
        gen[i] += 1;
    }
}

}  // namespace fgpu

using namespace fgpu;

// Surrogate screening state attached to an islands handle.
struct SurrogateState {
    ffs_mlp *mlp = nullptr;
    ffs_surrogate_params sp{};
    int P = 0, ldx = 0, nfeat = 40;
    int xw = 0;                    // width of a candidate's scoring input row (the job positions)
    int cells_total = 0;           // cells of all cellular islands
    int16_t *cand = nullptr;       // [cells_total * K][ld]
    void *X = nullptr;             // BF16 [cells_total * K][xw]
    float *scores = nullptr;       // [cells_total * K]
    int32_t *chosen = nullptr;     // [cells_total]
    // screened pseudo pairs (screen_pseudo): every pair's candidate children,
    // their scoring rows and scores after the cellular ones in X and scores,
    // the picks
    int pairs_total = 0;           // pairs of all pseudo islands
    int pseudo_size = 0;           // rows of each pseudo island
    int16_t *cand_p = nullptr;     // [pairs_total * K * 2][ld]
    int32_t *chosen_p = nullptr;   // [pairs_total]
    std::vector<int> pseudo_islands;
    int16_t *ring_rows = nullptr;  // [ring_cap][ld]
    int32_t *ring_ms = nullptr;
    long long ring_cap = 0, ring_count = 0;
    float *inst_feat = nullptr;    // [nfeat]
    void *train_X = nullptr;       // BF16 [train_steps][train_batch][ldx]
    float *train_t = nullptr, *loss = nullptr;
    long long train_rounds = 0;
    std::vector<int> cell_islands;
    // device counters read by the kernels: [0] ring pairs appended, [1]
    // training batches drawn (host mirrors: ring_count, train_rounds), [2]
    // the ring count when the current generation began, [3] blocks of the
    // running gather that have finished (0 between launches)
    long long *d_ctr = nullptr;
    float *d_norm = nullptr;       // training-target standardisation (mean, 1 / std)
    // generations replayed from CUDA graphs, [warm][train][migration]: before /
    // after the warm-up, without / with a training round, without / with the
    // migration launches; the pseudo islands run
    // on `side` beside the screen, the training round on `side2` beside the
    // selection (after the forward pass, which reads the weights it updates)
    cudaGraphExec_t g_gen[2][2][2] = {};   // [warm][train][migration due]
    cudaStream_t side = nullptr, side2 = nullptr;
    cudaEvent_t fork_ev = nullptr, join_ev = nullptr, fork2_ev = nullptr, join2_ev = nullptr, fold_ev = nullptr;
    cudaEvent_t pcand_ev = nullptr, pfwd_ev = nullptr;   // screened pseudo: candidates built, scores written
    void drop_graphs()
    {
        for (auto &plane : g_gen)
            for (auto &row : plane)
                for (auto &g : row)
                    if (g) { cudaGraphExecDestroy(g); g = nullptr; }
    }
    ~SurrogateState()
    {
        drop_graphs();
        if (side) cudaStreamDestroy(side);
        if (side2) cudaStreamDestroy(side2);
        for (cudaEvent_t e : {fork_ev, join_ev, fork2_ev, join2_ev, fold_ev, pcand_ev, pfwd_ev})
            if (e) cudaEventDestroy(e);
    }
};

struct ffs_islands {
    SurrogateState *sur = nullptr;
    const ffs_instance *inst = nullptr;
    ffs_params prm{};
    int I = 0, ld = 0, rows = 0, cols = 0;
    std::vector<int> kind, size;
    std::vector<int> host_cur;
    std::vector<long long> host_gen;
    std::vector<IslandDesc> desc;
    IslandDesc *d_desc = nullptr;
    int32_t *d_cur = nullptr, *d_gen = nullptr, *d_counts = nullptr;
    unsigned long long *d_rank_keys = nullptr;   // [total_rows] sorted chunks of the ranking
    int total_rows = 0;
    void *d_scratch = nullptr;        // pseudo scratch (shared by the pseudo islands)
    int16_t *d_cell_children = nullptr;   // child rows of the cellular cells (fused generations)
    unsigned long long *d_decoded = nullptr;
    int32_t *d_best_so_far = nullptr;     // [I] lowest makespan a metrics pass has seen
    unsigned long long *d_mig = nullptr;  // [I][2] migrations received: events, rows
    long long *d_stats_now = nullptr;     // [I][kStatWords] the last ffs_islands_stats pass
    long long *d_hist = nullptr;          // [stats_cap][I][kStatWords] per-generation records
    int stats_cap = 0;
    long long stats_from = 0;             // generation of the oldest record kept
    int ring_rows = 0, max_N = 0, min_pair_rows = 0;
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph_all[2] = {nullptr, nullptr};   // [migration launches included]
    std::vector<void *> allocs;
};

namespace fgpu {

static IslandRef device_ref(const ffs_islands *S, int i)
{
    IslandRef r;
    memset(&r, 0, sizeof(r));
    r.pop[0] = S->desc[i].pop[0];
    r.pop[1] = S->desc[i].pop[1];
    r.ms[0] = S->desc[i].ms[0];
    r.ms[1] = S->desc[i].ms[1];
    r.dev_cur = S->d_cur + i;
    r.dev_gen = S->d_gen + i;
    r.island = (uint32_t)i;
    return r;
}

template <typename F, typename H>
static int screened_cellular_launch(ffs_islands *S, const std::vector<int> &sel, bool warm, bool use_copy,
                                    bool fold_ready, cudaStream_t st, F between, H after_scores);
static int screened_pseudo_candidates(ffs_islands *S, bool warm, cudaStream_t st);
static int screened_pseudo_scores(ffs_islands *S, bool warm, bool use_copy, cudaStream_t st);
static int screened_pseudo_finish(ffs_islands *S, cudaStream_t st);

// CTAs of the scoring forward's persistent GEMM while a training round runs
// beside it: the SMs left over take the round's kernels.
constexpr int kScreenForwardCtas = 96;

// One generation of the islands in `ids` (all of one kind): cellular islands
// in launches of up to kMaxBatch, pseudo islands likewise, one decode of all
// their children per launch.  With a surrogate attached, the cellular
// islands take the screened path.
static int islands_generation_launch(ffs_islands *S, const std::vector<int> &ids, cudaStream_t st,
                                     bool decode_only = false)
{
    const GaScalars g = scalars_of(&S->prm);
    if (!S->sur) {
        // both kinds present and each fits one batch: one fused decode launch
        std::vector<int> cel, pse;
        for (int i : ids) (S->kind[i] == 0 ? cel : pse).push_back(i);
        if (!cel.empty() && !pse.empty() && (int)cel.size() <= kMaxBatch && (int)pse.size() <= kMaxBatch &&
            S->d_cell_children) {
            IslandBatch cb, pb;
            memset(&cb, 0, sizeof(cb));
            memset(&pb, 0, sizeof(pb));
            cb.count = (int)cel.size();
            pb.count = (int)pse.size();
            for (int t = 0; t < cb.count; ++t) cb.ref[t] = device_ref(S, cel[t]);
            for (int t = 0; t < pb.count; ++t) pb.ref[t] = device_ref(S, pse[t]);
            return launch_step_fused(S->inst, g, cb, S->rows, S->cols, pb, S->size[pse[0]], S->ld, S->d_scratch,
                                     S->d_cell_children, S->prm.decode_chunk, S->prm.block_threads, S->d_decoded, st,
                                     decode_only);
        }
    }
    if (decode_only) return set_error(FFS_EINVAL, "the decode launch alone exists only for generations that decode both "
                                                  "kinds in one launch");
    for (int kind = 0; kind < 2; ++kind) {
        std::vector<int> sel;
        for (int i : ids)
            if (S->kind[i] == kind) sel.push_back(i);
        if (kind == 0 && S->sur && !sel.empty()) {
            // (single-island steps: no training round inside the generation)
            FFS_CUDA_TRY(cudaGetLastError());
            int rc = launch_sur_tick(S->sur->d_ctr, 2, -1, st);
            if (rc) return rc;
            rc = screened_cellular_launch(S, sel, S->host_gen[sel[0]] + 1 > S->sur->sp.warmup_generations, false,
                                          false, st, [](cudaStream_t) { return (int)FFS_OK; },
                                          [](cudaStream_t) { return (int)FFS_OK; });
            if (rc) return rc;
            continue;
        }
        if (kind == 1 && S->sur && S->sur->sp.screen_pseudo && !sel.empty()) {
            // a screened pseudo generation alone (every pseudo island together)
            if (sel.size() != S->sur->pseudo_islands.size())
                return set_error(FFS_EUNSUPPORTED, "screened pseudo islands step together");
            const bool warm = S->host_gen[sel[0]] + 1 > S->sur->sp.warmup_generations;
            int rc = screened_pseudo_candidates(S, warm, st);
            if (!rc && warm)
                rc = mlp_fold_bias(S->sur->mlp, false, S->sur->P, S->sur->inst_feat, S->sur->nfeat, st);
            if (!rc) rc = screened_pseudo_scores(S, warm, false, st);
            if (!rc) rc = screened_pseudo_finish(S, st);
            if (rc) return rc;
            continue;
        }
        for (size_t b0 = 0; b0 < sel.size(); b0 += kMaxBatch) {
            IslandBatch batch;
            memset(&batch, 0, sizeof(batch));
            batch.count = (int)std::min(sel.size() - b0, (size_t)kMaxBatch);
            for (int t = 0; t < batch.count; ++t) batch.ref[t] = device_ref(S, sel[b0 + t]);
            int rc = kind == 0
                         ? launch_cellular(S->inst, g, batch, S->rows, S->cols, S->ld, S->prm.decode_chunk,
                                           S->prm.block_threads, S->d_decoded, st)
                         : launch_pseudo(S->inst, g, batch, S->size[sel[b0]], S->ld, S->d_scratch,
                                         S->prm.decode_chunk, S->prm.block_threads, S->d_decoded, st);
            if (rc) return rc;
        }
    }
    return FFS_OK;
}

static int migrate_launch(ffs_islands *S, int mode, bool gated, cudaStream_t st)
{
    if (mode == FFS_MIG_NONE || S->I < 2) return FFS_OK;
    if (S->max_N > kMaxMigrationRows)
        return set_error(FFS_EUNSUPPORTED, "migration ranks islands of at most %d rows", kMaxMigrationRows);
    const int32_t *gate = gated ? S->d_gen : nullptr;
    const int gap = S->prm.migration_gap;
    const int chunks = (S->max_N + kRankChunk - 1) / kRankChunk;
    k_rank_chunks<<<dim3(chunks, S->I), kRankThreads, 0, st>>>(S->d_desc, S->d_cur, gate, gap, S->d_rank_keys);
    FFS_CUDA_TRY(cudaGetLastError());
    const size_t msmem = (size_t)S->max_N * 8;
    FFS_CUDA_TRY(cudaFuncSetAttribute(k_rank_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)msmem));
    k_rank_merge<<<dim3((S->max_N + kRankMergeThreads - 1) / kRankMergeThreads, S->I), kRankMergeThreads, msmem, st>>>(
        S->d_desc, gate, gap, S->d_rank_keys);
    FFS_CUDA_TRY(cudaGetLastError());
    if (mode == FFS_MIG_RING) {
        const int warps = S->ring_rows;
        int blocks = (warps * 32 + 255) / 256;
        if (blocks > 1024) blocks = 1024;
        k_ring_copy<<<blocks, 256, 0, st>>>(S->d_desc, S->I, S->d_cur, S->ld, S->ring_rows, gate, gap, S->d_mig);
        FFS_CUDA_TRY(cudaGetLastError());
    } else {
        const int pairs = S->I / 2;
        k_penetration<<<1, 64, 0, st>>>(S->d_desc, pairs, S->d_cur, S->prm.theta_num, S->prm.theta_den,
                                       S->d_counts, gate, gap, S->d_mig);
        FFS_CUDA_TRY(cudaGetLastError());
        int blocks = (pairs * S->min_pair_rows * 32 + 255) / 256;
        if (blocks > 2048) blocks = 2048;
        if (blocks < 1) blocks = 1;
        k_penetration_copy<<<blocks, 256, 0, st>>>(S->d_desc, pairs, S->d_cur, S->ld, S->d_counts,
                                                  S->min_pair_rows, gate, gap);
        FFS_CUDA_TRY(cudaGetLastError());
    }
    return FFS_OK;
}

// The metrics pass over every island (k_island_stats) into `out` (cap
// records per island).
static int stats_launch(ffs_islands *S, long long *out, int cap, cudaStream_t st)
{
    k_island_stats<<<S->I, 256, 0, st>>>(S->d_desc, S->I, S->d_cur, S->d_gen, S->d_best_so_far, S->d_mig, out, cap);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

// The end of every generation: the metrics record when recording is on, and
// in the FFS_DEBUG_CHECKS build the validity pass over every island's rows.
static int record_launch(ffs_islands *S, cudaStream_t st)
{
#ifdef FFS_DEBUG_CHECKS
    const int words = (S->inst->n + 31) >> 5;
    const int bx = std::min((S->max_N + 3) / 4, 1024);
    k_check_islands<<<dim3(bx, S->I), 128, 4 * words * 4, st>>>(S->d_desc, S->d_cur, S->inst->n, S->ld);
    FFS_CUDA_TRY(cudaGetLastError());
#endif
    return S->stats_cap > 0 ? stats_launch(S, S->d_hist, S->stats_cap, st) : FFS_OK;
}

// Screened generation of the cellular islands in `sel`: phase 1 builds every
// batch's candidates (with their network inputs when warm); `between` then
// runs (the wait for the training round); phase 2 scores each batch with the
// network (all scores 0 during the warm-up: candidate 0 is taken), decodes
// each cell's best-scored candidate exactly, replaces the cell iff better and
// appends the pair to the ring (the device ring counter advanced by the
// cells of each batch).
template <typename F, typename H>
static int screened_cellular_launch(ffs_islands *S, const std::vector<int> &sel, bool warm, bool use_copy,
                                    bool fold_ready, cudaStream_t st, F between, H after_scores)
{
    SurrogateState *R = S->sur;
    const GaScalars g = scalars_of(&S->prm);
    const int K = R->sp.candidates, cells = S->rows * S->cols;
    std::vector<IslandBatch> batches;
    for (size_t b0 = 0; b0 < sel.size(); b0 += kMaxBatch) {
        IslandBatch batch;
        memset(&batch, 0, sizeof(batch));
        batch.count = (int)std::min(sel.size() - b0, (size_t)kMaxBatch);
        for (int t = 0; t < batch.count; ++t) batch.ref[t] = device_ref(S, sel[b0 + t]);
        batches.push_back(batch);
    }
    int offset = 0;   // cells before this batch among the cellular islands
    for (const IslandBatch &batch : batches) {
        const int ncells = batch.count * cells;
        int16_t *cand = R->cand + (int64_t)offset * K * S->ld;
        // the candidates, and in warm generations their network inputs in the same launch
        void *X = static_cast<char *>(R->X) + (int64_t)offset * K * R->xw * 2;
        int rc = launch_sur_candidates(S->inst, g, batch, S->rows, S->cols, S->ld, K, cand, warm ? X : nullptr, R->xw,
                                       st);
        if (rc) return rc;
        offset += ncells;
    }
    int rc = between(st);
    if (rc) return rc;
    // layer 1's folded bias (unless `between` made it ready on another stream)
    if (warm && !fold_ready &&
        (rc = mlp_fold_bias(R->mlp, use_copy, R->P, R->inst_feat, R->nfeat, st)))
        return rc;
    // every batch's scores, then `after_scores` (more scoring on this
    // stream), then every batch's selection
    offset = 0;
    for (const IslandBatch &batch : batches) {
        const int ncells = batch.count * cells;
        float *scores = R->scores + (int64_t)offset * K;
        if (warm) {
            const void *X = static_cast<const char *>(R->X) + (int64_t)offset * K * R->xw * 2;
            rc = mlp_forward_folded(R->mlp, use_copy, X, R->xw, S->inst->n, R->P, R->inst_feat, R->nfeat, ncells * K,
                                    scores, use_copy ? kScreenForwardCtas : 0, st);
            if (rc) return rc;
        } else if ((rc = launch_fill_f32(scores, (int64_t)ncells * K, 0.0f, st))) {
            return rc;
        }
        offset += ncells;
    }
    if ((rc = after_scores(st))) return rc;
    offset = 0;
    for (const IslandBatch &batch : batches) {
        const int ncells = batch.count * cells;
        const int16_t *cand = R->cand + (int64_t)offset * K * S->ld;
        const float *scores = R->scores + (int64_t)offset * K;
        if ((rc = launch_sur_select(S->inst, g, batch, S->rows, S->cols, S->ld, K, cand, scores, R->chosen + offset,
                                    R->ring_rows, R->ring_ms, R->ring_cap, R->d_ctr, S->prm.decode_chunk,
                                    S->prm.block_threads, S->d_decoded, st)))
            return rc;
        if ((rc = launch_sur_tick(R->d_ctr, 0, ncells, st))) return rc;
        offset += ncells;
    }
    return FFS_OK;
}

// Screened pseudo islands (all of them, one batch): candidates on `st` into
// cand_p and, warm, their scoring rows after the cellular ones in X.
static IslandBatch pseudo_batch(const ffs_islands *S)
{
    IslandBatch b;
    memset(&b, 0, sizeof(b));
    b.count = (int)S->sur->pseudo_islands.size();
    for (int t = 0; t < b.count; ++t) b.ref[t] = device_ref(S, S->sur->pseudo_islands[t]);
    return b;
}

static int screened_pseudo_candidates(ffs_islands *S, bool warm, cudaStream_t st)
{
    SurrogateState *R = S->sur;
    const int K = R->sp.candidates;
    void *Xp = static_cast<char *>(R->X) + (int64_t)R->cells_total * K * R->xw * 2;
    return launch_sur_pseudo_candidates(S->inst, scalars_of(&S->prm), pseudo_batch(S), R->pseudo_size, S->ld, K,
                                        R->cand_p, warm ? Xp : nullptr, R->xw, st);
}

// Their scores (after the cellular ones): the forward pass over their rows
// (layer 1's folded bias computed before, in stream order), or zeros during
// the warm-up.
static int screened_pseudo_scores(ffs_islands *S, bool warm, bool use_copy, cudaStream_t st)
{
    SurrogateState *R = S->sur;
    const int K = R->sp.candidates;
    const int64_t rows = (int64_t)R->pairs_total * K * 2;
    float *sp = R->scores + (int64_t)R->cells_total * K;
    if (!warm) return launch_fill_f32(sp, rows, 0.0f, st);
    const void *Xp = static_cast<const char *>(R->X) + (int64_t)R->cells_total * K * R->xw * 2;
    return mlp_forward_folded(R->mlp, use_copy, Xp, R->xw, S->inst->n, R->P, R->inst_feat, R->nfeat, (int)rows, sp,
                              use_copy ? kScreenForwardCtas : 0, st);
}

// The picks, their exact decode and the replacement.
static int screened_pseudo_finish(ffs_islands *S, cudaStream_t st)
{
    SurrogateState *R = S->sur;
    const int K = R->sp.candidates;
    const float *sp = R->scores + (int64_t)R->cells_total * K;
    return launch_pseudo_screened(S->inst, scalars_of(&S->prm), pseudo_batch(S), R->pseudo_size, S->ld, K, R->cand_p,
                                  sp, R->chosen_p, S->d_scratch, S->prm.decode_chunk, S->prm.block_threads,
                                  S->d_decoded, st);
}

// One round of online training of the surrogate on pairs from the ring
// buffer: train_steps batches, each drawn with the device's batch counter.
static int surrogate_train_launch(ffs_islands *S, cudaStream_t st)
{
    SurrogateState *R = S->sur;
    // every step's batch in one launch (batch k drawn as the (ctr[1] + k)-th)
    const int B = R->sp.train_batch, steps = R->sp.train_steps;
    int rc = launch_sur_gather(R->ring_rows, R->ring_ms, R->ring_cap, R->cells_total, R->d_ctr, S->ld, S->prm.seed, B,
                               steps, R->train_t, R->d_norm, S->inst->n, R->P, R->inst_feat, R->nfeat, R->train_X,
                               R->ldx, st);
    if (rc) return rc;   // the gather also advanced the batch count ctr[1]
    for (int s = 0; s < steps; ++s) {
        const void *X = static_cast<const char *>(R->train_X) + (int64_t)s * B * R->ldx * 2;
        if ((rc = ffs_mlp_train_step(R->mlp, static_cast<const uint16_t *>(X), R->ldx, R->train_t + (int64_t)s * B, B,
                                     R->sp.lr, R->loss, st)))
            return rc;
    }
    return FFS_OK;
}

// One screened generation of every island: the ring-count snapshot (the
// pairs of the generations before this one), the pseudo islands on the side
// stream beside the cellular screen, and (train = true) the training round
// on the previous generations' pairs on the second side stream, beside the
// candidate building and joined before the forward pass that reads the
// updated weights -- or, with overlap, beside the whole screen, which then
// scores with a copy of the weights taken before the round starts (the
// round draws only pairs of earlier generations and the standardisation of
// the latest one, slots that this generation's picks do not overwrite while
// the ring holds two generations); then, everything joined, the generation
// advance and migration, as generation_all does.
static int screened_generation(ffs_islands *S, bool warm, bool train, bool migrate, cudaStream_t st)
{
    SurrogateState *R = S->sur;
    std::vector<int> cel, pse;
    for (int i = 0; i < S->I; ++i) (S->kind[i] == 0 ? cel : pse).push_back(i);
    const bool overlap = train && R->sp.overlap;
    int rc = launch_sur_tick(R->d_ctr, 2, -1, st);
    if (rc) return rc;
    if (overlap && warm && (rc = mlp_take_copy(R->mlp, st))) return rc;
    // screened pseudo islands: their candidates on the side stream now,
    // scored after the cellular candidates, then picked and decoded there
    const bool screen_pse = R->sp.screen_pseudo && !pse.empty();
    if (!pse.empty()) {
        NvtxRange r("ffs pseudo islands (side stream)");
        FFS_CUDA_TRY(cudaEventRecord(R->fork_ev, st));
        FFS_CUDA_TRY(cudaStreamWaitEvent(R->side, R->fork_ev, 0));
        if (screen_pse) {
            if ((rc = screened_pseudo_candidates(S, warm, R->side))) return rc;
            FFS_CUDA_TRY(cudaEventRecord(R->pcand_ev, R->side));
        } else if ((rc = islands_generation_launch(S, pse, R->side))) {
            return rc;
        }
    }
    // with overlap, the training stream first folds the copy's layer-1 bias
    // (beside the candidate building), then runs the round
    const bool fold_side = overlap && warm;
    if (train) {
        NvtxRange r("ffs surrogate training round (side stream)");
        FFS_CUDA_TRY(cudaEventRecord(R->fork2_ev, st));
        FFS_CUDA_TRY(cudaStreamWaitEvent(R->side2, R->fork2_ev, 0));
        if (fold_side) {
            if ((rc = mlp_fold_bias(R->mlp, true, R->P, R->inst_feat, R->nfeat, R->side2))) return rc;
            FFS_CUDA_TRY(cudaEventRecord(R->fold_ev, R->side2));
        }
        if ((rc = surrogate_train_launch(S, R->side2))) return rc;
        FFS_CUDA_TRY(cudaEventRecord(R->join2_ev, R->side2));
    }
    {
        NvtxRange r("ffs screened cellular islands: candidates, scores, select");
        rc = screened_cellular_launch(
            S, cel, warm, overlap, fold_side, st,
            [&](cudaStream_t cs) -> int {
                if (train && !overlap) FFS_CUDA_TRY(cudaStreamWaitEvent(cs, R->join2_ev, 0));
                if (fold_side) FFS_CUDA_TRY(cudaStreamWaitEvent(cs, R->fold_ev, 0));
                return FFS_OK;
            },
            [&](cudaStream_t cs) -> int {
                if (!screen_pse) return FFS_OK;
                // the pseudo candidates' scores on this stream (after the
                // cellular ones: one forward at a time), the rest on `side`
                FFS_CUDA_TRY(cudaStreamWaitEvent(cs, R->pcand_ev, 0));
                int r2 = screened_pseudo_scores(S, warm, overlap, cs);
                if (r2) return r2;
                FFS_CUDA_TRY(cudaEventRecord(R->pfwd_ev, cs));
                FFS_CUDA_TRY(cudaStreamWaitEvent(R->side, R->pfwd_ev, 0));
                return screened_pseudo_finish(S, R->side);
            });
        if (rc) return rc;
    }
    if (overlap) FFS_CUDA_TRY(cudaStreamWaitEvent(st, R->join2_ev, 0));
    if (!pse.empty()) {
        FFS_CUDA_TRY(cudaEventRecord(R->join_ev, R->side));
        FFS_CUDA_TRY(cudaStreamWaitEvent(st, R->join_ev, 0));
    }
    k_advance<<<(S->I + 63) / 64, 64, 0, st>>>(S->d_cur, S->d_gen, 0, S->I);
    FFS_CUDA_TRY(cudaGetLastError());
    if (migrate && S->prm.migration_gap > 0) {
        NvtxRange r("ffs migration (gated by the gap)");
        int rc = migrate_launch(S, S->prm.migration_mode, true, st);
        if (rc) return rc;
    }
    NvtxRange r("ffs metrics / checks");
    return record_launch(S, st);
}

// Capture `body` on the islands' capture stream into an executable graph.
template <typename F>
static int capture_graph(ffs_islands *S, cudaGraphExec_t *out, F body)
{
    if (!S->cap_stream) FFS_CUDA_TRY(cudaStreamCreateWithFlags(&S->cap_stream, cudaStreamNonBlocking));
    cudaGraph_t graph = nullptr;
    FFS_CUDA_TRY(cudaStreamBeginCapture(S->cap_stream, cudaStreamCaptureModeRelaxed));
    const int rc = body(S->cap_stream);
    cudaError_t e = cudaStreamEndCapture(S->cap_stream, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return set_error(FFS_ECUDA, "graph capture: %s", cudaGetErrorString(e));
    e = cudaGraphInstantiateWithFlags(out, graph, cudaGraphInstantiateFlagUseNodePriority);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        *out = nullptr;
        return set_error(FFS_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
    return FFS_OK;
}

// One generation of every island; `migrate`: this generation completes a
// multiple of the migration gap, so the (device-gated) migration launches
// are part of it.
static int generation_all(ffs_islands *S, bool migrate, cudaStream_t st)
{
    std::vector<int> all(S->I);
    for (int i = 0; i < S->I; ++i) all[i] = i;
    {
        NvtxRange r("ffs breed + decode + replace");
        int rc0 = islands_generation_launch(S, all, st);
        if (rc0) return rc0;
    }
    // flip to the new generation first: migration works on it
    k_advance<<<(S->I + 63) / 64, 64, 0, st>>>(S->d_cur, S->d_gen, 0, S->I);
    FFS_CUDA_TRY(cudaGetLastError());
    if (migrate && S->prm.migration_gap > 0) {
        NvtxRange r("ffs migration (gated by the gap)");
        int rc = migrate_launch(S, S->prm.migration_mode, true, st);
        if (rc) return rc;
    }
    NvtxRange r("ffs metrics / checks");
    return record_launch(S, st);
}

// Whether the generation about to run (all islands at the same count)
// completes a multiple of the migration gap: the host's choice of the
// generation graph with or without the migration launches, which check the
// same condition on the device.
static int migration_due_host(const ffs_islands *S)
{
    const long long G = S->host_gen[0] + 1;
    return S->prm.migration_mode != FFS_MIG_NONE && S->I >= 2 && S->prm.migration_gap > 0 &&
                   G % S->prm.migration_gap == 0
               ? 1 : 0;
}

}  // namespace fgpu

extern "C" {

int ffs_cellular_step(const ffs_instance *I, const ffs_params *prm, uint32_t island, uint32_t generation,
                      int32_t rows, int32_t cols, int32_t ld, const int16_t *pop_in, const int32_t *ms_in,
                      int16_t *pop_out, int32_t *ms_out, ffs_stream stream)
{
    clear_error();
    if (!I || !prm || !pop_in || !ms_in || !pop_out || !ms_out) return set_error(FFS_EINVAL, "NULL argument");
    if (rows < 1 || cols < 1 || (int64_t)rows * cols > (1 << 30)) return set_error(FFS_EINVAL, "bad torus %dx%d", rows, cols);
    if (pop_in == pop_out) return set_error(FFS_EINVAL, "pop_in and pop_out must differ");
    int rc = validate_rows(pop_in, ld, I->n);
    if (rc) return rc;
    if ((rc = validate_rows(pop_out, ld, I->n))) return rc;
    IslandBatch b;
    memset(&b, 0, sizeof(b));
    b.count = 1;
    IslandRef &r = b.ref[0];
    r.pop_in = pop_in; r.ms_in = ms_in; r.pop_out = pop_out; r.ms_out = ms_out;
    r.generation = generation;
    r.island = island;
    return launch_cellular(I, scalars_of(prm), b, rows, cols, ld, prm->decode_chunk, prm->block_threads, nullptr,
                           (cudaStream_t)stream);
}

int64_t ffs_pseudo_scratch_bytes(int32_t size, int32_t ld)
{
    if (size < 0 || ld < 0) return -1;
    return pseudo_scratch_bytes(size, ld);
}

int ffs_pseudo_step(const ffs_instance *I, const ffs_params *prm, uint32_t island, uint32_t generation,
                    int32_t size, int32_t ld, const int16_t *pop_in, const int32_t *ms_in, int16_t *pop_out,
                    int32_t *ms_out, void *scratch, ffs_stream stream)
{
    clear_error();
    if (!I || !prm || !pop_in || !ms_in || !pop_out || !ms_out || !scratch)
        return set_error(FFS_EINVAL, "NULL argument");
    if (size < 2 || (size & 1)) return set_error(FFS_EINVAL, "pseudo island size %d must be even and >= 2", size);
    if (pop_in == pop_out) return set_error(FFS_EINVAL, "pop_in and pop_out must differ");
    if (((uintptr_t)scratch & 255u) != 0) return set_error(FFS_EINVAL, "scratch must be 256-byte aligned");
    int rc = validate_rows(pop_in, ld, I->n);
    if (rc) return rc;
    if ((rc = validate_rows(pop_out, ld, I->n))) return rc;
    IslandBatch b;
    memset(&b, 0, sizeof(b));
    b.count = 1;
    IslandRef &r = b.ref[0];
    r.pop_in = pop_in; r.ms_in = ms_in; r.pop_out = pop_out; r.ms_out = ms_out;
    r.generation = generation;
    r.island = island;
    return launch_pseudo(I, scalars_of(prm), b, size, ld, scratch, prm->decode_chunk, prm->block_threads, nullptr,
                         (cudaStream_t)stream);
}

static void islands_free(ffs_islands *S)
{
    if (!S) return;
    delete S->sur;
    for (cudaGraphExec_t g : S->graph_all)
        if (g) cudaGraphExecDestroy(g);
    if (S->cap_stream) cudaStreamDestroy(S->cap_stream);
    for (void *p : S->allocs) cudaFree(p);
    if (S->d_hist) cudaFree(S->d_hist);
    delete S;
}

// Captured generation graphs include the metrics record or not: after the
// recording is switched, they are captured again.
static void drop_generation_graphs(ffs_islands *S)
{
    for (cudaGraphExec_t &g : S->graph_all)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    if (S->sur) S->sur->drop_graphs();
}

// The GA parameters' own limits (at creation and when a checkpoint brings
// them back).
static int check_ga_params(const ffs_params *prm)
{
    if (prm->migration_mode < FFS_MIG_NONE || prm->migration_mode > FFS_MIG_PENETRATION)
        return set_error(FFS_EINVAL, "migration_mode %d", prm->migration_mode);
    if (prm->ring_den <= 0 || prm->ring_num < 0 || prm->theta_den <= 0 || prm->theta_num < 0 ||
        prm->theta_num > prm->theta_den)
        return set_error(FFS_EINVAL, "migration fractions must be num >= 0, den > 0, theta <= 1");
    if (prm->migration_gap < 0) return set_error(FFS_EINVAL, "migration_gap %d < 0", prm->migration_gap);
    return FFS_OK;
}

int ffs_islands_create(const ffs_instance *inst, const ffs_params *prm, int32_t n_cellular, int32_t rows,
                       int32_t cols, int32_t n_pseudo, int32_t pseudo_size, ffs_stream stream, ffs_islands **out)
{
    clear_error();
    if (!inst || !prm || !out) return set_error(FFS_EINVAL, "NULL argument");
    *out = nullptr;
    if (n_cellular < 0 || n_pseudo < 0 || n_cellular + n_pseudo < 1 || n_cellular + n_pseudo > 4096)
        return set_error(FFS_EINVAL, "island counts %d + %d", n_cellular, n_pseudo);
    if (n_cellular > 0 && (rows < 1 || cols < 1 || (int64_t)rows * cols > kMaxMigrationRows * 64))
        return set_error(FFS_EINVAL, "bad torus %dx%d", rows, cols);
    if (n_pseudo > 0 && (pseudo_size < 2 || (pseudo_size & 1)))
        return set_error(FFS_EINVAL, "pseudo island size %d must be even and >= 2", pseudo_size);
    if (int rc = check_ga_params(prm)) return rc;
    ffs_islands *S = new ffs_islands();
    S->inst = inst;
    S->prm = *prm;
    S->rows = rows;
    S->cols = cols;
    S->ld = round_up(inst->n, 8);
    for (int q = 0; q < std::max(n_cellular, n_pseudo); ++q) {
        if (q < n_cellular) { S->kind.push_back(0); S->size.push_back(rows * cols); }
        if (q < n_pseudo) { S->kind.push_back(1); S->size.push_back(pseudo_size); }
    }
    S->I = (int)S->kind.size();
    S->host_cur.assign(S->I, 0);
    S->host_gen.assign(S->I, 0);
    S->desc.resize(S->I);
    cudaStream_t st = (cudaStream_t)stream;
    auto alloc = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) { (void)cudaGetLastError(); return nullptr; }
        S->allocs.push_back(p);
        return p;
    };
    int ring_off = 0, max_pseudo = 0;
    S->total_rows = 0;
    for (int i = 0; i < S->I; ++i) {
        const int N = S->size[i];
        S->max_N = std::max(S->max_N, N);
        IslandDesc &d = S->desc[i];
        memset(&d, 0, sizeof(d));
        d.N = N;
        d.row_off = S->total_rows;
        S->total_rows += N + (N & 1);   // keeps every island's keys 16-byte aligned
        d.kind = S->kind[i];
        for (int b = 0; b < 2; ++b) {
            d.pop[b] = (int16_t *)alloc((size_t)N * S->ld * 2);
            d.ms[b] = (int32_t *)alloc((size_t)N * 4);
        }
        d.order = (int32_t *)alloc((size_t)N * 4);
        if (!d.pop[0] || !d.pop[1] || !d.ms[0] || !d.ms[1] || !d.order) {
            islands_free(S);
            return set_error(FFS_ENOMEM, "island %d buffers", i);
        }
        if (S->kind[i] == 1) max_pseudo = std::max(max_pseudo, N);
    }
    if (S->I > 1 && prm->migration_mode != FFS_MIG_NONE && S->max_N > kMaxMigrationRows) {
        islands_free(S);
        return set_error(FFS_EUNSUPPORTED, "migration ranks islands of at most %d rows", kMaxMigrationRows);
    }
    for (int i = 0; i < S->I; ++i) {
        const int j = (i + 1) % S->I;
        const int nmin = std::min(S->size[i], S->size[j]);
        long long k = (long long)(prm->ring_num * (long long)nmin / prm->ring_den);
        if (k < 1) k = 1;
        if (2 * k > nmin) {
            islands_free(S);
            return set_error(FFS_EINVAL, "ring migration of %lld rows exceeds half of %d", k, nmin);
        }
        S->desc[i].k_ring = (int)k;
        S->desc[i].ring_off = ring_off;
        ring_off += (int)k;
    }
    S->ring_rows = ring_off;
    S->min_pair_rows = 0;
    for (int q = 0; q + 1 < S->I; q += 2) S->min_pair_rows = std::max(S->min_pair_rows, std::min(S->size[q], S->size[q + 1]));
    S->d_desc = (IslandDesc *)alloc(sizeof(IslandDesc) * S->I);
    S->d_cur = (int32_t *)alloc(4 * S->I);
    S->d_gen = (int32_t *)alloc(4 * S->I);
    S->d_counts = (int32_t *)alloc(4 * (S->I / 2 + 1));
    S->d_decoded = (unsigned long long *)alloc(8);
    S->d_rank_keys = (unsigned long long *)alloc((size_t)S->total_rows * 8);
    S->d_best_so_far = (int32_t *)alloc(4 * (size_t)S->I);
    S->d_mig = (unsigned long long *)alloc(16 * (size_t)S->I);
    S->d_stats_now = (long long *)alloc(8 * (size_t)kStatWords * S->I);
    int n_pseudo_islands = 0;
    for (int i = 0; i < S->I; ++i) n_pseudo_islands += S->kind[i] == 1;
    if (max_pseudo > 0)
        S->d_scratch = alloc((size_t)pseudo_scratch_bytes(max_pseudo, S->ld, std::min(n_pseudo_islands, kMaxBatch)));
    // child rows of the cellular cells, for generations of both kinds in one
    // decode launch (at most kMaxBatch islands of each kind)
    const int n_cellular_islands = S->I - n_pseudo_islands;
    const bool fused = n_cellular_islands > 0 && n_pseudo_islands > 0 && n_cellular_islands <= kMaxBatch &&
                       n_pseudo_islands <= kMaxBatch;
    if (fused) S->d_cell_children = (int16_t *)alloc((size_t)n_cellular_islands * S->rows * S->cols * S->ld * 2);
    if (!S->d_desc || !S->d_cur || !S->d_gen || !S->d_counts || !S->d_decoded || !S->d_rank_keys ||
        !S->d_best_so_far || !S->d_mig || !S->d_stats_now || (max_pseudo > 0 && !S->d_scratch) ||
        (fused && !S->d_cell_children)) {
        islands_free(S);
        return set_error(FFS_ENOMEM, "island state");
    }
    int rc = FFS_OK;
    if (cudaMemcpyAsync(S->d_desc, S->desc.data(), sizeof(IslandDesc) * S->I, cudaMemcpyHostToDevice, st) ||
        cudaMemsetAsync(S->d_cur, 0, 4 * S->I, st) || cudaMemsetAsync(S->d_gen, 0, 4 * S->I, st) ||
        cudaMemsetAsync(S->d_decoded, 0, 8, st) || cudaMemsetAsync(S->d_mig, 0, 16 * (size_t)S->I, st))
        rc = set_error(FFS_ECUDA, "island state initialisation");
    const std::vector<int32_t> none(S->I, 0x7FFFFFFF);   // no makespan seen yet
    if (!rc && cudaMemcpy(S->d_best_so_far, none.data(), 4 * (size_t)S->I, cudaMemcpyHostToDevice) != cudaSuccess)
        rc = set_error(FFS_ECUDA, "island state initialisation");
    for (int i = 0; i < S->I && !rc; ++i) {
        rc = launch_init(inst, prm->seed, (uint32_t)i, S->kind[i], S->size[i], S->ld, S->desc[i].pop[0], st);
        if (!rc)
            rc = launch_eval(inst, S->desc[i].pop[0], S->size[i], S->ld, S->desc[i].ms[0], nullptr, prm->decode_chunk,
                             prm->block_threads, nullptr, st);
    }
    if (!rc && cudaStreamSynchronize(st) != cudaSuccess) rc = set_error(FFS_ECUDA, "initialisation failed");
    if (rc) {
        islands_free(S);
        return rc;
    }
    *out = S;
    return FFS_OK;
}

void ffs_surrogate_params_default(ffs_surrogate_params *p)
{
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->candidates = 8;
    p->train_every = 1;
    p->train_steps = 2;
    p->train_batch = 1024;
    p->ring_capacity = 1 << 17;
    p->warmup_generations = 5;
    p->lr = 1e-3f;
    p->overlap = 1;
}

// The training round's stream.  With overlap it takes the device's highest
// stream priority (kept by the captured graphs' kernel nodes), so that its
// short kernels take SMs as soon as the screen's blocks free them.
static cudaError_t side2_create(cudaStream_t *st, bool high_priority)
{
    int least = 0, greatest = 0;
    if (!high_priority || cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess)
        return cudaStreamCreateWithFlags(st, cudaStreamNonBlocking);
    return cudaStreamCreateWithPriority(st, cudaStreamNonBlocking, greatest);
}

int ffs_islands_attach_surrogate(ffs_islands *S, ffs_mlp *mlp, const ffs_surrogate_params *sp, ffs_stream stream)
{
    clear_error();
    if (!S || !mlp || !sp) return set_error(FFS_EINVAL, "NULL argument");
    if (S->sur) return set_error(FFS_EINVAL, "a surrogate is already attached");
    if (sp->candidates < 1 || sp->candidates > 16) return set_error(FFS_EINVAL, "candidates %d outside [1, 16]", sp->candidates);
    if (sp->train_batch < 128 || sp->train_batch % 128) return set_error(FFS_EINVAL, "train_batch must be a multiple of 128");
    if (sp->train_steps < 0 || sp->train_every < 0 || sp->warmup_generations < 0)
        return set_error(FFS_EINVAL, "negative training schedule");
    const int n = S->inst->n, nfeat = 40;
    const int in_dim = mlp_in_dim(mlp);
    if (in_dim < n + nfeat) return set_error(FFS_EINVAL, "network input %d < n + %d", in_dim, nfeat);
    std::vector<int> cell_islands;
    for (int i = 0; i < S->I; ++i)
        if (S->kind[i] == 0) cell_islands.push_back(i);
    if (cell_islands.empty()) return set_error(FFS_EINVAL, "no cellular island to screen");
    const int cells_total = (int)cell_islands.size() * S->rows * S->cols;
    const int K = sp->candidates;
    if ((long long)cells_total * K > mlp_max_batch(mlp))
        return set_error(FFS_EINVAL, "network max_batch %d < %lld candidates per generation", mlp_max_batch(mlp),
                         (long long)cells_total * K);
    if (sp->train_batch > mlp_max_batch(mlp)) return set_error(FFS_EINVAL, "train_batch above the network's max_batch");
    if ((long long)sp->ring_capacity < (long long)cells_total + sp->train_batch)
        return set_error(FFS_EINVAL, "ring_capacity must hold one generation's pairs plus a training batch");
    if (sp->overlap != 0 && sp->overlap != 1) return set_error(FFS_EINVAL, "overlap must be 0 or 1");
    if (sp->screen_pseudo != 0 && sp->screen_pseudo != 1) return set_error(FFS_EINVAL, "screen_pseudo must be 0 or 1");
    std::vector<int> pseudo_islands;
    long long pairs_total = 0;
    for (int i = 0; i < S->I; ++i)
        if (S->kind[i] == 1) {
            pseudo_islands.push_back(i);
            pairs_total += S->size[i] / 2;
        }
    if (!sp->screen_pseudo) pairs_total = 0;
    if (sp->screen_pseudo && (int)pseudo_islands.size() > kMaxBatch)
        return set_error(FFS_EUNSUPPORTED, "screened pseudo islands: at most %d", kMaxBatch);
    if (pairs_total * K * 2 > mlp_max_batch(mlp))
        return set_error(FFS_EINVAL, "network max_batch %d < %lld pseudo candidate children per generation",
                         mlp_max_batch(mlp), pairs_total * K * 2);
    if (sp->overlap && (long long)sp->ring_capacity < 2LL * cells_total)
        return set_error(FFS_EINVAL, "with overlap, ring_capacity must hold two generations' pairs");
    if (sp->overlap) {
        int rc = mlp_enable_copy(mlp);
        if (rc) return rc;
    }
    SurrogateState *R = new SurrogateState();
    R->mlp = mlp;
    R->sp = *sp;
    R->P = in_dim - nfeat;
    R->ldx = ffs_mlp_input_width(mlp);
    R->nfeat = nfeat;
    R->cells_total = cells_total;
    R->cell_islands = cell_islands;
    R->ring_cap = sp->ring_capacity;
    auto alloc = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (cudaMalloc(&p, bytes) != cudaSuccess) { (void)cudaGetLastError(); return nullptr; }
        S->allocs.push_back(p);
        return p;
    };
    const size_t ncand = (size_t)cells_total * K, npc = (size_t)pairs_total * K * 2;
    R->cand = (int16_t *)alloc(ncand * S->ld * 2);
    R->xw = round_up(n, 8);
    R->X = alloc((ncand + npc) * R->xw * 2);
    R->scores = (float *)alloc((ncand + npc) * 4);
    R->pairs_total = (int)pairs_total;
    R->pseudo_islands = pseudo_islands;
    R->pseudo_size = pseudo_islands.empty() ? 0 : S->size[pseudo_islands[0]];
    if (npc) {
        R->cand_p = (int16_t *)alloc(npc * S->ld * 2);
        R->chosen_p = (int32_t *)alloc((size_t)pairs_total * 4);
    }
    R->chosen = (int32_t *)alloc((size_t)cells_total * 4);
    R->ring_rows = (int16_t *)alloc((size_t)R->ring_cap * S->ld * 2);
    R->ring_ms = (int32_t *)alloc((size_t)R->ring_cap * 4);
    R->inst_feat = (float *)alloc(nfeat * 4);
    const size_t train_rows = (size_t)sp->train_batch * std::max(sp->train_steps, 1);
    R->train_X = alloc(train_rows * R->ldx * 2);
    R->train_t = (float *)alloc(train_rows * 4);
    R->loss = (float *)alloc(4);
    R->d_ctr = (long long *)alloc(4 * sizeof(long long));
    R->d_norm = (float *)alloc(2 * sizeof(float));
    if (!R->cand || !R->X || !R->scores || !R->chosen || !R->ring_rows || !R->ring_ms || !R->inst_feat ||
        !R->train_X || !R->train_t || !R->loss || !R->d_ctr || !R->d_norm || (npc && (!R->cand_p || !R->chosen_p))) {
        delete R;
        return set_error(FFS_ENOMEM, "surrogate buffers");
    }
    // instance summary features (host): per stage s < 12 (M_s/10, mean p/99, load/(M_s LB)), n/500, S/20, LB/sum p
    const ffs_instance *I = S->inst;
    std::vector<double> load(I->S, 0.0), job(I->n, 0.0);
    for (int j = 0; j < I->n; ++j)
        for (int s = 0; s < I->S; ++s) {
            const double p = I->host_p[(size_t)j * I->S + s];
            load[s] += p;
            job[j] += p;
        }
    double lb = 0.0, total = 0.0;
    for (int j = 0; j < I->n; ++j) lb = std::max(lb, job[j]);
    for (int s = 0; s < I->S; ++s) {
        lb = std::max(lb, std::ceil(load[s] / I->host_M[s]));
        total += load[s];
    }
    std::vector<float> f(nfeat, 0.0f);
    for (int s = 0; s < std::min(I->S, 12); ++s) {
        f[3 * s] = (float)(I->host_M[s] / 10.0);
        f[3 * s + 1] = (float)(load[s] / I->n / 99.0);
        f[3 * s + 2] = (float)(load[s] / (I->host_M[s] * lb));
    }
    f[36] = (float)(I->n / 500.0);
    f[37] = (float)(I->S / 20.0);
    f[38] = (float)(lb / total);
    if (cudaMemcpy(R->inst_feat, f.data(), nfeat * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(R->d_ctr, 0, 4 * sizeof(long long)) != cudaSuccess ||
        cudaStreamCreateWithFlags(&R->side, cudaStreamNonBlocking) != cudaSuccess ||
        side2_create(&R->side2, sp->overlap != 0) != cudaSuccess ||
        cudaEventCreateWithFlags(&R->fork_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&R->join_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&R->fork2_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&R->join2_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&R->fold_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&R->pcand_ev, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&R->pfwd_ev, cudaEventDisableTiming) != cudaSuccess) {
        (void)cudaGetLastError();
        delete R;
        return set_error(FFS_ECUDA, "surrogate state initialisation");
    }
    (void)stream;
    S->sur = R;
    for (cudaGraphExec_t &g : S->graph_all)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    return FFS_OK;
}

int ffs_islands_surrogate_last(const ffs_islands *S, float *scores, int32_t *chosen, float *loss, int64_t *pairs,
                               int16_t *candidates, int32_t ld_out, ffs_stream stream)
{
    clear_error();
    if (!S || !S->sur) return set_error(FFS_EINVAL, "no surrogate attached");
    const SurrogateState *R = S->sur;
    cudaStream_t st = (cudaStream_t)stream;
    if (scores)
        FFS_CUDA_TRY(cudaMemcpyAsync(scores, R->scores, (size_t)R->cells_total * R->sp.candidates * 4, cudaMemcpyDefault, st));
    if (chosen) FFS_CUDA_TRY(cudaMemcpyAsync(chosen, R->chosen, (size_t)R->cells_total * 4, cudaMemcpyDefault, st));
    if (loss) FFS_CUDA_TRY(cudaMemcpyAsync(loss, R->loss, 4, cudaMemcpyDefault, st));
    if (candidates) {
        if (ld_out < S->inst->n) return set_error(FFS_EINVAL, "ld_out %d < n %d", ld_out, S->inst->n);
        FFS_CUDA_TRY(cudaMemcpy2DAsync(candidates, (size_t)ld_out * 2, R->cand, (size_t)S->ld * 2, (size_t)S->inst->n * 2,
                                       (size_t)R->cells_total * R->sp.candidates, cudaMemcpyDefault, st));
    }
    if (pairs) *pairs = R->ring_count;
    return FFS_OK;
}

int ffs_islands_surrogate_last_pseudo(const ffs_islands *S, float *scores, int32_t *chosen, int16_t *candidates,
                                      int32_t ld_out, ffs_stream stream)
{
    clear_error();
    if (!S || !S->sur) return set_error(FFS_EINVAL, "no surrogate attached");
    const SurrogateState *R = S->sur;
    if (!R->sp.screen_pseudo || !R->pairs_total) return set_error(FFS_EINVAL, "no screened pseudo islands");
    cudaStream_t st = (cudaStream_t)stream;
    const size_t rows = (size_t)R->pairs_total * R->sp.candidates * 2;
    if (scores)
        FFS_CUDA_TRY(cudaMemcpyAsync(scores, R->scores + (size_t)R->cells_total * R->sp.candidates, rows * 4,
                                     cudaMemcpyDefault, st));
    if (chosen) FFS_CUDA_TRY(cudaMemcpyAsync(chosen, R->chosen_p, (size_t)R->pairs_total * 4, cudaMemcpyDefault, st));
    if (candidates) {
        if (ld_out < S->inst->n) return set_error(FFS_EINVAL, "ld_out %d < n %d", ld_out, S->inst->n);
        FFS_CUDA_TRY(cudaMemcpy2DAsync(candidates, (size_t)ld_out * 2, R->cand_p, (size_t)S->ld * 2,
                                       (size_t)S->inst->n * 2, rows, cudaMemcpyDefault, st));
    }
    return FFS_OK;
}

int ffs_islands_set_generation(ffs_islands *S, int64_t generation)
{
    clear_error();
    if (!S) return set_error(FFS_EINVAL, "NULL islands");
    if (generation < 0 || generation > 0x7FFFFFFF) return set_error(FFS_EINVAL, "generation %lld", (long long)generation);
    std::vector<int32_t> gen(S->I, (int32_t)generation);
    FFS_CUDA_TRY(cudaMemcpy(S->d_gen, gen.data(), 4 * S->I, cudaMemcpyHostToDevice));
    for (int i = 0; i < S->I; ++i) S->host_gen[i] = generation;
    return FFS_OK;
}

int ffs_islands_dry_run(ffs_islands *S, int32_t kind, ffs_stream stream)
{
    clear_error();
    if (!S) return set_error(FFS_EINVAL, "NULL islands");
    if (S->sur) return set_error(FFS_EINVAL, "not with a surrogate attached");
    if (kind < 0 || kind > 3) return set_error(FFS_EINVAL, "kind %d", kind);
    std::vector<int> ids;
    for (int i = 0; i < S->I; ++i)
        if (kind >= 2 || S->kind[i] == kind) ids.push_back(i);
    unsigned long long *saved = S->d_decoded;
    S->d_decoded = nullptr;
    const int rc = islands_generation_launch(S, ids, (cudaStream_t)stream, kind == 3);
    S->d_decoded = saved;
    return rc;
}

int ffs_islands_autotune(ffs_islands *S, int32_t repeats, ffs_stream stream, int32_t *threads_out, int32_t *chunk_out,
                         float *best_ms)
{
    clear_error();
    if (!S) return set_error(FFS_EINVAL, "NULL islands");
    if (S->sur) return set_error(FFS_EINVAL, "autotune before attaching a surrogate (its ring would record the timing runs)");
    if (repeats < 1) repeats = 1;
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int> all(S->I);
    for (int i = 0; i < S->I; ++i) all[i] = i;
    cudaEvent_t e0, e1;
    FFS_CUDA_TRY(cudaEventCreate(&e0));
    FFS_CUDA_TRY(cudaEventCreate(&e1));
    const ffs_params saved = S->prm;
    unsigned long long *saved_counter = S->d_decoded;
    S->d_decoded = nullptr;   // the timing runs are not counted
    float best = -1.0f;
    int bestT = 0, bestB = 0, bestV = 1;
    int rc = FFS_OK;
    // 320 .. 448 threads are in the list for their balance: warp work items
    // are whole decodes, and the last wave of a launch is as long as one item
    const int Ts[7] = {64, 128, 256, 320, 384, 448, 512};
    const int Bs[10] = {8, 16, 32, 48, 64, 96, 104, 112, 128, 0};
    for (int vi = 1; vi <= kMaxVariant && !rc; ++vi)
    for (int ti = 0; ti < 7 && !rc; ++ti) {
        for (int bi = 0; bi < 10 && !rc; ++bi) {
            const int B = Bs[bi] == 0 ? round_up(S->inst->n, 8) : Bs[bi];
            if (Bs[bi] != 0 && B >= S->inst->n) continue;
            Plan p;
            if (plan_decode(S->inst, cellular_kernel(), B, Ts[ti], mark_words(S->inst->n), &p, vi)) continue;
            S->prm.decode_chunk = B;
            S->prm.block_threads = Ts[ti];
            S->prm.decode_variant = vi;
            // one untimed run, then the timed ones; they only rewrite the next-generation buffers
            if ((rc = islands_generation_launch(S, all, st))) break;
            float fastest = -1.0f;   // the fastest of the timed runs: the least disturbed
            for (int r = 0; r < repeats && !rc; ++r) {
                cudaEventRecord(e0, st);
                rc = islands_generation_launch(S, all, st);
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
                bestB = B;
                bestV = vi;
            }
        }
    }
    (void)cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    S->d_decoded = saved_counter;
    S->prm = saved;
    if (rc) return rc;
    if (best < 0.0f) return set_error(FFS_EUNSUPPORTED, "no launch shape could be timed");
    S->prm.decode_chunk = bestB;
    S->prm.block_threads = bestT;
    S->prm.decode_variant = bestV;
    for (cudaGraphExec_t &g : S->graph_all)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    if (threads_out) *threads_out = bestT;
    if (chunk_out) *chunk_out = bestB;
    if (best_ms) *best_ms = best;
    return FFS_OK;
}

int ffs_islands_params(const ffs_islands *S, ffs_params *out)
{
    clear_error();
    if (!S || !out) return set_error(FFS_EINVAL, "NULL argument");
    *out = S->prm;
    return FFS_OK;
}

int ffs_islands_destroy(ffs_islands *S)
{
    islands_free(S);
    return FFS_OK;
}

int ffs_islands_info(const ffs_islands *S, int32_t *n_islands, int32_t *ld, int64_t *generation, int32_t *sizes,
                     int32_t *kinds)
{
    clear_error();
    if (!S) return set_error(FFS_EINVAL, "NULL islands");
    if (n_islands) *n_islands = S->I;
    if (ld) *ld = S->ld;
    if (generation) *generation = S->host_gen.empty() ? 0 : S->host_gen[0];
    for (int i = 0; i < S->I; ++i) {
        if (sizes) sizes[i] = S->size[i];
        if (kinds) kinds[i] = S->kind[i];
    }
    return FFS_OK;
}

int ffs_island_step(ffs_islands *S, int32_t island, int32_t n_generations, ffs_stream stream)
{
    clear_error();
    if (!S) return set_error(FFS_EINVAL, "NULL islands");
    if (island < -1 || island >= S->I) return set_error(FFS_EINVAL, "island %d outside [-1, %d)", island, S->I);
    if (n_generations < 0) return set_error(FFS_EINVAL, "n_generations %d < 0", n_generations);
    if (n_generations == 0) return FFS_OK;
    cudaStream_t st = (cudaStream_t)stream;
    NvtxRange call("ffs_island_step");
    if (island >= 0) {
        for (int g = 0; g < n_generations; ++g) {
            NvtxRange gen("ffs generation (one island)");
            int rc = islands_generation_launch(S, std::vector<int>{island}, st);
            if (rc) return rc;
            k_advance<<<1, 32, 0, st>>>(S->d_cur, S->d_gen, island, island + 1);
            FFS_CUDA_TRY(cudaGetLastError());
            if ((rc = record_launch(S, st))) return rc;
            S->host_cur[island] ^= 1;
            S->host_gen[island] += 1;
            if (S->sur && S->kind[island] == 0) S->sur->ring_count += (long long)S->rows * S->cols;
        }
        return FFS_OK;
    }
    for (int i = 1; i < S->I; ++i)
        if (S->host_gen[i] != S->host_gen[0])
            return set_error(FFS_EINVAL, "islands were stepped separately; generation counts differ");
    if (S->sur) {
        // screened generations and training rounds, each replayed from its
        // CUDA graph; the kernels read the ring and batch counters on the
        // device, the host keeps mirrors to decide warm-up and training
        SurrogateState *R = S->sur;
        for (int g = 0; g < n_generations; ++g) {
            const long long G = S->host_gen[0] + 1;   // the generation about to run
            const int warm = G > R->sp.warmup_generations ? 1 : 0;
            // the training round after every train_every-th generation runs at the start
            // of the next one, on the pairs of the generations before it (at least a batch)
            const int train = (R->sp.train_every > 0 && R->sp.train_steps > 0 && G >= 2 &&
                               (G - 1) % R->sp.train_every == 0 &&
                               std::min(R->ring_count, R->ring_cap - R->cells_total) >= R->sp.train_batch)
                                  ? 1 : 0;
            const int mig = migration_due_host(S);
            NvtxRange gen(train ? "ffs screened generation + training round" : "ffs screened generation");
            if (eager_generations()) {
                int rc = screened_generation(S, warm != 0, train != 0, mig != 0, st);
                if (rc) return rc;
            } else {
                cudaGraphExec_t &ge = R->g_gen[warm][train][mig];
                if (!ge) {
                    int rc = capture_graph(S, &ge, [&](cudaStream_t cs) {
                        return screened_generation(S, warm != 0, train != 0, mig != 0, cs);
                    });
                    if (rc) return rc;
                }
                FFS_CUDA_TRY(cudaGraphLaunch(ge, st));
            }
            for (int i = 0; i < S->I; ++i) {
                S->host_cur[i] ^= 1;
                S->host_gen[i] += 1;
            }
            R->ring_count += R->cells_total;
            if (train) R->train_rounds += 1;
        }
        return FFS_OK;
    }
    if (eager_generations()) {
        for (int g = 0; g < n_generations; ++g) {
            NvtxRange gen("ffs generation");
            int rc = generation_all(S, migration_due_host(S) != 0, st);
            if (rc) return rc;
            for (int i = 0; i < S->I; ++i) {
                S->host_cur[i] ^= 1;
                S->host_gen[i] += 1;
            }
        }
        return FFS_OK;
    }
    // two graphs: the generation with and without the migration launches
    for (int g = 0; g < n_generations; ++g) {
        const int mig = migration_due_host(S);
        cudaGraphExec_t &ge = S->graph_all[mig];
        if (!ge) {
            NvtxRange cap("ffs capture of the generation graph");
            int rc = capture_graph(S, &ge, [&](cudaStream_t cs) { return generation_all(S, mig != 0, cs); });
            if (rc) return rc;
        }
        NvtxRange gen("ffs generation (graph)");
        FFS_CUDA_TRY(cudaGraphLaunch(ge, st));
        for (int i = 0; i < S->I; ++i) {
            S->host_cur[i] ^= 1;
            S->host_gen[i] += 1;
        }
    }
    return FFS_OK;
}

int ffs_migrate(ffs_islands *S, int32_t mode, ffs_stream stream)
{
    clear_error();
    NvtxRange call("ffs_migrate");
    if (!S) return set_error(FFS_EINVAL, "NULL islands");
    if (mode < FFS_MIG_NONE || mode > FFS_MIG_PENETRATION) return set_error(FFS_EINVAL, "mode %d", mode);
    return migrate_launch(S, mode, false, (cudaStream_t)stream);
}

int ffs_islands_get(const ffs_islands *S, int32_t island, int16_t *pop, int32_t ld_out, int32_t *ms, ffs_stream stream)
{
    clear_error();
    if (!S) return set_error(FFS_EINVAL, "NULL islands");
    if (island < 0 || island >= S->I) return set_error(FFS_EINVAL, "island %d", island);
    const int c = S->host_cur[island], N = S->size[island], n = S->inst->n;
    cudaStream_t st = (cudaStream_t)stream;
    if (pop) {
        if (ld_out < n) return set_error(FFS_EINVAL, "ld_out %d < n %d", ld_out, n);
        if (ld_out == S->ld)   // same row stride: one contiguous copy (padding genes included)
            FFS_CUDA_TRY(cudaMemcpyAsync(pop, S->desc[island].pop[c], (size_t)N * S->ld * 2, cudaMemcpyDefault, st));
        else
            FFS_CUDA_TRY(cudaMemcpy2DAsync(pop, (size_t)ld_out * 2, S->desc[island].pop[c], (size_t)S->ld * 2,
                                           (size_t)n * 2, N, cudaMemcpyDefault, st));
    }
    if (ms) FFS_CUDA_TRY(cudaMemcpyAsync(ms, S->desc[island].ms[c], (size_t)N * 4, cudaMemcpyDefault, st));
    return FFS_OK;
}

int ffs_islands_set(ffs_islands *S, int32_t island, const int16_t *pop, int32_t ld_in, const int32_t *ms,
                    ffs_stream stream)
{
    clear_error();
    if (!S) return set_error(FFS_EINVAL, "NULL islands");
    if (island < 0 || island >= S->I) return set_error(FFS_EINVAL, "island %d", island);
    const int c = S->host_cur[island], N = S->size[island], n = S->inst->n;
    cudaStream_t st = (cudaStream_t)stream;
    if (pop) {
        if (ld_in < n) return set_error(FFS_EINVAL, "ld_in %d < n %d", ld_in, n);
        if (ld_in == S->ld)   // same row stride: one contiguous copy (padding genes included)
            FFS_CUDA_TRY(cudaMemcpyAsync(S->desc[island].pop[c], pop, (size_t)N * S->ld * 2, cudaMemcpyDefault, st));
        else
            FFS_CUDA_TRY(cudaMemcpy2DAsync(S->desc[island].pop[c], (size_t)S->ld * 2, pop, (size_t)ld_in * 2,
                                           (size_t)n * 2, N, cudaMemcpyDefault, st));
    }
    if (ms) FFS_CUDA_TRY(cudaMemcpyAsync(S->desc[island].ms[c], ms, (size_t)N * 4, cudaMemcpyDefault, st));
    return FFS_OK;
}

int ffs_islands_get_all(const ffs_islands *S, int16_t *pop, int32_t ld_out, int32_t *ms, ffs_stream stream)
{
    clear_error();
    if (!S) return set_error(FFS_EINVAL, "NULL islands");
    int64_t row = 0;
    for (int i = 0; i < S->I; ++i) {
        const int rc = ffs_islands_get(S, i, pop ? pop + row * ld_out : nullptr, ld_out, ms ? ms + row : nullptr,
                                       stream);
        if (rc) return rc;
        row += S->size[i];
    }
    return FFS_OK;
}

int ffs_islands_set_all(ffs_islands *S, const int16_t *pop, int32_t ld_in, const int32_t *ms, ffs_stream stream)
{
    clear_error();
    if (!S) return set_error(FFS_EINVAL, "NULL islands");
    int64_t row = 0;
    for (int i = 0; i < S->I; ++i) {
        const int rc = ffs_islands_set(S, i, pop ? pop + row * ld_in : nullptr, ld_in, ms ? ms + row : nullptr,
                                       stream);
        if (rc) return rc;
        row += S->size[i];
    }
    return FFS_OK;
}

int ffs_islands_best(const ffs_islands *S, int32_t *best_ms, int32_t *best_island, int32_t *best_row,
                     ffs_stream stream)
{
    clear_error();
    if (!S) return set_error(FFS_EINVAL, "NULL islands");
    cudaStream_t st = (cudaStream_t)stream;
    int32_t bm = -1, bi = -1, br = -1;
    std::vector<int32_t> h;
    for (int i = 0; i < S->I; ++i) {
        h.resize(S->size[i]);
        FFS_CUDA_TRY(cudaMemcpyAsync(h.data(), S->desc[i].ms[S->host_cur[i]], h.size() * 4, cudaMemcpyDeviceToHost, st));
        FFS_CUDA_TRY(cudaStreamSynchronize(st));
        for (int r = 0; r < S->size[i]; ++r)
            if (h[r] >= 0 && (bm < 0 || h[r] < bm)) { bm = h[r]; bi = i; br = r; }
    }
    if (best_ms) *best_ms = bm;
    if (best_island) *best_island = bi;
    if (best_row) *best_row = br;
    return FFS_OK;
}

int ffs_islands_stats(ffs_islands *S, int64_t *out, ffs_stream stream)
{
    clear_error();
    if (!S || !out) return set_error(FFS_EINVAL, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    int rc = stats_launch(S, S->d_stats_now, 1, st);
    if (rc) return rc;
    FFS_CUDA_TRY(cudaMemcpyAsync(out, S->d_stats_now, 8 * (size_t)kStatWords * S->I, cudaMemcpyDeviceToHost, st));
    FFS_CUDA_TRY(cudaStreamSynchronize(st));
    return FFS_OK;
}

int ffs_islands_record_stats(ffs_islands *S, int32_t capacity, ffs_stream stream)
{
    clear_error();
    if (!S) return set_error(FFS_EINVAL, "NULL islands");
    if (capacity < 0 || capacity > (1 << 24)) return set_error(FFS_EINVAL, "capacity %d outside [0, 2^24]", capacity);
    for (int i = 1; i < S->I; ++i)
        if (S->host_gen[i] != S->host_gen[0])
            return set_error(FFS_EINVAL, "islands were stepped separately; generation counts differ");
    cudaStream_t st = (cudaStream_t)stream;
    FFS_CUDA_TRY(cudaStreamSynchronize(st));
    if (S->d_hist) {
        FFS_CUDA_TRY(cudaFree(S->d_hist));
        S->d_hist = nullptr;
    }
    S->stats_cap = 0;
    drop_generation_graphs(S);
    if (capacity == 0) return FFS_OK;
    if (cudaMalloc(&S->d_hist, 8 * (size_t)kStatWords * S->I * capacity) != cudaSuccess) {
        (void)cudaGetLastError();
        S->d_hist = nullptr;
        return set_error(FFS_ENOMEM, "metrics history of %d generations", capacity);
    }
    S->stats_cap = capacity;
    S->stats_from = S->host_gen[0];
    return record_launch(S, st);   // the current generation is the first record
}

int ffs_islands_stats_history(const ffs_islands *S, int64_t *out, int32_t max_records, int32_t *count,
                              ffs_stream stream)
{
    clear_error();
    if (!S || !count) return set_error(FFS_EINVAL, "NULL argument");
    *count = 0;
    if (!S->stats_cap) return FFS_OK;
    for (int i = 1; i < S->I; ++i)
        if (S->host_gen[i] != S->host_gen[0])
            return set_error(FFS_EINVAL, "islands were stepped separately; generation counts differ");
    const long long G = S->host_gen[0];
    const long long first = std::max(S->stats_from, G - S->stats_cap + 1);
    const int n = (int)(G - first + 1);
    *count = n;
    if (!out) return FFS_OK;
    if (max_records < n) return set_error(FFS_EINVAL, "max_records %d < %d records kept", max_records, n);
    cudaStream_t st = (cudaStream_t)stream;
    // the kept records are slots first % cap .. G % cap of the ring: one copy,
    // or two where the range wraps
    const long long per = (long long)kStatWords * S->I;   // words of one generation, every island
    const long long s0 = first % S->stats_cap, s1 = G % S->stats_cap;
    const long long a = s0 <= s1 ? n : S->stats_cap - s0;
    FFS_CUDA_TRY(cudaMemcpyAsync(out, S->d_hist + s0 * per, (size_t)(a * per) * 8, cudaMemcpyDeviceToHost, st));
    if (a < n)
        FFS_CUDA_TRY(cudaMemcpyAsync(out + a * per, S->d_hist, (size_t)((n - a) * per) * 8, cudaMemcpyDeviceToHost, st));
    FFS_CUDA_TRY(cudaStreamSynchronize(st));
    return FFS_OK;
}

int ffs_islands_decoded(const ffs_islands *S, int64_t *count, ffs_stream stream)
{
    clear_error();
    if (!S || !count) return set_error(FFS_EINVAL, "NULL argument");
    unsigned long long v = 0;
    FFS_CUDA_TRY(cudaMemcpyAsync(&v, S->d_decoded, 8, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    FFS_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    *count = (int64_t)v;
    return FFS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Checkpoint / resume of an islands handle.  Blob (host memory), every
// section padded to 16 bytes:
//   IslandsBlobHeader; per island (kind, size, generation);
//   per island its current rows [size][ld] int16 and makespans [size] int32;
//   with a surrogate attached: SurrogateBlob, the filled ring slots' rows
//   [valid][ld] and makespans [valid], and the network's state (parameters,
//   Adam moments and step count).
// ---------------------------------------------------------------------------
namespace fgpu {

struct IslandsBlobHeader {
    uint32_t magic, version;
    int32_t I, ld, n, has_surrogate;
    uint64_t fingerprint;
    int64_t decoded;
    int64_t bytes;       // the blob's length
    uint64_t checksum;   // blob_checksum of the whole blob, this field taken as zero
    ffs_params prm;
};
struct IslandBlobEntry {
    int32_t kind, size;
    int64_t generation;
    int32_t best_so_far, pad;
    int64_t mig_events, mig_rows;
};
struct SurrogateBlob {
    int32_t candidates, pad;
    int64_t ring_cap, ring_count, train_rounds, valid;
};
constexpr uint32_t kIslandsBlobMagic = 0x49534646u, kIslandsBlobVersion = 3;

static int64_t r16(int64_t b) { return (b + 15) / 16 * 16; }

static int64_t islands_blob_bytes(const ffs_islands *S)
{
    int64_t b = r16(sizeof(IslandsBlobHeader)) + r16((int64_t)S->I * sizeof(IslandBlobEntry));
    for (int i = 0; i < S->I; ++i) b += r16((int64_t)S->size[i] * S->ld * 2) + r16((int64_t)S->size[i] * 4);
    if (S->sur) {
        const SurrogateState *R = S->sur;
        const int64_t valid = std::min(R->ring_count, R->ring_cap);
        b += r16(sizeof(SurrogateBlob)) + r16(valid * S->ld * 2) + r16(valid * 4) + r16(mlp_state_bytes(R->mlp));
    }
    return b;
}

}  // namespace fgpu

extern "C" {

int64_t ffs_checkpoint_bytes(const ffs_islands *S) { return S ? islands_blob_bytes(S) : -1; }

int ffs_checkpoint_save(const ffs_islands *S, void *host, int64_t capacity, ffs_stream stream)
{
    clear_error();
    NvtxRange call("ffs_checkpoint_save");
    if (!S || !host) return set_error(FFS_EINVAL, "NULL argument");
    const int64_t need = islands_blob_bytes(S);
    if (capacity < need) return set_error(FFS_EINVAL, "capacity %lld < %lld bytes", (long long)capacity, (long long)need);
    cudaStream_t st = (cudaStream_t)stream;
    BlobWriter w{static_cast<char *>(host), capacity};
    IslandsBlobHeader h;
    memset(&h, 0, sizeof(h));
    h.magic = kIslandsBlobMagic;
    h.version = kIslandsBlobVersion;
    h.I = S->I;
    h.ld = S->ld;
    h.n = S->inst->n;
    h.has_surrogate = S->sur ? 1 : 0;
    h.fingerprint = instance_fingerprint(S->inst);
    h.bytes = need;
    h.prm = S->prm;
    unsigned long long dec = 0;
    FFS_CUDA_TRY(cudaMemcpyAsync(&dec, S->d_decoded, 8, cudaMemcpyDeviceToHost, st));
    FFS_CUDA_TRY(cudaStreamSynchronize(st));
    h.decoded = (int64_t)dec;
    memcpy(w.take(r16(sizeof(h))), &h, sizeof(h));
    std::vector<int32_t> bsf(S->I);
    std::vector<unsigned long long> mig(2 * (size_t)S->I);
    FFS_CUDA_TRY(cudaMemcpyAsync(bsf.data(), S->d_best_so_far, 4 * (size_t)S->I, cudaMemcpyDeviceToHost, st));
    FFS_CUDA_TRY(cudaMemcpyAsync(mig.data(), S->d_mig, 16 * (size_t)S->I, cudaMemcpyDeviceToHost, st));
    FFS_CUDA_TRY(cudaStreamSynchronize(st));
    char *ent = w.take(r16((int64_t)S->I * sizeof(IslandBlobEntry)));
    for (int i = 0; i < S->I; ++i) {
        IslandBlobEntry e;
        memset(&e, 0, sizeof(e));
        e.kind = S->kind[i];
        e.size = S->size[i];
        e.generation = S->host_gen[i];
        e.best_so_far = bsf[i];
        e.mig_events = (int64_t)mig[2 * i];
        e.mig_rows = (int64_t)mig[2 * i + 1];
        memcpy(ent + i * sizeof(IslandBlobEntry), &e, sizeof(e));
    }
    for (int i = 0; i < S->I; ++i) {
        const int c = S->host_cur[i];
        char *rows = w.take(r16((int64_t)S->size[i] * S->ld * 2));
        char *ms = w.take(r16((int64_t)S->size[i] * 4));
        FFS_CUDA_TRY(cudaMemcpyAsync(rows, S->desc[i].pop[c], (size_t)S->size[i] * S->ld * 2, cudaMemcpyDefault, st));
        FFS_CUDA_TRY(cudaMemcpyAsync(ms, S->desc[i].ms[c], (size_t)S->size[i] * 4, cudaMemcpyDefault, st));
    }
    if (S->sur) {
        const SurrogateState *R = S->sur;
        SurrogateBlob sb;
        memset(&sb, 0, sizeof(sb));
        sb.candidates = R->sp.candidates;
        sb.ring_cap = R->ring_cap;
        sb.ring_count = R->ring_count;
        sb.train_rounds = R->train_rounds;
        sb.valid = std::min(R->ring_count, R->ring_cap);
        memcpy(w.take(r16(sizeof(sb))), &sb, sizeof(sb));
        char *rows = w.take(r16(sb.valid * S->ld * 2));
        char *ms = w.take(r16(sb.valid * 4));
        if (sb.valid > 0) {
            FFS_CUDA_TRY(cudaMemcpyAsync(rows, R->ring_rows, (size_t)sb.valid * S->ld * 2, cudaMemcpyDefault, st));
            FFS_CUDA_TRY(cudaMemcpyAsync(ms, R->ring_ms, (size_t)sb.valid * 4, cudaMemcpyDefault, st));
        }
        char *net = w.take(r16(mlp_state_bytes(R->mlp)));
        int rc = mlp_save(R->mlp, net, st);
        if (rc) return rc;
    }
    FFS_CUDA_TRY(cudaStreamSynchronize(st));
    // the checksum over everything written, its own field taken as zero
    const uint64_t ck = blob_checksum(static_cast<const char *>(host), need, offsetof(IslandsBlobHeader, checksum));
    memcpy(static_cast<char *>(host) + offsetof(IslandsBlobHeader, checksum), &ck, 8);
    return FFS_OK;
}

int ffs_checkpoint_load(ffs_islands *S, const void *host, int64_t size, ffs_stream stream)
{
    clear_error();
    NvtxRange call("ffs_checkpoint_load");
    if (!S || !host) return set_error(FFS_EINVAL, "NULL argument");
    cudaStream_t st = (cudaStream_t)stream;
    BlobReader r{static_cast<const char *>(host), size};
    const char *hp = r.take(r16(sizeof(IslandsBlobHeader)));
    if (!hp) return set_error(FFS_EINVAL, "checkpoint truncated (header)");
    IslandsBlobHeader h;
    memcpy(&h, hp, sizeof(h));
    if (h.magic != kIslandsBlobMagic || h.version != kIslandsBlobVersion)
        return set_error(FFS_EINVAL, "not an islands checkpoint of this version");
    if (h.bytes < (int64_t)sizeof(h) || h.bytes > size || h.bytes % 16)
        return set_error(FFS_EINVAL, "checkpoint truncated (%lld of %lld bytes)", (long long)size, (long long)h.bytes);
    if (blob_checksum(static_cast<const char *>(host), h.bytes, offsetof(IslandsBlobHeader, checksum)) != h.checksum)
        return set_error(FFS_EINVAL, "checkpoint corrupted (checksum differs)");
    r.size = h.bytes;   // only what the checksum covers is read
    if (int rc = check_ga_params(&h.prm)) return rc;
    if (h.I != S->I || h.ld != S->ld || h.n != S->inst->n)
        return set_error(FFS_EINVAL, "checkpoint of %d islands (ld %d, n %d); this handle has %d (ld %d, n %d)", h.I, h.ld,
                         h.n, S->I, S->ld, S->inst->n);
    if (h.fingerprint != instance_fingerprint(S->inst))
        return set_error(FFS_EINVAL, "checkpoint of another instance (fingerprint differs)");
    if (h.has_surrogate != (S->sur ? 1 : 0))
        return set_error(FFS_EINVAL, h.has_surrogate ? "checkpoint has a surrogate; attach one first"
                                                     : "checkpoint has no surrogate but one is attached");
    const char *ent = r.take(r16((int64_t)S->I * sizeof(IslandBlobEntry)));
    if (!ent) return set_error(FFS_EINVAL, "checkpoint truncated (islands)");
    std::vector<IslandBlobEntry> es(S->I);
    for (int i = 0; i < S->I; ++i) {
        memcpy(&es[i], ent + i * sizeof(IslandBlobEntry), sizeof(IslandBlobEntry));
        if (es[i].kind != S->kind[i] || es[i].size != S->size[i])
            return set_error(FFS_EINVAL, "island %d differs in kind or size", i);
        if (es[i].generation < 0 || es[i].generation > 0x7FFFFFFF)
            return set_error(FFS_EINVAL, "island %d generation %lld", i, (long long)es[i].generation);
        if (es[i].best_so_far < 0 || es[i].mig_events < 0 || es[i].mig_rows < 0)
            return set_error(FFS_EINVAL, "island %d metrics counters", i);
    }
    std::vector<const char *> rows(S->I), mss(S->I);
    for (int i = 0; i < S->I; ++i) {
        rows[i] = r.take(r16((int64_t)S->size[i] * S->ld * 2));
        mss[i] = r.take(r16((int64_t)S->size[i] * 4));
        if (!rows[i] || !mss[i]) return set_error(FFS_EINVAL, "checkpoint truncated (island %d)", i);
    }
    SurrogateBlob sb;
    memset(&sb, 0, sizeof(sb));
    const char *ring_rows = nullptr, *ring_ms = nullptr, *net = nullptr;
    int64_t net_bytes = 0;
    if (S->sur) {
        const SurrogateState *R = S->sur;
        const char *sp = r.take(r16(sizeof(SurrogateBlob)));
        if (!sp) return set_error(FFS_EINVAL, "checkpoint truncated (surrogate)");
        memcpy(&sb, sp, sizeof(sb));
        if (sb.candidates != R->sp.candidates || sb.ring_cap != R->ring_cap)
            return set_error(FFS_EINVAL, "surrogate of %d candidates / ring %lld; attached: %d / %lld", sb.candidates,
                             (long long)sb.ring_cap, R->sp.candidates, (long long)R->ring_cap);
        if (sb.ring_count < 0 || sb.train_rounds < 0 || sb.valid != std::min(sb.ring_count, sb.ring_cap))
            return set_error(FFS_EINVAL, "surrogate ring counters inconsistent");
        ring_rows = r.take(r16(sb.valid * S->ld * 2));
        ring_ms = r.take(r16(sb.valid * 4));
        net_bytes = r16(mlp_state_bytes(R->mlp));
        net = r.take(net_bytes);
        if (!ring_rows || !ring_ms || !net) return set_error(FFS_EINVAL, "checkpoint truncated (surrogate state)");
        if (int rc = mlp_check_state(R->mlp, net, net_bytes)) return rc;
    }
    if (r.off != h.bytes)
        return set_error(FFS_EINVAL, "checkpoint of %lld bytes, its sections %lld", (long long)h.bytes, (long long)r.off);
    // everything validated: write the state
    for (int i = 0; i < S->I; ++i) {
        const int c = S->host_cur[i];
        FFS_CUDA_TRY(cudaMemcpyAsync(S->desc[i].pop[c], rows[i], (size_t)S->size[i] * S->ld * 2, cudaMemcpyDefault, st));
        FFS_CUDA_TRY(cudaMemcpyAsync(S->desc[i].ms[c], mss[i], (size_t)S->size[i] * 4, cudaMemcpyDefault, st));
    }
    std::vector<int32_t> gen(S->I);
    for (int i = 0; i < S->I; ++i) gen[i] = (int32_t)es[i].generation;
    FFS_CUDA_TRY(cudaMemcpyAsync(S->d_gen, gen.data(), 4 * (size_t)S->I, cudaMemcpyHostToDevice, st));
    const unsigned long long dec = (unsigned long long)h.decoded;
    FFS_CUDA_TRY(cudaMemcpyAsync(S->d_decoded, &dec, 8, cudaMemcpyHostToDevice, st));
    std::vector<int32_t> bsf(S->I);
    std::vector<unsigned long long> mig(2 * (size_t)S->I);
    for (int i = 0; i < S->I; ++i) {
        bsf[i] = es[i].best_so_far;
        mig[2 * i] = (unsigned long long)es[i].mig_events;
        mig[2 * i + 1] = (unsigned long long)es[i].mig_rows;
    }
    FFS_CUDA_TRY(cudaMemcpyAsync(S->d_best_so_far, bsf.data(), 4 * (size_t)S->I, cudaMemcpyHostToDevice, st));
    FFS_CUDA_TRY(cudaMemcpyAsync(S->d_mig, mig.data(), 16 * (size_t)S->I, cudaMemcpyHostToDevice, st));
    if (S->sur) {
        SurrogateState *R = S->sur;
        if (sb.valid > 0) {
            FFS_CUDA_TRY(cudaMemcpyAsync(R->ring_rows, ring_rows, (size_t)sb.valid * S->ld * 2, cudaMemcpyDefault, st));
            FFS_CUDA_TRY(cudaMemcpyAsync(R->ring_ms, ring_ms, (size_t)sb.valid * 4, cudaMemcpyDefault, st));
        }
        int rc = mlp_load(R->mlp, net, net_bytes, st);
        if (rc) return rc;
        R->ring_count = sb.ring_count;
        R->train_rounds = sb.train_rounds;
        const long long ctr[2] = {sb.ring_count, sb.train_rounds * (long long)R->sp.train_steps};
        FFS_CUDA_TRY(cudaMemcpyAsync(R->d_ctr, ctr, sizeof(ctr), cudaMemcpyHostToDevice, st));
        FFS_CUDA_TRY(cudaStreamSynchronize(st));
        R->drop_graphs();   // they carry the GA parameters, which the load may change
    }
    FFS_CUDA_TRY(cudaStreamSynchronize(st));
    for (int i = 0; i < S->I; ++i) S->host_gen[i] = es[i].generation;
    // the GA parameters come back; the launch shape stays the one in use
    const ffs_params keep = S->prm;
    S->prm = h.prm;
    S->prm.decode_chunk = keep.decode_chunk;
    S->prm.block_threads = keep.block_threads;
    S->prm.decode_variant = keep.decode_variant;
    for (cudaGraphExec_t &g : S->graph_all)
        if (g) {
            cudaGraphExecDestroy(g);
            g = nullptr;
        }
    return FFS_OK;
}

}  // extern "C"
