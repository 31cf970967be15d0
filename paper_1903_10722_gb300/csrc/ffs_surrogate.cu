// ffs_surrogate.cu -- the surrogate-screened cellular generation: every
// cell makes K candidate children, the network scores them, and only the
// best-scored candidate per cell is decoded exactly (the decoder stays the
// only source of makespans).  The exact (chromosome, makespan) pairs feed a
// ring buffer from which the network is trained online.
#include <cuda_bf16.h>

#include "ffs_internal.cuh"
#include "ffs_ga_device.cuh"

namespace fgpu {

// Candidate k of cell c: the cellular child (two tournaments, order
// crossover, swap mutation) drawn from the stream of purpose kPurposeSurrogateBase + k.
__global__ void k_sur_candidates(GaScalars g, const __grid_constant__ IslandBatch batch, int rows, int cols, int n,
                                 int ld, int K, int16_t *cand)
{
    extern __shared__ uint32_t bits_smem[];
    const int cells = rows * cols;
    const int total = batch.count * cells * K;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = t < total;
    const int tt = valid ? t : total - 1;
    const int bi = tt / (cells * K);
    const int rem = tt - bi * cells * K;
    const int c = rem / K, k = rem - (rem / K) * K;
    const IslandRef &ref = batch.ref[bi];
    const int16_t *pin;
    const int32_t *msin;
    int16_t *pout;
    int32_t *msout;
    uint32_t gen;
    resolve(ref, pin, msin, pout, msout, gen);
    const uint32_t purpose = kPurposeSurrogateBase + (uint32_t)k;
    ChildJob job;
    job.active = valid;
    job.child = cand + (int64_t)tt * ld;
    bool mutate = false;
    U4 b2{0, 0, 0, 0};
    {
        const U4 b0 = draw_block(g.seed, purpose, ref.island, gen, (uint32_t)c, 0u);
        const U4 b1 = draw_block(g.seed, purpose, ref.island, gen, (uint32_t)c, 1u);
        b2 = draw_block(g.seed, purpose, ref.island, gen, (uint32_t)c, 2u);
        const int r = c / cols, q = c - r * cols;
        const int up = ((r + rows - 1) % rows) * cols + q, down = ((r + 1) % rows) * cols + q;
        const int west = r * cols + (q + cols - 1) % cols, east = r * cols + (q + 1) % cols;
        auto slot = [&](uint32_t x) {
            const uint32_t s = uniform_below(x, 5u);
            return s == 0 ? c : s == 1 ? up : s == 2 ? down : s == 3 ? west : east;
        };
        int a = slot(b0.x), b = slot(b0.y);
        const int par1 = (msin[b] < msin[a]) ? b : a;
        a = slot(b0.z);
        b = slot(b0.w);
        const int par2 = (msin[b] < msin[a]) ? b : a;
        job.p1 = pin + (int64_t)par1 * ld;
        job.p2 = pin + (int64_t)par2 * ld;
        job.cross = fires(b1.x, g.cell_pc);
        const int u = (int)uniform_below(b1.y, (uint32_t)n), v = (int)uniform_below(b1.z, (uint32_t)n);
        job.l = min(u, v);
        job.r = max(u, v);
        mutate = valid && fires(b1.w, g.cell_pm);
    }
    uint32_t *bits = bits_smem + (threadIdx.x >> 5) * mark_words(n);
    warp_build_children(job, n, ld, bits);
    if (mutate) {
        int16_t *child = job.child;
        const int i = (int)uniform_below(b2.x, (uint32_t)n), j = (int)uniform_below(b2.y, (uint32_t)n);
        const int16_t tmp = child[i];
        child[i] = child[j];
        child[j] = tmp;
    }
}

// Network input of job-order rows, one warp per row: x[j] = position of job j
// / (n - 1) for j < n, 0 for n <= j < P, then the instance features; BF16.
__global__ void k_sur_features(const int16_t *rows, int64_t nrows, int n, int ld, int P, const float *inst_feat,
                               int nfeat, __nv_bfloat16 *X, int ldx)
{
    const int lane = threadIdx.x & 31;
    const float denom = (float)(n > 1 ? n - 1 : 1);
    for (int64_t r = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5; r < nrows;
         r += ((int64_t)gridDim.x * blockDim.x) >> 5) {
        __nv_bfloat16 *x = X + r * ldx;
        for (int j = lane; j < ldx; j += 32) x[j] = __float2bfloat16_rn(0.0f);
        __syncwarp();
        const int16_t *row = rows + r * ld;
        for (int k = lane; k < n; k += 32) {
            const int j = row[k];
            if ((unsigned)j < (unsigned)n) x[j] = __float2bfloat16_rn((float)k / denom);
        }
        for (int f = lane; f < nfeat; f += 32) x[P + f] = __float2bfloat16_rn(inst_feat[f]);
        __syncwarp();
    }
}

// Per cell: the best-scored candidate (lowest score, lowest index on ties)
// is decoded exactly and replaces the cell iff better; the pair is appended
// to the ring buffer at slot (ring_base + cell) mod ring_cap.
__global__ void __launch_bounds__(512) k_sur_select(DecodeLayout L, const uint32_t *__restrict__ tab_g,
                                                    const int32_t *__restrict__ stage_g, GaScalars g,
                                                    const __grid_constant__ IslandBatch batch, int rows, int cols,
                                                    int ld, int K, const int16_t *cand, const float *scores,
                                                    int32_t *chosen, int16_t *ring_rows, int32_t *ring_ms,
                                                    long long ring_cap, long long ring_base,
                                                    unsigned long long *decoded)
{
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ DecodeLayout s_L;
    const int T = blockDim.x;
    const SmemMap map = smem_map(L.n, L.S, T, 0, L.obj_words);
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
    uint32_t *region = smem + map.region + threadIdx.x;
    const uint16_t *tab = reinterpret_cast<const uint16_t *>(smem + map.tab);
    const int cells = rows * cols;
    const int total = cells * batch.count;
    if (decoded && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(decoded, (unsigned long long)total);
    for (int base = blockIdx.x * T + warp * 32; base < total; base += gridDim.x * T) {
        const int gc = base + lane;
        const bool valid = gc < total;
        const int gq = valid ? gc : total - 1;
        const int bi = gq / cells, c = gq - bi * cells;
        const int16_t *pin;
        const int32_t *msin;
        int16_t *pout;
        int32_t *msout;
        uint32_t gen;
        resolve(batch.ref[bi], pin, msin, pout, msout, gen);
        const float *sc = scores + (int64_t)gq * K;
        int pick = 0;
        for (int k = 1; k < K; ++k)
            if (sc[k] < sc[pick]) pick = k;
        const int16_t *drow = cand + ((int64_t)gq * K + pick) * ld;
        const int32_t ms = decode_chromosome(Ls, drow, region, T, tab, wst);
        bool better = false, keep = false;
        if (valid) {
            const int32_t old = msin[c];
            better = ms >= 0 && (g.replace_le ? (uint32_t)ms <= (uint32_t)old : (uint32_t)ms < (uint32_t)old);
            keep = !better;
            msout[c] = better ? ms : old;
            chosen[gq] = pick;
            const long long slot = (ring_base + gq) % ring_cap;
            ring_ms[slot] = ms;
        }
        warp_copy_rows(better, drow, pout + (int64_t)c * ld, ld);
        warp_copy_rows(keep, pin + (int64_t)c * ld, pout + (int64_t)c * ld, ld);
        warp_copy_rows(valid, drow, ring_rows + ((ring_base + gq) % ring_cap) * ld, ld);
    }
    decode_tmem_end(Ls);
}

// Training batch: B rows drawn uniformly (Philox, purpose kPurposeTrainSample)
// from the first `valid` ring slots; target = makespan * inv_lb - 1.
__global__ void k_sur_gather(const int16_t *ring_rows, const int32_t *ring_ms, long long valid, int ld, uint64_t seed,
                             uint32_t draw_gen, int B, int16_t *out_rows, float *targets, float inv_lb)
{
    const int lane = threadIdx.x & 31;
    for (int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < B; b += (gridDim.x * blockDim.x) >> 5) {
        const U4 d = draw_block(seed, kPurposeTrainSample, 0u, draw_gen, (uint32_t)b, 0u);
        const long long idx = (long long)(((unsigned long long)d.x * (unsigned long long)valid) >> 32);
        const int4 *s4 = reinterpret_cast<const int4 *>(ring_rows + idx * ld);
        int4 *d4 = reinterpret_cast<int4 *>(out_rows + (int64_t)b * ld);
        for (int k = lane; k < (ld >> 3); k += 32) d4[k] = s4[k];
        if (lane == 0) targets[b] = (float)ring_ms[idx] * inv_lb - 1.0f;
    }
}

__global__ void k_fill_f32(float *p, int64_t n, float v)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

int launch_sur_candidates(const ffs_instance *inst, const GaScalars &g, const IslandBatch &batch, int rows, int cols,
                          int ld, int K, int16_t *cand, cudaStream_t st)
{
    const int total = batch.count * rows * cols * K;
    const int T = 128;
    const size_t smem = (size_t)(T / 32) * mark_words(inst->n) * 4;
    FFS_CUDA_TRY(cudaFuncSetAttribute(k_sur_candidates, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_sur_candidates<<<(total + T - 1) / T, T, smem, st>>>(g, batch, rows, cols, inst->n, ld, K, cand);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

int launch_sur_features(const int16_t *rows, int64_t nrows, int n, int ld, int P, const float *inst_feat, int nfeat,
                        void *X, int ldx, cudaStream_t st)
{
    if (nrows <= 0) return FFS_OK;
    int64_t blocks = (nrows * 32 + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    k_sur_features<<<(int)blocks, 256, 0, st>>>(rows, nrows, n, ld, P, inst_feat, nfeat,
                                                static_cast<__nv_bfloat16 *>(X), ldx);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

int launch_sur_select(const ffs_instance *inst, const GaScalars &g, const IslandBatch &batch, int rows, int cols,
                      int ld, int K, const int16_t *cand, const float *scores, int32_t *chosen, int16_t *ring_rows,
                      int32_t *ring_ms, long long ring_cap, long long ring_base, int B_req, int T_req,
                      unsigned long long *decoded, cudaStream_t st)
{
    Plan p;
    int rc = plan_decode(inst, (const void *)k_sur_select, B_req, T_req, 0, &p, g.variant);
    if (rc) return rc;
    FFS_CUDA_TRY(cudaFuncSetAttribute(k_sur_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
    const int grid = grid_for(inst, p, (int64_t)rows * cols * batch.count);
    k_sur_select<<<grid, p.T, p.smem, st>>>(p.L, inst->d_tab, inst->d_stage, g, batch, rows, cols, ld, K, cand, scores,
                                             chosen, ring_rows, ring_ms, ring_cap, ring_base, decoded);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

int launch_sur_gather(const int16_t *ring_rows, const int32_t *ring_ms, long long valid, int ld, uint64_t seed,
                      uint32_t draw_gen, int B, int16_t *out_rows, float *targets, float inv_lb, cudaStream_t st)
{
    k_sur_gather<<<(B * 32 + 255) / 256, 256, 0, st>>>(ring_rows, ring_ms, valid, ld, seed, draw_gen, B, out_rows,
                                                       targets, inv_lb);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

int launch_fill_f32(float *p, int64_t n, float v, cudaStream_t st)
{
    if (n <= 0) return FFS_OK;
    k_fill_f32<<<256, 256, 0, st>>>(p, n, v);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

}  // namespace fgpu
