// ffs_surrogate.cu -- the surrogate-screened cellular generation: every
// cell makes K candidate children, the network scores them, and only the
// best-scored candidate per cell is decoded exactly (the decoder stays the
// only source of makespans).  The exact (chromosome, makespan) pairs feed a
// ring buffer from which the network is trained online.
#include <cuda_bf16.h>

#include "ffs_internal.cuh"
#include "ffs_ga_device.cuh"
#include "ffs_lanes.cuh"

namespace fgpu {

// Network input of one job-order row, written by the whole warp: x[j] =
// position of job j / (n - 1) for j < n (0 when n = 1), zero for n <= j < P,
// the instance features at [P, P + nfeat), zero beyond (BF16, ldx a multiple
// of 8, x 16-byte aligned).  Zeros and features go eight values per 16-byte
// store; the positions are then scattered by job.
__device__ __forceinline__ void warp_write_features(const int16_t *row, int n, int P, const float *inst_feat,
                                                    int nfeat, __nv_bfloat16 *x, int ldx)
{
    const int lane = threadIdx.x & 31;
    const float denom = (float)(n > 1 ? n - 1 : 1);
    for (int g8 = lane; g8 < (ldx >> 3); g8 += 32) {
        uint32_t w4[4];
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            const int j = 8 * g8 + 2 * h;
            const float a = (j >= P && j < P + nfeat) ? inst_feat[j - P] : 0.0f;
            const float b = (j + 1 >= P && j + 1 < P + nfeat) ? inst_feat[j + 1 - P] : 0.0f;
            const __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
            w4[h] = *reinterpret_cast<const uint32_t *>(&v);
        }
        reinterpret_cast<uint4 *>(x)[g8] = make_uint4(w4[0], w4[1], w4[2], w4[3]);
    }
    __syncwarp();
    for (int q = lane; q < n; q += 32) {
        const int j = row[q];
        if ((unsigned)j < (unsigned)n) x[j] = __float2bfloat16_rn((float)q / denom);
    }
    __syncwarp();
}

// The scoring form of a row's network input, written by the whole warp:
// the job positions x[j] = position of job j / (n - 1) for j < n and zeros
// up to xw (a multiple of 8); the constant rest of the input (zeros, the
// instance features) is folded into the first layer's bias by the forward
// pass that reads these rows.
__device__ __forceinline__ void warp_write_positions(const int16_t *row, int n, int xw, __nv_bfloat16 *x)
{
    const int lane = threadIdx.x & 31;
    const float denom = (float)(n > 1 ? n - 1 : 1);
    for (int g8 = lane; g8 < (xw >> 3); g8 += 32) reinterpret_cast<uint4 *>(x)[g8] = make_uint4(0u, 0u, 0u, 0u);
    __syncwarp();
    for (int q = lane; q < n; q += 32) {
        const int j = row[q];
        if ((unsigned)j < (unsigned)n) x[j] = __float2bfloat16_rn((float)q / denom);
    }
    __syncwarp();
}

// Candidates built per warp: a warp builds its children one after another
// with all 32 lanes, so few children per warp and many warps hide the
// parents' load latency.
constexpr int kCandPerWarp = 4;

// Candidate k of cell c: the cellular child (two tournaments, order
// crossover, swap mutation) drawn from the stream of purpose
// kPurposeSurrogateBase + k.  Lane l < kCandPerWarp of warp w builds
// candidate w * kCandPerWarp + l.  With X non-null, the warp then writes its
// candidates' job positions as network input rows of xw values
// (warp_write_positions).
__global__ void k_sur_candidates(GaScalars g, const __grid_constant__ IslandBatch batch, int rows, int cols, int n,
                                 int ld, int K, int16_t *cand, __nv_bfloat16 *X, int xw)
{
    extern __shared__ uint32_t bits_smem[];
    const int cells = rows * cols;
    const int total = batch.count * cells * K;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    const int t = gw * kCandPerWarp + lane;
    const bool valid = lane < kCandPerWarp && t < total;
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
    job.p1 = job.p2 = pin;
    job.l = job.r = 0;
    job.cross = false;
    bool mutate = false;
    U4 b2{0, 0, 0, 0};
    if (valid) {
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
        mutate = fires(b1.w, g.cell_pm);
    }
    if (pairs_build_fits(n)) {
        warp_build_children_pairs(job, n, ld, bits_smem + (threadIdx.x >> 5) * 2 * mark_words(n));
    } else {
        warp_build_children(job, n, ld, bits_smem + (threadIdx.x >> 5) * mark_words(n));
    }
    if (mutate) {
        int16_t *child = job.child;
        const int i = (int)uniform_below(b2.x, (uint32_t)n), j = (int)uniform_below(b2.y, (uint32_t)n);
        const int16_t tmp = child[i];
        child[i] = child[j];
        child[j] = tmp;
    }
    if (!X) return;
    __syncwarp();
    // network inputs of the warp's candidates, all lanes on one row at a time
    unsigned todo = __ballot_sync(0xFFFFFFFFu, valid);
    while (todo) {
        const int j0 = __ffs(todo) - 1;
        todo &= todo - 1u;
        const int tj = gw * kCandPerWarp + j0;
        warp_write_positions(cand + (int64_t)tj * ld, n, xw, X + (int64_t)tj * xw);
    }
}

// Candidate cut pairs of screened pseudo pairs: job jj = (pair q, candidate
// t, child w) with jj = 2 (q K + t) + w over the batch's pairs; candidate t
// of pair k takes its cuts from draws 1 and 2 of purpose
// kPurposeSurrogatePseudoBase + t (l = min, r = max of two uniforms in
// [0, n)), child 0 = OX(a, b), child 1 = OX(b, a).  Lane l < kCandPerWarp of
// warp w builds job w * kCandPerWarp + l; with X non-null the warp then
// writes its jobs' job positions (rows of xw values).
__global__ void k_sur_pseudo_candidates(GaScalars g, const __grid_constant__ IslandBatch batch, int size, int n,
                                        int ld, int K, int16_t *cand, __nv_bfloat16 *X, int xw)
{
    extern __shared__ uint32_t bits_smem[];
    const int pairs = size / 2;
    const int total = batch.count * pairs * K * 2;
    const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (gw * kCandPerWarp >= total) return;   // whole warps leave together
    const int jj = gw * kCandPerWarp + lane;
    const bool valid = lane < kCandPerWarp && jj < total;
    const int tj = valid ? jj : gw * kCandPerWarp;
    const int q = tj >> 1, w = tj & 1;
    const int gp = q / K, t = q - gp * K;
    const int bi = gp / pairs, k = gp - bi * pairs;
    const IslandRef &ref = batch.ref[bi];
    const int16_t *pin;
    const int32_t *msin;
    int16_t *pout;
    int32_t *msout;
    uint32_t gen;
    resolve(ref, pin, msin, pout, msout, gen);
    const U4 d = draw_block(g.seed, kPurposeSurrogatePseudoBase + (uint32_t)t, ref.island, gen, (uint32_t)k, 0u);
    const int u = (int)uniform_below(d.y, (uint32_t)n), v = (int)uniform_below(d.z, (uint32_t)n);
    const int16_t *a = pin + (int64_t)(2 * k) * ld, *b = a + ld;
    ChildJob job;
    job.active = valid;
    job.cross = true;
    job.l = min(u, v);
    job.r = max(u, v);
    job.p1 = w ? b : a;
    job.p2 = w ? a : b;
    job.child = cand + (int64_t)tj * ld;
    if (pairs_build_fits(n)) {
        warp_build_children_pairs(job, n, ld, bits_smem + (threadIdx.x >> 5) * 2 * mark_words(n));
    } else {
        warp_build_children(job, n, ld, bits_smem + (threadIdx.x >> 5) * mark_words(n));
    }
    if (!X) return;
    __syncwarp();
    unsigned todo = __ballot_sync(0xFFFFFFFFu, valid);
    while (todo) {
        const int j0 = __ffs(todo) - 1;
        todo &= todo - 1u;
        const int r = gw * kCandPerWarp + j0;
        warp_write_positions(cand + (int64_t)r * ld, n, xw, X + (int64_t)r * xw);
    }
}

// Per cell: the best-scored candidate (lowest score, lowest index on ties)
// is decoded exactly and replaces the cell iff better; the pair is appended
// to the ring buffer at slot (ring_base + cell) mod ring_cap, ring_base =
// ctr[0], the pairs appended before this generation (a device counter, so
// the generation can be replayed from a CUDA graph; k_sur_tick advances it).
__global__ void __launch_bounds__(512) k_sur_select(DecodeLayout L, const uint32_t *__restrict__ tab_g,
                                                    const int32_t *__restrict__ stage_g, GaScalars g,
                                                    const __grid_constant__ IslandBatch batch, int rows, int cols,
                                                    int ld, int K, const int16_t *cand, const float *scores,
                                                    int32_t *chosen, int16_t *ring_rows, int32_t *ring_ms,
                                                    long long ring_cap, const long long *ctr,
                                                    unsigned long long *decoded)
{
    const long long ring_base = ctr[0];
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
    uint32_t *region = thread_region(smem + map.region, Ls.thread_words);
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
        if (!FFS_DCHECK(pick >= 0 && pick < K, kCheckPick)) pick = 0;
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

// k_sur_select with the stage-parallel decoder (ffs_lanes.cuh), for screens
// too small to fill the GPU one cell per lane: a warp takes floor(32 / S)
// cells at a time.  Lane l < C of the warp picks cell l's best-scored
// candidate (lowest score, lowest k on ties), the warp stages the picked
// rows in shared memory, each group of S lanes decodes one of them, and
// lane l then replaces its cell iff better and appends the pair to the ring
// exactly as k_sur_select does.
__global__ void __launch_bounds__(128) k_sur_select_lanes(int n, int S, uint32_t SH, int MM, int obj_words,
                                                          int has_rel, int has_due, uint32_t wt,
                                                          const uint32_t *__restrict__ tab_g,
                                                          const int32_t *__restrict__ stage_g, GaScalars g,
                                                          const __grid_constant__ IslandBatch batch, int rows, int cols,
                                                          int ld, int K, const int16_t *cand, const float *scores,
                                                          int32_t *chosen, int16_t *ring_rows, int32_t *ring_ms,
                                                          long long ring_cap, const long long *ctr,
                                                          unsigned long long *decoded)
{
    const long long ring_base = ctr[0];
    extern __shared__ __align__(16) uint32_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, W = blockDim.x >> 5;
    const LaneSetup u = lanes_block_setup(smem, n, S, obj_words, has_rel, has_due, tab_g, stage_g, ld);
    const int cells = rows * cols, total = cells * batch.count, C = u.C;
    if (decoded && blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(decoded, (unsigned long long)total);
    const int items = (total + C - 1) / C;
    for (int it = blockIdx.x * W + warp; it < items; it += gridDim.x * W) {
        const int gq0 = it * C;
        const int nrows = min(C, total - gq0);
        const bool mine = lane < nrows;          // lane l handles cell gq0 + l
        const int gq = gq0 + (mine ? lane : 0);
        int pick = 0;
        if (mine) {
            // the cell's K (<= 16) scores loaded together, then the lowest
            // (the lowest k on ties)
            const float *sc = scores + (int64_t)gq * K;
            float v[16];
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] = k < K ? sc[k] : 0.0f;
            float best = v[0];
#pragma unroll
            for (int k = 1; k < 16; ++k)
                if (k < K && v[k] < best) {
                    best = v[k];
                    pick = k;
                }
            if (!FFS_DCHECK(pick >= 0 && pick < K, kCheckPick)) pick = 0;
        }
        const int16_t *drow = cand + ((int64_t)gq * K + pick) * ld;
        // the picked rows into the warp's buffer, every 16-byte block of them
        // in flight at once (block w of the nrows x q: row w / q)
        const int q = ld >> 3, tot = nrows * q;
        int4 *buf = reinterpret_cast<int4 *>(u.rows);
        for (int w0 = 0; w0 < tot; w0 += 128) {
            int4 v4[4];
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int w = w0 + 32 * h + lane;
                const int j = w < tot ? w / q : 0;
                const int4 *src = reinterpret_cast<const int4 *>(__shfl_sync(0xFFFFFFFFu, (unsigned long long)drow, j));
                if (w < tot) v4[h] = src[w - j * q];
            }
#pragma unroll
            for (int h = 0; h < 4; ++h) {
                const int w = w0 + 32 * h + lane;
                if (w < tot) buf[w] = v4[h];
            }
        }
        __syncwarp();
        // the cell's current makespan, read before the decode
        const int bi = gq / cells, c = gq - bi * cells;
        const int16_t *pin;
        const int32_t *msin;
        int16_t *pout;
        int32_t *msout;
        uint32_t gen;
        resolve(batch.ref[bi], pin, msin, pout, msout, gen);
        const int32_t old = mine ? msin[c] : 0;
        const bool active = u.g < nrows;
        const uint32_t sM = (active ? (uint32_t)u.s : 0xFFu) | (u.Ms << 8) | (SH << 16);
        const uint32_t genes = u.rows_sa + (active ? (uint32_t)(u.g * ld * 2) : 0u);
        const int32_t v = lane_decode_dispatch(MM, u.tab, u.row_bytes, genes, u.nS, sM, u.win, u.rel, u.due, wt);
        // lane l takes its cell's objective from its group's last lane
        const int32_t ms = __shfl_sync(0xFFFFFFFFu, v, (mine ? lane : 0) * S + S - 1);
        const long long slot = (ring_base + gq) % ring_cap;
        bool better = false;
        if (mine) {
            better = ms >= 0 && (g.replace_le ? (uint32_t)ms <= (uint32_t)old : (uint32_t)ms < (uint32_t)old);
            msout[c] = better ? ms : old;
            chosen[gq] = pick;
            ring_ms[slot] = ms;
        }
        // rows out: the cell's output row takes the pick (from the buffer) or
        // its old row, the ring slot the pick; all blocks in flight at once
        const int16_t *staged = reinterpret_cast<const int16_t *>(u.rows) + (int64_t)(mine ? lane : 0) * ld;
        const int16_t *out_src = better ? staged : pin + (int64_t)c * ld;
        int16_t *out_dst = pout + (int64_t)c * ld;
        int16_t *ring_dst = ring_rows + slot * ld;
        for (int w0 = 0; w0 < tot; w0 += 64) {
            int4 a4[2], b4[2];
            int4 *da[2], *db[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int w = w0 + 32 * h + lane;
                const int j = w < tot ? w / q : 0, k = w - j * q;
                const int4 *sa = reinterpret_cast<const int4 *>(__shfl_sync(0xFFFFFFFFu, (unsigned long long)out_src, j));
                const int4 *sb = reinterpret_cast<const int4 *>(__shfl_sync(0xFFFFFFFFu, (unsigned long long)staged, j));
                da[h] = reinterpret_cast<int4 *>(__shfl_sync(0xFFFFFFFFu, (unsigned long long)out_dst, j)) + k;
                db[h] = reinterpret_cast<int4 *>(__shfl_sync(0xFFFFFFFFu, (unsigned long long)ring_dst, j)) + k;
                if (w < tot) {
                    a4[h] = sa[k];
                    b4[h] = sb[k];
                }
            }
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if (w0 + 32 * h + lane < tot) {
                    *da[h] = a4[h];
                    *db[h] = b4[h];
                }
        }
        __syncwarp();   // the buffer is refilled next
    }
}

// The surrogate's device counters: ctr[0] ring pairs appended, ctr[1]
// training batches drawn, ctr[2] the ring count when the current generation
// began (set by k_sur_snapshot).  A training round runs beside the current
// generation's selection, which appends to the ring; it reads only the
// snapshot and the pairs before it, which the selection does not touch.

// Standardisation of the training targets: mean and 1 / std (std at least 1)
// of the makespans of the `recent` newest ring pairs before the current
// generation (the last generation's exact decodes).  The screen needs only
// the ranking of a cell's candidates, whose makespans differ by a few tenths
// of a percent late in a run: standardised targets keep those differences at
// the scale the network learns.  Computed by every block of the gather that
// uses it (the ring's makespans are L2-resident): the sums of the makespans
// and of their squares in exact integers, then mean = S / m and var = Q / m -
// mean^2 in double.  The whole block calls it; the result is in norm[0..1].
__device__ void block_target_norm(const int32_t *ring_ms, long long ring_cap, const long long *ctr, int recent,
                                  float *norm)
{
    __shared__ long long part[2][32];
    const long long cnt = ctr[2] < ring_cap ? ctr[2] : ring_cap;
    const int m = (int)(cnt < recent ? cnt : recent);
    long long s = 0, q = 0;
    const long long last = (ctr[2] - 1) % ring_cap;   // slot of the newest pair (m > 0 only)
    for (int i0 = threadIdx.x; i0 < m; i0 += 8 * blockDim.x) {
        long long v[8];   // eight loads in flight
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * (int)blockDim.x;
            const long long slot = last - i;
            v[u] = i < m ? ring_ms[slot >= 0 ? slot : slot + ring_cap] : 0;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            s += v[u];
            q += v[u] * v[u];
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
        q += __shfl_xor_sync(0xFFFFFFFFu, q, o);
    }
    if ((threadIdx.x & 31) == 0) {
        part[0][threadIdx.x >> 5] = s;
        part[1][threadIdx.x >> 5] = q;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        long long S = 0, Q = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
            S += part[0][w];
            Q += part[1][w];
        }
        const double mean = m > 0 ? (double)S / m : 0.0;
        double var = m > 0 ? (double)Q / m - mean * mean : 1.0;
        if (var < 1.0) var = 1.0;
        norm[0] = (float)mean;
        norm[1] = (float)(1.0 / sqrt(var));
    }
    __syncthreads();
}

// Training batches k = 0 .. batches - 1 of B pairs each, drawn uniformly
// (Philox, purpose kPurposeTrainSample, generation field = batches drawn
// before it, ctr[1] + k) from the V = min(ctr[2], ring_cap - recent) newest
// pairs before the current generation (pair i = the i-th newest, slot
// (ctr[2] - 1 - i) mod ring_cap; the current generation writes the `recent`
// slots after them), written as network inputs X (row k B + b, one warp per
// sample); target = (makespan - norm[0]) * norm[1] (block_target_norm; block
// 0 also leaves it in norm_out).  The last block to finish (counted in
// ctr[3], reset by it) advances the batch count ctr[1] by `batches`, after
// every block has read it.
__global__ void k_sur_gather(const int16_t *ring_rows, const int32_t *ring_ms, long long ring_cap, int recent,
                             long long *ctr, int ld, uint64_t seed, int B, int batches, float *targets,
                             float *norm_out, int n, int P, const float *inst_feat, int nfeat, __nv_bfloat16 *X,
                             int ldx)
{
    __shared__ float norm[2];
    block_target_norm(ring_ms, ring_cap, ctr, recent, norm);
    if (blockIdx.x == 0 && threadIdx.x < 2) norm_out[threadIdx.x] = norm[threadIdx.x];
    const long long room = ring_cap - recent;
    const long long valid = ctr[2] < room ? ctr[2] : room;
    const long long newest = (ctr[2] - 1) % ring_cap;
    const long long drawn = ctr[1];   // batches drawn before this launch
    const int lane = threadIdx.x & 31;
    const int rows = B * batches;
    for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < rows; r += (gridDim.x * blockDim.x) >> 5) {
        const int k = r / B, b = r - k * B;
        const U4 d = draw_block(seed, kPurposeTrainSample, 0u, (uint32_t)(drawn + k), (uint32_t)b, 0u);
        const long long i = (long long)(((unsigned long long)d.x * (unsigned long long)valid) >> 32);
        const long long slot = newest - i >= 0 ? newest - i : newest - i + ring_cap;
        if (!FFS_DCHECK(slot >= 0 && slot < ring_cap, kCheckRingSlot)) continue;   // warp-uniform
        warp_write_features(ring_rows + slot * ld, n, P, inst_feat, nfeat, X + (int64_t)r * ldx, ldx);
        if (lane == 0) targets[r] = ((float)ring_ms[slot] - norm[0]) * norm[1];
    }
    __syncthreads();   // this block's warps have read ctr[1]
    if (threadIdx.x == 0) {
        __threadfence();
        unsigned long long *done = reinterpret_cast<unsigned long long *>(ctr + 3);
        if (atomicAdd(done, 1ull) == (unsigned long long)gridDim.x - 1ull) {
            ctr[1] += batches;
            *done = 0ull;
        }
    }
}

// ctr[which] += add (one thread): the surrogate's device counters; with
// add < 0, the snapshot ctr[2] = ctr[0] instead.
__global__ void k_sur_tick(long long *ctr, int which, long long add)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        if (add < 0) ctr[2] = ctr[0];
        else ctr[which] += add;
    }
}

__global__ void k_fill_f32(float *p, int64_t n, float v)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) p[i] = v;
}

int launch_sur_candidates(const ffs_instance *inst, const GaScalars &g, const IslandBatch &batch, int rows, int cols,
                          int ld, int K, int16_t *cand, void *X, int xw, cudaStream_t st)
{
    const int total = batch.count * rows * cols * K;
    const int T = 128;
    const int warps = (total + kCandPerWarp - 1) / kCandPerWarp;
    const size_t smem = (size_t)(T / 32) * (pairs_build_fits(inst->n) ? 2 : 1) * mark_words(inst->n) * 4;
    FFS_CUDA_TRY(cudaFuncSetAttribute(k_sur_candidates, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_sur_candidates<<<(warps * 32 + T - 1) / T, T, smem, st>>>(g, batch, rows, cols, inst->n, ld, K, cand,
                                                                static_cast<__nv_bfloat16 *>(X), xw);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

int launch_sur_pseudo_candidates(const ffs_instance *inst, const GaScalars &g, const IslandBatch &batch, int size,
                                 int ld, int K, int16_t *cand, void *X, int xw, cudaStream_t st)
{
    const long long total = (long long)batch.count * (size / 2) * K * 2;
    if (total <= 0) return FFS_OK;
    const int T = 128;
    const long long warps = (total + kCandPerWarp - 1) / kCandPerWarp;
    const size_t smem = (size_t)(T / 32) * (pairs_build_fits(inst->n) ? 2 : 1) * mark_words(inst->n) * 4;
    FFS_CUDA_TRY(cudaFuncSetAttribute(k_sur_pseudo_candidates, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    k_sur_pseudo_candidates<<<(unsigned)((warps * 32 + T - 1) / T), T, smem, st>>>(
        g, batch, size, inst->n, ld, K, cand, static_cast<__nv_bfloat16 *>(X), xw);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

int launch_sur_select(const ffs_instance *inst, const GaScalars &g, const IslandBatch &batch, int rows, int cols,
                      int ld, int K, const int16_t *cand, const float *scores, int32_t *chosen, int16_t *ring_rows,
                      int32_t *ring_ms, long long ring_cap, const long long *ctr, int B_req, int T_req,
                      unsigned long long *decoded, cudaStream_t st)
{
    const int64_t total = (int64_t)rows * cols * batch.count;
    if (lanes_decode_pays(inst, total, (B_req || T_req) && g.variant == 0 ? -1 : g.variant)) {
        LanesPlan lp;
        int rc = plan_lanes(inst, total, ld, &lp);
        if (rc) return rc;
        FFS_CUDA_TRY(cudaFuncSetAttribute(k_sur_select_lanes, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lp.smem));
        k_sur_select_lanes<<<lp.blocks, lp.T, lp.smem, st>>>(inst->n, inst->S, (uint32_t)inst->SH, lp.MM,
                                                            inst->obj_words, inst->has_rel, inst->has_due,
                                                            (uint32_t)inst->wt, inst->d_tab, inst->d_stage, g, batch,
                                                            rows, cols, ld, K, cand, scores, chosen, ring_rows, ring_ms,
                                                            ring_cap, ctr, decoded);
        FFS_CUDA_TRY(cudaGetLastError());
        return FFS_OK;
    }
    Plan p;
    const int T_sp = spread_threads(inst, total, T_req);
    int rc = plan_decode(inst, (const void *)k_sur_select, B_req, T_sp, 0, &p, g.variant);
    if (rc && T_sp != T_req) rc = plan_decode(inst, (const void *)k_sur_select, B_req, T_req, 0, &p, g.variant);
    if (rc) return rc;
    FFS_CUDA_TRY(cudaFuncSetAttribute(k_sur_select, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
    const int grid = grid_for(inst, p, (int64_t)rows * cols * batch.count);
    k_sur_select<<<grid, p.T, p.smem, st>>>(p.L, inst->d_tab, inst->d_stage, g, batch, rows, cols, ld, K, cand, scores,
                                             chosen, ring_rows, ring_ms, ring_cap, ctr, decoded);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

int launch_sur_gather(const int16_t *ring_rows, const int32_t *ring_ms, long long ring_cap, int recent,
                      long long *ctr, int ld, uint64_t seed, int B, int batches, float *targets,
                      float *norm, int n, int P, const float *inst_feat, int nfeat, void *X, int ldx,
                      cudaStream_t st)
{
    const long long warps = (long long)B * batches;
    k_sur_gather<<<(unsigned)((warps * 32 + 255) / 256), 256, 0, st>>>(
        ring_rows, ring_ms, ring_cap, recent, ctr, ld, seed, B, batches, targets, norm, n, P, inst_feat, nfeat,
        static_cast<__nv_bfloat16 *>(X), ldx);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

int launch_sur_tick(long long *ctr, int which, long long add, cudaStream_t st)
{
    k_sur_tick<<<1, 32, 0, st>>>(ctr, which, add);
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
