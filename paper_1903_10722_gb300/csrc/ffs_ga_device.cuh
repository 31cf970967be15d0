// ffs_ga_device.cuh -- device-side GA building blocks shared by the island and
// batch kernels: warp-cooperative child construction and the fused cellular
// generation of one cell per lane.
#pragma once

#include "ffs_internal.cuh"

namespace fgpu {

// ---------------------------------------------------------------------------
// Warp-cooperative child construction.  Each lane of the warp supplies one
// child to build (parents, cut points, whether crossover fires, output row);
// the warp builds them one after the other with all 32 lanes on the genes,
// so rows are read and written in coalesced 64-byte runs.
//
// Order crossover: the child keeps p1[l..r]; the other positions, from r+1
// onward cyclically, take p2's genes met from position r+1 onward
// cyclically, skipping genes already placed.  Without crossover the child
// copies p1.  `mark` is the warp's shared mark of mark_words(n) words, one
// byte per gene.
// ---------------------------------------------------------------------------
struct ChildJob {
    const int16_t *p1;
    const int16_t *p2;
    int16_t *child;
    int l, r;
    bool cross;
    bool active;
};

__device__ __forceinline__ void warp_build_children(const ChildJob &me, int n, int ld, uint32_t *mark)
{
    uint8_t *flag = reinterpret_cast<uint8_t *>(mark);
    const int lane = threadIdx.x & 31;
    const int words = mark_words(n);
    unsigned todo = __ballot_sync(0xFFFFFFFFu, me.active);
    while (todo) {
        const int j = __ffs(todo) - 1;
        todo &= todo - 1u;
        const int16_t *p1 = (const int16_t *)__shfl_sync(0xFFFFFFFFu, (unsigned long long)me.p1, j);
        const int16_t *p2 = (const int16_t *)__shfl_sync(0xFFFFFFFFu, (unsigned long long)me.p2, j);
        int16_t *child = (int16_t *)__shfl_sync(0xFFFFFFFFu, (unsigned long long)me.child, j);
        const int l = __shfl_sync(0xFFFFFFFFu, me.l, j);
        const int r = __shfl_sync(0xFFFFFFFFu, me.r, j);
        // (a cut outside the row is recorded and the child copies p1)
        const bool cross = __shfl_sync(0xFFFFFFFFu, (int)me.cross, j) != 0 &&
                           FFS_DCHECK(l >= 0 && l <= r && r < n, kCheckCut);
        if (!cross) {
            const int4 *s4 = reinterpret_cast<const int4 *>(p1);
            int4 *d4 = reinterpret_cast<int4 *>(child);
            for (int k = lane; k < (ld >> 3); k += 32) d4[k] = s4[k];
            __syncwarp();
            continue;
        }
        const int nb = (n + 7) >> 3;
        const int4 *p1v = reinterpret_cast<const int4 *>(p1);
        const int4 *p2v = reinterpret_cast<const int4 *>(p2);
        int4 *cv = reinterpret_cast<int4 *>(child);
        const int4 zero4 = make_int4(0, 0, 0, 0);
        // rows of at most 64 blocks (512 genes): every block of both parents in
        // registers first (block q with lane q % 32), so that a child costs one
        // trip to memory instead of one per pass
        const bool regs = nb <= 64;   // warp-uniform
        int4 a0 = zero4, a1 = zero4, c0 = zero4, c1 = zero4;
        if (regs) {
            if (lane < nb) {
                a0 = p1v[lane];
                c0 = p2v[lane];
            }
            if (lane + 32 < nb) {
                a1 = p1v[lane + 32];
                c1 = p2v[lane + 32];
            }
        }
        for (int w = lane; 4 * w < words; w += 32) reinterpret_cast<uint4 *>(mark)[w] = make_uint4(0u, 0u, 0u, 0u);
        __syncwarp();
        // the segment p1[l..r], eight genes (one 16-byte block) per lane
        auto segment_block = [&](int q, const int4 &v) {
            const uint32_t wv[4] = {(uint32_t)v.x, (uint32_t)v.y, (uint32_t)v.z, (uint32_t)v.w};
            const bool full = 8 * q >= l && 8 * q + 7 <= r;
            if (full) cv[q] = v;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = 8 * q + u;
                if (idx >= l && idx <= r) {
                    const int g = (int)(int16_t)(wv[u >> 1] >> (16 * (u & 1)));
                    if (!full) child[idx] = (int16_t)g;
                    if ((unsigned)g < (unsigned)n) flag[g] = 1u;
                }
            }
        };
        if (regs) {
            if (lane < nb && 8 * lane <= r && 8 * lane + 7 >= l) segment_block(lane, a0);
            if (lane + 32 < nb && 8 * (lane + 32) <= r && 8 * (lane + 32) + 7 >= l) segment_block(lane + 32, a1);
        } else {
            for (int q = (l >> 3) + lane; q <= (r >> 3); q += 32) segment_block(q, p1v[q]);
        }
        __syncwarp();
        // p2 from position start = r + 1 onward cyclically, in 16-byte blocks:
        // pass t takes block (start / 8 + t) mod nb; pass 0 keeps the genes
        // from start on, pass nb those before start.  A lane's taken genes
        // get consecutive ranks after a warp prefix sum of the lanes' counts.
        const int start = (r + 1 == n) ? 0 : r + 1;
        const int b0 = start >> 3;
        int placed = 0;
        for (int t0 = 0; t0 <= nb; t0 += 32) {
            const int t = t0 + lane;
            int q = b0 + t;
            if (q >= nb) q -= nb;
            int4 v = zero4;
            if (regs) {   // block q from the lane that holds it (every lane shuffles)
                const int src = q & 31;
                int4 w0, w1;
                w0.x = __shfl_sync(0xFFFFFFFFu, c0.x, src);
                w0.y = __shfl_sync(0xFFFFFFFFu, c0.y, src);
                w0.z = __shfl_sync(0xFFFFFFFFu, c0.z, src);
                w0.w = __shfl_sync(0xFFFFFFFFu, c0.w, src);
                w1.x = __shfl_sync(0xFFFFFFFFu, c1.x, src);
                w1.y = __shfl_sync(0xFFFFFFFFu, c1.y, src);
                w1.z = __shfl_sync(0xFFFFFFFFu, c1.z, src);
                w1.w = __shfl_sync(0xFFFFFFFFu, c1.w, src);
                if (t <= nb) v = q >= 32 ? w1 : w0;
            } else if (t <= nb) {
                v = p2v[q];
            }
            const uint32_t wv[4] = {(uint32_t)v.x, (uint32_t)v.y, (uint32_t)v.z, (uint32_t)v.w};
            const int lo = t == 0 ? start : 0, hi = t == nb ? start : n;   // natural indices kept in this pass
            unsigned take = 0u;
            int gv[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = 8 * q + u;
                const int g = (int)(int16_t)(wv[u >> 1] >> (16 * (u & 1)));
                gv[u] = g;
                const bool in_seg = (unsigned)g < (unsigned)n && flag[g] != 0u;
                if (t <= nb && idx >= lo && idx < hi && !in_seg) take |= 1u << u;
            }
            const int cnt = __popc(take);
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                if (lane >= o) incl += y;
            }
            const int first = start + placed + incl - cnt;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if ((take >> u) & 1u) {
                    int pos = first + __popc(take & ((1u << u) - 1u));
                    if (pos >= n) pos -= n;
                    if (FFS_DCHECK(pos >= 0 && pos < n, kCheckWrite)) child[pos] = (int16_t)gv[u];
                }
            }
            placed += __shfl_sync(0xFFFFFFFFu, incl, 31);
        }
        __syncwarp();
    }
}

// Two children at a time, one per 16-lane half of the warp, for rows of at
// most 120 genes (nb = ceil(n / 8) blocks, nb + 1 <= 16 passes of the p2
// sweep): the construction of warp_build_children, with shuffles and the
// prefix sum confined to each half and a mark of mark_words(n) words per
// half (`mark` holds two).  Children are identical to warp_build_children's.
__host__ __device__ inline bool pairs_build_fits(int n) { return ((n + 7) >> 3) + 1 <= 16; }

__device__ __forceinline__ void warp_build_children_pairs(const ChildJob &me, int n, int ld, uint32_t *mark)
{
    const int lane = threadIdx.x & 31, half = lane >> 4, hl = lane & 15;
    const int words = mark_words(n);
    uint8_t *flag = reinterpret_cast<uint8_t *>(mark + half * words);
    const int nb = (n + 7) >> 3;
    const int4 zero4 = make_int4(0, 0, 0, 0);
    unsigned todo = __ballot_sync(0xFFFFFFFFu, me.active);
    while (todo) {
        // the next two jobs: the lower half takes the first, the upper half
        // the second (and idles when there is none)
        const int j0 = __ffs(todo) - 1;
        todo &= todo - 1u;
        int j1 = -1;
        if (todo) {
            j1 = __ffs(todo) - 1;
            todo &= todo - 1u;
        }
        const bool mine = half == 0 || j1 >= 0;
        const int j = (half && j1 >= 0) ? j1 : j0;
        const int16_t *p1 = (const int16_t *)__shfl_sync(0xFFFFFFFFu, (unsigned long long)me.p1, j);
        const int16_t *p2 = (const int16_t *)__shfl_sync(0xFFFFFFFFu, (unsigned long long)me.p2, j);
        int16_t *child = (int16_t *)__shfl_sync(0xFFFFFFFFu, (unsigned long long)me.child, j);
        const int l = __shfl_sync(0xFFFFFFFFu, me.l, j);
        const int r = __shfl_sync(0xFFFFFFFFu, me.r, j);
        // (a cut outside the row is recorded and the child copies p1)
        const bool cross = __shfl_sync(0xFFFFFFFFu, (int)me.cross, j) != 0 &&
                           FFS_DCHECK(l >= 0 && l <= r && r < n, kCheckCut);
        const int4 *p1v = reinterpret_cast<const int4 *>(p1);
        const int4 *p2v = reinterpret_cast<const int4 *>(p2);
        int4 *cv = reinterpret_cast<int4 *>(child);
        if (mine && !cross)
            for (int k = hl; k < (ld >> 3); k += 16) cv[k] = p1v[k];
        const bool xo = mine && cross;
        // both parents' blocks in registers (block q with lane q of the half)
        int4 a0 = zero4, c0 = zero4;
        if (xo && hl < nb) {
            a0 = p1v[hl];
            c0 = p2v[hl];
        }
        if (xo)
            for (int w = hl; 4 * w < words; w += 16) reinterpret_cast<uint4 *>(flag)[w] = make_uint4(0u, 0u, 0u, 0u);
        __syncwarp();
        // the segment p1[l..r], eight genes (one 16-byte block) per lane
        if (xo && hl < nb && 8 * hl <= r && 8 * hl + 7 >= l) {
            const uint32_t wv[4] = {(uint32_t)a0.x, (uint32_t)a0.y, (uint32_t)a0.z, (uint32_t)a0.w};
            const bool full = 8 * hl >= l && 8 * hl + 7 <= r;
            if (full) cv[hl] = a0;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int idx = 8 * hl + u;
                if (idx >= l && idx <= r) {
                    const int g = (int)(int16_t)(wv[u >> 1] >> (16 * (u & 1)));
                    if (!full) child[idx] = (int16_t)g;
                    if ((unsigned)g < (unsigned)n) flag[g] = 1u;
                }
            }
        }
        __syncwarp();
        // p2 from position start = r + 1 onward cyclically: pass t (lane t of
        // the half) takes block (start / 8 + t) mod nb
        const int start = (r + 1 == n) ? 0 : r + 1;
        const int t = hl;
        int q = (start >> 3) + t;
        if (q >= nb) q -= nb;
        const int src = q & 15;   // lanes with t > nb read an ignored block
        int4 v;
        v.x = __shfl_sync(0xFFFFFFFFu, c0.x, src, 16);
        v.y = __shfl_sync(0xFFFFFFFFu, c0.y, src, 16);
        v.z = __shfl_sync(0xFFFFFFFFu, c0.z, src, 16);
        v.w = __shfl_sync(0xFFFFFFFFu, c0.w, src, 16);
        const bool pass = xo && t <= nb;
        const uint32_t wv[4] = {(uint32_t)v.x, (uint32_t)v.y, (uint32_t)v.z, (uint32_t)v.w};
        const int lo = t == 0 ? start : 0, hi = t == nb ? start : n;   // natural indices kept in this pass
        unsigned take = 0u;
        int gv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int idx = 8 * q + u;
            const int g = (int)(int16_t)(wv[u >> 1] >> (16 * (u & 1)));
            gv[u] = g;
            const bool in_seg = (unsigned)g < (unsigned)n && flag[g] != 0u;
            if (pass && idx >= lo && idx < hi && !in_seg) take |= 1u << u;
        }
        const int cnt = __popc(take);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 16; o <<= 1) {
            const int y = __shfl_up_sync(0xFFFFFFFFu, incl, o, 16);
            if (hl >= o) incl += y;
        }
        const int first = start + incl - cnt;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            if ((take >> u) & 1u) {
                int pos = first + __popc(take & ((1u << u) - 1u));
                if (pos >= n) pos -= n;
                if (FFS_DCHECK(pos >= 0 && pos < n, kCheckWrite)) child[pos] = (int16_t)gv[u];
            }
        }
        __syncwarp();
    }
}

// The FFS_DEBUG_CHECKS build's validity check of one row by one warp: every
// gene in [0, n), no gene twice (a bit per job in `bits`, (n + 31) / 32
// words of this warp's shared memory), and a makespan >= 0; a failure is
// recorded as kCheckPermutation.
__device__ __forceinline__ void warp_check_row(const int16_t *row, int n, int32_t ms, uint32_t *bits)
{
    const int lane = threadIdx.x & 31;
    const int words = (n + 31) >> 5;
    for (int w = lane; w < words; w += 32) bits[w] = 0u;
    __syncwarp();
    bool ok = ms >= 0;
    for (int i = lane; i < n; i += 32) {
        const int gj = row[i];
        if (gj < 0 || gj >= n) {
            ok = false;
        } else {
            const uint32_t bit = 1u << (gj & 31);
            if (atomicOr(&bits[gj >> 5], bit) & bit) ok = false;
        }
    }
    ok = __all_sync(0xFFFFFFFFu, ok);
    if (lane == 0) (void)FFS_DCHECK(ok, kCheckPermutation);
    __syncwarp();
}

// Warp-cooperative row copies: lane j's (src, dst) pair when `active`.  Four
// rows at a time, their loads issued before their stores (no destination row
// may overlap a source row of the same call).
__device__ __forceinline__ void warp_copy_rows(bool active, const int16_t *src, int16_t *dst, int ld)
{
    const int lane = threadIdx.x & 31;
    const int q = ld >> 3;
    unsigned todo = __ballot_sync(0xFFFFFFFFu, active);
    while (todo) {
        const int4 *s4[4];
        int4 *d4[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            s4[u] = nullptr;
            d4[u] = nullptr;
            if (todo) {   // warp-uniform
                const int j = __ffs(todo) - 1;
                todo &= todo - 1u;
                s4[u] = (const int4 *)__shfl_sync(0xFFFFFFFFu, (unsigned long long)src, j);
                d4[u] = (int4 *)__shfl_sync(0xFFFFFFFFu, (unsigned long long)dst, j);
            }
        }
        for (int k = lane; k < q; k += 32) {
            int4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (s4[u]) v[u] = s4[u][k];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                if (d4[u]) d4[u][k] = v[u];
        }
    }
    __syncwarp();
}


// Two rows per active lane (s0 -> d0, s1 -> d1), four lanes at a time: the
// loads of all eight rows are issued before their stores (no destination
// row may overlap a source row of the same call).
__device__ __forceinline__ void warp_copy_row_pairs(bool active, const int16_t *s0, int16_t *d0, const int16_t *s1,
                                                    int16_t *d1, int ld)
{
    const int lane = threadIdx.x & 31;
    const int q = ld >> 3;
    unsigned todo = __ballot_sync(0xFFFFFFFFu, active);
    while (todo) {
        const int4 *src[8];
        int4 *dst[8];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            src[2 * u] = src[2 * u + 1] = nullptr;
            dst[2 * u] = dst[2 * u + 1] = nullptr;
            if (todo) {   // warp-uniform
                const int j = __ffs(todo) - 1;
                todo &= todo - 1u;
                src[2 * u] = (const int4 *)__shfl_sync(0xFFFFFFFFu, (unsigned long long)s0, j);
                dst[2 * u] = (int4 *)__shfl_sync(0xFFFFFFFFu, (unsigned long long)d0, j);
                src[2 * u + 1] = (const int4 *)__shfl_sync(0xFFFFFFFFu, (unsigned long long)s1, j);
                dst[2 * u + 1] = (int4 *)__shfl_sync(0xFFFFFFFFu, (unsigned long long)d1, j);
            }
        }
        for (int k = lane; k < q; k += 32) {
            int4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (src[u]) v[u] = src[u][k];
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (dst[u]) dst[u][k] = v[u];
        }
    }
    __syncwarp();
}

// The breeding half of a cellular generation for the cell `c` of each lane
// (lanes with !valid only keep the warp in lock step): draws, two binary
// tournaments over the von Neumann neighbourhood (previous generation's
// makespans), order crossover, swap mutation.  The child is built in the
// cell's output row, or in `child_row` when that is given: then the cell
// itself is copied to its output row (row and makespan), which the decoding
// overwrites only if the child is better.  `wbits`: the warp's crossover
// mark (warp_build_children).
__device__ __forceinline__ void cellular_warp_breed(const IslandRef &ref, const GaScalars &g, int n, int c, bool valid,
                                                    int rows, int cols, int ld, uint32_t *wbits,
                                                    int16_t *child_row = nullptr)
{
    const int16_t *pin;
    const int32_t *msin;
    int16_t *pout;
    int32_t *msout;
    uint32_t gen;
    resolve(ref, pin, msin, pout, msout, gen);
    ChildJob job;
    job.active = valid;
    job.child = child_row ? child_row : pout + (int64_t)c * ld;
    job.p1 = job.p2 = pin;
    job.l = job.r = 0;
    job.cross = false;
    U4 b2{0, 0, 0, 0};
    bool mutate = false;
    if (valid) {
        const U4 b0 = draw_block(g.seed, kPurposeCellular, ref.island, gen, (uint32_t)c, 0u);
        const U4 b1 = draw_block(g.seed, kPurposeCellular, ref.island, gen, (uint32_t)c, 1u);
        b2 = draw_block(g.seed, kPurposeCellular, ref.island, gen, (uint32_t)c, 2u);
        const int r = c / cols, q = c - r * cols;
        const int up = ((r + rows - 1) % rows) * cols + q, down = ((r + 1) % rows) * cols + q;
        const int west = r * cols + (q + cols - 1) % cols, east = r * cols + (q + 1) % cols;
        auto slot = [&](uint32_t x) {
            const uint32_t k = uniform_below(x, 5u);
            return k == 0 ? c : k == 1 ? up : k == 2 ? down : k == 3 ? west : east;
        };
        int a = slot(b0.x), b = slot(b0.y);
        int par1 = (msin[b] < msin[a]) ? b : a;
        a = slot(b0.z);
        b = slot(b0.w);
        int par2 = (msin[b] < msin[a]) ? b : a;
        if (!FFS_DCHECK(par1 >= 0 && par1 < rows * cols && par2 >= 0 && par2 < rows * cols, kCheckParent))
            par1 = par2 = c;
        job.p1 = pin + (int64_t)par1 * ld;
        job.p2 = pin + (int64_t)par2 * ld;
        job.cross = fires(b1.x, g.cell_pc);
        const int u = (int)uniform_below(b1.y, (uint32_t)n), v = (int)uniform_below(b1.z, (uint32_t)n);
        job.l = min(u, v);
        job.r = max(u, v);
        mutate = fires(b1.w, g.cell_pm);
    }
    warp_build_children(job, n, ld, wbits);
    if (mutate) {
        int16_t *child = job.child;
        const int i = (int)uniform_below(b2.x, (uint32_t)n), j = (int)uniform_below(b2.y, (uint32_t)n);
        const int16_t t = child[i];
        child[i] = child[j];
        child[j] = t;
    }
    __syncwarp();
    if (child_row) {   // warp-uniform
        if (valid) msout[c] = msin[c];
        warp_copy_rows(valid, pin + (int64_t)c * ld, pout + (int64_t)c * ld, ld);
    }
}

// The other half: decode the child in the cell's output row and replace the
// cell iff the child is better (else the output row takes the old cell back).
__device__ __forceinline__ void cellular_warp_decode(const DecodeLayout &Ls, const GaScalars &g, const IslandRef &ref,
                                                     int c, bool valid, int ld, uint32_t *region, int T,
                                                     const uint16_t *tab, WarpStageState *wst)
{
    const int16_t *pin;
    const int32_t *msin;
    int16_t *pout;
    int32_t *msout;
    uint32_t gen;
    resolve(ref, pin, msin, pout, msout, gen);
    // lanes past the end decode a row of their island in lock step; nothing is written
    const int16_t *drow = valid ? pout + (int64_t)c * ld : pin + (int64_t)c * ld;
    const int32_t ms = decode_chromosome(Ls, drow, region, T, tab, wst);
    bool keep_old = false;
    if (valid) {
        const int32_t old = msin[c];
        const bool better = ms >= 0 && (g.replace_le ? (uint32_t)ms <= (uint32_t)old : (uint32_t)ms < (uint32_t)old);
        msout[c] = better ? ms : old;
        keep_old = !better;
    }
    warp_copy_rows(keep_old, pin + (int64_t)c * ld, pout + (int64_t)c * ld, ld);
}

// As cellular_warp_decode for a child bred into `child_row` (the cell was
// already copied to its output row): decode the child and, iff it is
// better, write it and its makespan over the copy.
__device__ __forceinline__ void cellular_warp_decode_child(const DecodeLayout &Ls, const GaScalars &g,
                                                           const IslandRef &ref, int c, bool valid, int ld,
                                                           const int16_t *child_row, uint32_t *region, int T,
                                                           const uint16_t *tab, WarpStageState *wst)
{
    const int16_t *pin;
    const int32_t *msin;
    int16_t *pout;
    int32_t *msout;
    uint32_t gen;
    resolve(ref, pin, msin, pout, msout, gen);
    // lanes past the end decode a row of their island in lock step; nothing is written
    const int32_t ms = decode_chromosome(Ls, valid ? child_row : pin + (int64_t)c * ld, region, T, tab, wst);
    bool better = false;
    if (valid) {
        const int32_t old = msin[c];
        better = ms >= 0 && (g.replace_le ? (uint32_t)ms <= (uint32_t)old : (uint32_t)ms < (uint32_t)old);
        if (better) msout[c] = ms;
    }
    warp_copy_rows(better, child_row, pout + (int64_t)c * ld, ld);
}

// One cellular generation for the cell `c` of each lane: breeding, then
// decoding and replacement (see the two halves above).
__device__ __forceinline__ void cellular_warp_cells(const DecodeLayout &Ls, const GaScalars &g, const IslandRef &ref,
                                                    int c, bool valid, int rows, int cols, int ld, uint32_t *wbits,
                                                    uint32_t *region, int T, const uint16_t *tab,
                                                    WarpStageState *wst)
{
    cellular_warp_breed(ref, g, Ls.n, c, valid, rows, cols, ld, wbits);
    cellular_warp_decode(Ls, g, ref, c, valid, ld, region, T, tab, wst);
}

}  // namespace fgpu
