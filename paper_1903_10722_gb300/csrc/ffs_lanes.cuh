// ffs_lanes.cuh -- the stage-parallel decoder: one lane per stage of a
// chromosome, for decode launches too small to fill the GPU with one
// chromosome per lane.
//
// The list-scheduling decoder dispatches stage s's jobs in the order in
// which stage s - 1 completes them (ascending (completion, job) keys), and
// the keys stage s - 1 pops from its sorted machine array come out in exactly
// that order (a completion is later than the free time it replaced).  So the
// stages of one chromosome can run side by side: lane s of a group of S
// lanes owns stage s's machine keys; every step each lane takes the key its
// predecessor popped the step before (lane 0: the next gene) and dispatches
// it (pop the earliest machine, complete, insert); once all n jobs are
// dispatched it drains one key per step (inserting +inf) so that the next
// stage receives its last completions.  The first M_s keys a lane pops are
// its initial machines; from then on it emits a completion every step, so
// lane s + 1 receives its n jobs in the n consecutive steps from start_{s+1}
// = start_s + M_s + 1: the schedule is fixed in advance, and the group ends
// after start_{S-1} + n steps (about n + sum_s M_s) instead of n * S
// dispatches.  A warp decodes floor(32 / S) chromosomes.
// The completion key and the tie order are the one-lane decoder's
// (dispatch_pp), so every objective is identical.
#pragma once

#include "ffs_internal.cuh"

namespace fgpu {

// All 32 lanes of the warp call it together.
//   tab       shared address of the time table (stage s's row at tab + s * row_bytes)
//   genes     shared address of this lane's group's chromosome (n int16)
//   nS        n | S << 16
//   sM        this lane's stage (0xFF: no stage) | M_eff(s) << 8 | SH << 16
//   win       start_s | steps << 16: lane s receives its n jobs in the steps
//             [start_s, start_s + n), start_s = sum_{j<s} (M_eff(j) + 1), and
//             drains in the M_eff(s) steps after; the group is done after
//             steps = start_{S-1} + n (the schedule does not depend on the data)
//   rel, due  shared addresses of the release / due tables (0: none); wt the tardiness weight
// Returns, on the group's last-stage lane, the objective: the makespan plus
// wt x total tardiness, or -1 if a gene is outside [0, n).  Other lanes
// return 0.
template <int MM>
__device__ __noinline__ int32_t lane_decode(uint32_t tab, uint32_t row_bytes, uint32_t genes, uint32_t nS, uint32_t sM,
                                            uint32_t win, uint32_t rel, uint32_t due, uint32_t wt);

#ifdef FFS_LANES_BODIES
// Sorted insertion of x into f[1..MM-1] after f[0] is popped (x > f[0]).
template <int MM>
__device__ __forceinline__ void lane_insert(uint32_t (&f)[MM], uint32_t x)
{
    if constexpr (MM == 1) {
        f[0] = x;
    } else {
#pragma unroll
        for (int m = 0; m < MM - 1; ++m) {
            const uint32_t lo = (m == 0) ? x : max(f[m], x);
            f[m] = min(f[m + 1], lo);
        }
        f[MM - 1] = max(f[MM - 1], x);
    }
}

template <int MM>
__device__ __noinline__ int32_t lane_decode(uint32_t tab, uint32_t row_bytes, uint32_t genes, uint32_t nS, uint32_t sM,
                                            uint32_t win, uint32_t rel, uint32_t due, uint32_t wt)
{
    const int lane = threadIdx.x & 31;
    const int n = (int)(nS & 0xFFFFu), S = (int)(nS >> 16);
    const int s = (int)(sM & 0xFFu), Ms = (int)((sM >> 8) & 0xFFu);
    const uint32_t SH = sM >> 16;
    const int start = (int)(win & 0xFFFFu), steps = (int)(win >> 16);
    // 2^SH through an opaque move (p * 2^SH + t stays one multiply-add)
    uint32_t mulSH;
    asm("mov.b32 %0, %1;" : "=r"(mulSH) : "r"(1u << SH));
    const uint32_t lowmask = mulSH - 1u, idmask = lowmask & ~1u;
    const bool idle = s == 0xFF;
    const bool first = s == 0, last = !idle && s == S - 1;
    const uint32_t prow = tab + (idle ? 0u : (uint32_t)s * row_bytes);
    // window bounds of this lane (an idle lane's windows are empty)
    const int d_end = idle ? -1 : n, r_end = idle || last ? -1 : n + Ms;
    uint32_t f[MM];
#pragma unroll
    for (int m = 0; m < MM; ++m) f[m] = m < Ms ? 0u : 0xFFFFFFFFu;
    uint32_t mk = 0u, tard = 0u;
    bool bad = false;
    // stage 0's key for a step is read one step ahead, by every lane (an
    // index clamped to the row; only stage-0 lanes use it), so that the gene
    // and release loads stay off the step's dependency chain
    auto gene_key = [&](int t) -> uint32_t {
        const int gi = t < n ? t : n - 1;
        const uint32_t g0 = (uint32_t)(int32_t)(int16_t)lds16(genes + 2u * (uint32_t)gi);
        const bool out = g0 >= (uint32_t)n;
        bad = bad || (out && first && t < n);
        const uint32_t k = ((out ? 0u : g0) + 1u) << 1;
        return rel ? k | (lds32(rel + (k << 1)) << SH) : k;   // stage-1 ready time R_j
    };
    // software-pipelined: step t first sends its emission (the heap's
    // minimum before its insert) and fetches step t + 1's input key and
    // processing time, then completes and inserts its own job while those
    // loads are in flight
    uint32_t in_t = first ? gene_key(0) : 0u;
    uint32_t p_t = lds16(prow + (in_t & idmask));
    for (int t = 0; t < steps; ++t) {
        const int r = t - start;
        const bool disp = r >= 0 && r < d_end;
        const bool drain = r >= n && r < r_end;
        const uint32_t f0 = f[0];
        const uint32_t emit = (disp || drain) ? f0 : 0u;
        const uint32_t recv = __shfl_up_sync(0xFFFFFFFFu, emit, 1);   // step t + 1's input
        const uint32_t k0 = gene_key(t + 1);
        const uint32_t in_next = first ? k0 : recv;
        const uint32_t p_next = lds16(prow + (in_next & idmask));
        const uint32_t c = p_t * mulSH + max((f0 & ~lowmask) | (in_t & lowmask), in_t);
        // branch-free: a dispatch inserts its completion, a drain +inf, and an
        // idle step f[0] itself (popping and re-inserting the minimum leaves
        // the sorted array as it was)
        const uint32_t x = disp ? c : (drain ? 0xFFFFFFFFu : f0);
        lane_insert<MM>(f, x);
        const bool fin = last && disp;   // a completion of the last stage
        mk = max(mk, fin ? c : 0u);
        if (due) tard += fin ? key_tardiness(c, due, SH, idmask) : 0u;   // `due` is the same in every lane
        in_t = in_next;
        p_t = p_next;
    }
    const int src = idle ? lane : lane - s;   // the group's stage-0 lane knows about bad genes
    const bool gbad = __shfl_sync(0xFFFFFFFFu, (int)bad, src) != 0;
    if (!last) return 0;
    return gbad ? -1 : (int32_t)((mk >> SH) + wt * tard);
}
#endif  // FFS_LANES_BODIES

// A block's setup for stage-parallel decoding: the instance's time table
// (and release / due tables) and its stage array in shared memory, then,
// for this lane, its group g and stage s, the stage's machine count, its
// window (start_s | steps << 16) and the shared addresses the decoder takes.
// Each warp's staged rows follow (rows: C rows of ld int16 per warp).
struct LaneSetup {
    uint32_t tab, row_bytes, rel, due, nS, win, Ms, rows_sa;
    uint32_t *rows;
    int g, s, C;
};

__device__ __forceinline__ LaneSetup lanes_block_setup(uint32_t *smem, int n, int S, int obj_words, int has_rel,
                                                       int has_due, const uint32_t *tab_g, const int32_t *stage_g,
                                                       int ld)
{
    LaneSetup u;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tw = table_words(n, S);
    stage_table(smem, tab_g, tw + obj_words);
    int32_t *st = reinterpret_cast<int32_t *>(smem + tw + obj_words);
    for (int i = threadIdx.x; i < S; i += blockDim.x) st[i] = stage_g[i];
    u.C = 32 / S;
    u.rows = smem + round_up(tw + obj_words + S, 4) + warp * (u.C * ld / 2);
    __syncthreads();
    u.tab = tc::smem_u32(smem);
    u.row_bytes = (uint32_t)table_row_halves(n) * 2u;
    const uint32_t objt = u.tab + (uint32_t)tw * 4u;
    u.rel = has_rel ? objt : 0u;
    u.due = has_due ? objt + (uint32_t)obj_words * 2u : 0u;
    u.g = lane / S;
    u.s = lane - u.g * S;
    u.Ms = u.g < u.C ? (uint32_t)st[u.s] : 1u;
    // start_s = sum_{j<s} (M_j + 1); the group ends after start_{S-1} + n steps
    int start = 0, last_start = 0;
    for (int j = 0; j < S - 1; ++j) {
        if (j < u.s) start += st[j] + 1;
        last_start += st[j] + 1;
    }
    u.win = (uint32_t)start | ((uint32_t)(last_start + n) << 16);
    u.nS = (uint32_t)n | ((uint32_t)S << 16);
    u.rows_sa = tc::smem_u32(u.rows);
    return u;
}

// lane_decode for the smallest compiled heap size >= MM (1..16, then 32).
__device__ __forceinline__ int32_t lane_decode_dispatch(int MM, uint32_t tab, uint32_t row_bytes, uint32_t genes,
                                                        uint32_t nS, uint32_t sM, uint32_t win, uint32_t rel,
                                                        uint32_t due, uint32_t wt)
{
#define FFS_LCASE(K) \
    case K: return lane_decode<K>(tab, row_bytes, genes, nS, sM, win, rel, due, wt);
    switch (MM) {
        FFS_LCASE(1) FFS_LCASE(2) FFS_LCASE(3) FFS_LCASE(4) FFS_LCASE(5) FFS_LCASE(6) FFS_LCASE(7) FFS_LCASE(8)
        FFS_LCASE(9) FFS_LCASE(10) FFS_LCASE(11) FFS_LCASE(12) FFS_LCASE(13) FFS_LCASE(14) FFS_LCASE(15)
        FFS_LCASE(16)
        default: return lane_decode<kMaxM>(tab, row_bytes, genes, nS, sM, win, rel, due, wt);
    }
#undef FFS_LCASE
}

}  // namespace fgpu
