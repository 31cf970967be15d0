// ffs_device.cuh -- device-side building blocks of the FFS island GA for
// sm_103a: Philox4x32-10 draws, the list-scheduling decoder, and the genetic
// operators.  Included by the library's .cu files only.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fgpu {

constexpr int kMaxM = 32;        // machines per stage after clamping to n
constexpr int kMaxStages = 64;

// Purpose codes of the Philox counter's fourth word (bits 24..31):
// surrogate candidate k of a cell uses kPurposeSurrogateBase + k (k < 16),
// the surrogate's training-batch sampling kPurposeTrainSample.
constexpr uint32_t kPurposeInit = 1, kPurposeCellular = 2, kPurposePseudo = 3,
                   kPurposeTrainSample = 15, kPurposeSurrogateBase = 16;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011): ten rounds of two
// 32x32->64 multiplies of the even counter words, the high halves xor'ed
// into the odd words with the round key, the key bumped by the Weyl pair.
// ---------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__device__ __forceinline__ U4 philox4x32_10(U4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = U4{hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0};
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// Block `blk` (draws 4*blk .. 4*blk+3) of the stream (seed, purpose, island,
// generation, cell).
__device__ __forceinline__ U4 draw_block(uint64_t seed, uint32_t purpose, uint32_t island,
                                         uint32_t generation, uint32_t cell, uint32_t blk)
{
    return philox4x32_10(U4{blk, cell, generation, (island & 0xFFFFFFu) | (purpose << 24)},
                         (uint32_t)seed, (uint32_t)(seed >> 32));
}

__device__ __forceinline__ uint32_t uniform_below(uint32_t x, uint32_t k) { return __umulhi(x, k); }
__device__ __forceinline__ bool fires(uint32_t x, uint64_t threshold) { return (uint64_t)x < threshold; }

// ---------------------------------------------------------------------------
// Decoder.
//
// A chromosome is decoded stage after stage by list scheduling.  The M
// machine free times of a stage live in registers as a sorted array of
// 32-bit keys  key = time << SH | (job + 1) << 1  (SH = bits(n) + 1); the
// initial free times are key 0.  Dispatching a job pops the smallest key f0
// (the earliest-free machine; among equal free times any choice gives the
// same start time, so the makespan is the one of the lowest-index rule) and
// pushes the job's completion key.  Because processing times are >= 1, the
// popped keys leave in ascending (time, job) order: after the first M
// (initial) pops, the pops of stage s are exactly stage s's completions
// sorted by (completion, job) -- the dispatch order of stage s+1 -- and the
// M keys left at the end complete that order.  So each stage streams its
// input keys from a small per-thread buffer and writes its output keys back
// in place, and no sort is needed.
//
// To bound shared memory for long chromosomes, the jobs flow through the
// stages in rounds of at most B keys: a stage consumes what the previous
// stage emitted this round; its heap is saved in shared memory between
// rounds.  Per-thread shared words: sum_s M_s (heaps, skipped when B >= n)
// + B (buffer), thread-interleaved (word w of thread t at w * T + t).
// ---------------------------------------------------------------------------
struct DecodeLayout {
    int32_t n, S, SH;
    uint32_t mulSH;        // 1 << SH
    int32_t B;             // keys per round (multiple of 8)
    int32_t single;        // 1 if B >= n: one round, heaps stay in registers
    int32_t heap_words;    // sum of M_s (0 when single)
    int32_t thread_words;  // words per thread in the interleaved region
    const int32_t *M;        // [S] machines per stage (clamped to n), shared memory
    const int32_t *heap_off; // [S] word offset of each stage's heap, shared memory
};

// Shared-memory table of processing times (uint16): row s holds n + 1
// entries (padded to an even count), entry j + 1 = p[j][s] (entry 0 = 0), so
// the low bits of a key, (job + 1) << 1, are the byte offset of the job's entry.
__device__ __forceinline__ uint32_t lds_u16(const uint16_t *row, uint32_t byte_off)
{
    return *reinterpret_cast<const uint16_t *>(reinterpret_cast<const char *>(row) + byte_off);
}

__host__ __device__ inline int table_row_halves(int n) { return (n + 2) & ~1; }

// One dispatch: f[] sorted ascending, pops f[0], inserts the completion key
// of the job `in` whose processing time at this stage is p:
// completion = max(machine free, release) + p, carrying the job's id.
template <int M>
__device__ __forceinline__ uint32_t dispatch_pp(uint32_t (&f)[M], uint32_t in, uint32_t p, uint32_t lowmask,
                                                uint32_t mulSH)
{
    const uint32_t f0 = f[0];
    // start = max(machine free, release); keep the incoming job id.
    const uint32_t u = (f0 & ~lowmask) | (in & lowmask);
    const uint32_t x = p * mulSH + max(u, in);
    if constexpr (M == 1) {
        f[0] = x;
    } else {
        // sorted insertion of x into f[1..M-1] (x > f[0])
#pragma unroll
        for (int m = 0; m < M - 1; ++m) {
            const uint32_t lo = (m == 0) ? x : max(f[m], x);
            f[m] = min(f[m + 1], lo);
        }
        f[M - 1] = max(f[M - 1], x);
    }
    return f0;
}

template <int M>
__device__ __forceinline__ uint32_t dispatch(uint32_t (&f)[M], uint32_t in, const uint16_t *prow,
                                             uint32_t lowmask, uint32_t mulSH)
{
    return dispatch_pp<M>(f, in, lds_u16(prow, in & lowmask), lowmask, mulSH);
}

// Per-warp round bookkeeping lives in shared memory (identical in all lanes).
struct WarpStageState {
    int32_t dispatched;
    int32_t flushed;
};

// Run one stage for one round.
//   FIRST: inputs are the chromosome's genes (global int16), else buf.
//   EMIT : write popped keys to buf (every stage but the last).
// Returns the number of keys written to buf this round.
template <int M, bool FIRST, bool EMIT>
__device__ __forceinline__ int stage_round(const DecodeLayout &L, uint32_t *__restrict__ heap,
                                           uint32_t *__restrict__ buf, const uint16_t *prow,
                                           const int16_t *__restrict__ genes, int T, int d0, int cnt,
                                           uint32_t lowmask, bool &bad_gene, uint32_t *last_key,
                                           int &flushed_out)
{
    uint32_t f[M];
    if (d0 > 0 && !L.single) {
#pragma unroll
        for (int m = 0; m < M; ++m) f[m] = heap[m * T];
    } else {
#pragma unroll
        for (int m = 0; m < M; ++m) f[m] = 0u;
    }
    int skip = M - d0;
    skip = skip < 0 ? 0 : (skip > cnt ? cnt : skip);
    int w = 0;
    if constexpr (FIRST) {
        // genes arrive 8 per 16-byte load, one load ahead; cnt is a multiple of 8
        // except at the tail (rows are padded to 8 genes, so the load stays in the row)
        const int4 *g4 = reinterpret_cast<const int4 *>(genes);
        const uint32_t n = (uint32_t)L.n;
        int4 vnext = g4[0];
        for (int i0 = 0; i0 < cnt; i0 += 8) {
            const int4 v = vnext;
            if (i0 + 8 < cnt) vnext = g4[(i0 >> 3) + 1];
            const uint32_t words[4] = {(uint32_t)v.x, (uint32_t)v.y, (uint32_t)v.z, (uint32_t)v.w};
#pragma unroll
            for (int h = 0; h < 8; ++h) {
                if (i0 + h < cnt) {
                    uint32_t g = (h & 1) ? (words[h >> 1] >> 16) : (words[h >> 1] & 0xFFFFu);
                    g = (uint32_t)(int32_t)(int16_t)g;
                    if (g >= n) { bad_gene = true; g = 0; }
                    const uint32_t in = (g + 1u) << 1;
                    const uint32_t popped = dispatch<M>(f, in, prow, lowmask, L.mulSH);
                    if constexpr (EMIT) {
                        if (i0 + h >= skip) { buf[w * T] = popped; ++w; }
                    }
                }
            }
        }
    } else {
        // The next key and its processing time are loaded one step ahead: the
        // store of step i goes to slot i - skip <= i, never to slot i + 1.
        // Slot cnt may be read (the region has one spare word per thread).
        const uint32_t idmask = lowmask & ~1u;
        const uint32_t mulSH = L.mulSH;
        uint32_t in = buf[0];
        uint32_t pp = lds_u16(prow, in & idmask);
        int i = 0;
        for (; i < skip; ++i) {
            const uint32_t in_n = buf[(i + 1) * T];
            const uint32_t pp_n = lds_u16(prow, in_n & idmask);
            (void)dispatch_pp<M>(f, in, pp, lowmask, mulSH);
            in = in_n;
            pp = pp_n;
        }
#pragma unroll 4
        for (; i < cnt; ++i) {
            const uint32_t in_n = buf[(i + 1) * T];
            const uint32_t pp_n = lds_u16(prow, in_n & idmask);
            const uint32_t popped = dispatch_pp<M>(f, in, pp, lowmask, mulSH);
            if constexpr (EMIT) buf[(i - skip) * T] = popped;
            in = in_n;
            pp = pp_n;
        }
        if constexpr (EMIT) w = cnt - skip;
    }
    const int d1 = d0 + cnt;
    flushed_out = 0;
    if constexpr (EMIT) {
        if (d1 == L.n && L.B - w >= M) {
            // stage complete and the whole heap fits in this round: flush from registers
#pragma unroll
            for (int m = 0; m < M; ++m) buf[(w + m) * T] = f[m];
            w += M;
            flushed_out = M;
        } else if (!L.single) {
#pragma unroll
            for (int m = 0; m < M; ++m) heap[m * T] = f[m];
        }
    } else {
        if (!L.single) {
#pragma unroll
            for (int m = 0; m < M; ++m) heap[m * T] = f[m];
        }
        *last_key = f[M - 1];
    }
    return w;
}

template <bool FIRST, bool EMIT>
__device__ __forceinline__ int stage_round_dispatch(int M, const DecodeLayout &L, uint32_t *heap,
                                                    uint32_t *buf, const uint16_t *prow,
                                                    const int16_t *genes, int T, int d0, int cnt,
                                                    uint32_t lowmask, bool &bad, uint32_t *last,
                                                    int &fl)
{
#define FFS_CASE(MM) \
    case MM: return stage_round<MM, FIRST, EMIT>(L, heap, buf, prow, genes, T, d0, cnt, lowmask, bad, last, fl);
    switch (M) {
        FFS_CASE(1) FFS_CASE(2) FFS_CASE(3) FFS_CASE(4) FFS_CASE(5) FFS_CASE(6) FFS_CASE(7)
        FFS_CASE(8) FFS_CASE(9) FFS_CASE(10) FFS_CASE(11) FFS_CASE(12) FFS_CASE(13) FFS_CASE(14)
        FFS_CASE(15) FFS_CASE(16) FFS_CASE(17) FFS_CASE(18) FFS_CASE(19) FFS_CASE(20)
        FFS_CASE(21) FFS_CASE(22) FFS_CASE(23) FFS_CASE(24) FFS_CASE(25) FFS_CASE(26)
        FFS_CASE(27) FFS_CASE(28) FFS_CASE(29) FFS_CASE(30) FFS_CASE(31) FFS_CASE(32)
        default: return 0;
    }
#undef FFS_CASE
}

// Decode one chromosome (row of genes in global memory, 16-byte aligned).
//   region: this thread's interleaved shared words (base + tid), stride T.
//   ptab  : shared uint16 table, row s at ptab + s * table_row_halves(n).
//   wst   : this warp's per-stage state, S entries (shared).
// All lanes of a warp must call this together for the same instance.
// Returns the makespan, or -1 if a gene is outside [0, n).
__device__ __forceinline__ int32_t decode_chromosome(const DecodeLayout &L, const int16_t *row,
                                                     uint32_t *region, int T, const uint16_t *ptab,
                                                     WarpStageState *wst)
{
    const int n = L.n, S = L.S;
    const uint32_t lowmask = (1u << L.SH) - 1u;
    uint32_t *buf = region + L.heap_words * T;
    // Every buffer slot holds a valid key (or 0) before the one-ahead reads
    // can touch it: clear the buffer and its spare slot.
    for (int w = 0; w <= L.B; ++w) buf[w * T] = 0u;
    bool bad = false;
    uint32_t last_key = 0;
    const int lane = threadIdx.x & 31;
    if (lane < S) { wst[lane].dispatched = 0; wst[lane].flushed = 0; }
    for (int s = 32 + lane; s < S; s += 32) { wst[s].dispatched = 0; wst[s].flushed = 0; }
    __syncwarp();
    // Every round moves stage 0 forward by B jobs or some stage's flush by
    // up to B keys; this bound is never reached by a correct schedule.
    const int max_rounds = (n + L.B - 1) / L.B + S * (kMaxM / 8 + 2) + 2;
    int s_lo = 0;   // stages before s_lo have dispatched and emitted everything
    for (int round = 0; round < max_rounds; ++round) {
        int avail = 0;  // keys in buf for the next stage
        for (int s = s_lo; s < S; ++s) {
            const int M = L.M[s];
            const int d0 = wst[s].dispatched;
            const int cnt = (s == 0) ? min(L.B, n - d0) : avail;
            const uint16_t *prow = ptab + s * table_row_halves(n);
            uint32_t *heap = region + L.heap_off[s] * T;
            const bool last = (s == S - 1);
            int w = 0, fl = 0;
            if (cnt > 0) {
                if (s == 0) {
                    if (last)
                        w = stage_round_dispatch<true, false>(M, L, heap, buf, prow, row + d0, T, d0, cnt,
                                                              lowmask, bad, &last_key, fl);
                    else
                        w = stage_round_dispatch<true, true>(M, L, heap, buf, prow, row + d0, T, d0, cnt,
                                                             lowmask, bad, &last_key, fl);
                } else {
                    if (last)
                        w = stage_round_dispatch<false, false>(M, L, heap, buf, prow, nullptr, T, d0, cnt,
                                                               lowmask, bad, &last_key, fl);
                    else
                        w = stage_round_dispatch<false, true>(M, L, heap, buf, prow, nullptr, T, d0, cnt,
                                                              lowmask, bad, &last_key, fl);
                }
            }
            const int d1 = d0 + cnt;
            int flushed = wst[s].flushed + fl;
            if (!last && d1 == n && flushed < M) {
                // finish (part of) the flush from the saved heap
                const int room = L.B - w;
                const int take = min(room, M - flushed);
                for (int t = 0; t < take; ++t) buf[(w + t) * T] = heap[(flushed + t) * T];
                w += take;
                flushed += take;
            }
            __syncwarp();
            if (lane == 0) { wst[s].dispatched = d1; wst[s].flushed = flushed; }
            __syncwarp();
            avail = w;
            const bool done = d1 == n && (last || flushed == M);
            if (done && s == s_lo) ++s_lo;
            // nothing reaches later stages this round unless this one is finished
            if (avail == 0 && !done) break;
        }
        if (wst[S - 1].dispatched >= n) break;
    }
    __syncwarp();
    if (bad) return -1;
    if (!L.single) last_key = region[(L.heap_off[S - 1] + L.M[S - 1] - 1) * T];
    return (int32_t)(last_key >> L.SH);
}

// Copy the instance's processing-time table (global, already laid out as
// the shared table) into shared memory; all threads of the block take part.
__device__ __forceinline__ void stage_table(uint32_t *dst, const uint32_t *src, int words)
{
    const int w4 = words >> 2;
    const int4 *s4 = reinterpret_cast<const int4 *>(src);
    int4 *d4 = reinterpret_cast<int4 *>(dst);
    for (int i = threadIdx.x; i < w4; i += blockDim.x) d4[i] = __ldg(s4 + i);
    for (int i = (w4 << 2) + threadIdx.x; i < words; i += blockDim.x) dst[i] = __ldg(src + i);
}

}  // namespace fgpu
