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
    int32_t pairs;         // 1: stages run two at a time, interleaved (see pair_round)
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
// Scalars of a round passed by value to the per-round functions, which are
// kept out of line (one call per stage and round, not per job): each is a
// small function for the compiler, instead of every instantiation inlined
// into one giant kernel.
struct RoundIn {
    int n, B, single;
    uint32_t mulSH, lowmask;
};

struct StageOut {
    int w;              // keys written to buf
    int flushed;        // heap keys flushed from registers this round
    uint32_t last_key;  // last stage: the largest key of its heap
    int bad;            // a gene outside [0, n) was read
};

// The heap holds Mr <= M real entries; slots from Mr up hold maximal keys,
// which never pop and never move (used when M is the 32-slot catch-all).
template <int M, bool FIRST, bool EMIT>
__device__ __noinline__ StageOut stage_round(RoundIn L, uint32_t *__restrict__ heap, uint32_t *__restrict__ buf,
                                             const uint16_t *prow, const int16_t *__restrict__ genes, int T, int d0,
                                             int cnt, int Mr)
{
    const uint32_t lowmask = L.lowmask;
    bool bad_gene = false;
    StageOut out{0, 0, 0u, 0};
    uint32_t f[M];
#pragma unroll
    for (int m = 0; m < M; ++m) f[m] = m < Mr ? ((d0 > 0 && !L.single) ? heap[m * T] : 0u) : 0xFFFFFFFFu;
    int skip = Mr - d0;
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
    if constexpr (EMIT) {
        if (d1 == L.n && L.B - w >= Mr) {
            // stage complete and the whole heap fits in this round: flush from registers
#pragma unroll
            for (int m = 0; m < M; ++m)
                if (m < Mr) buf[(w + m) * T] = f[m];
            w += Mr;
            out.flushed = Mr;
        } else if (!L.single) {
#pragma unroll
            for (int m = 0; m < M; ++m)
                if (m < Mr) heap[m * T] = f[m];
        }
    } else {
        if (!L.single) {
#pragma unroll
            for (int m = 0; m < M; ++m)
                if (m < Mr) heap[m * T] = f[m];
        }
        uint32_t lk = f[0];
#pragma unroll
        for (int m = 1; m < M; ++m)
            if (m == Mr - 1) lk = f[m];
        out.last_key = lk;
    }
    out.w = w;
    out.bad = bad_gene ? 1 : 0;
    return out;
}

template <bool FIRST, bool EMIT>
__device__ __forceinline__ int stage_round_dispatch(int M, const DecodeLayout &L, uint32_t *heap,
                                                    uint32_t *buf, const uint16_t *prow,
                                                    const int16_t *genes, int T, int d0, int cnt,
                                                    uint32_t lowmask, bool &bad, uint32_t *last,
                                                    int &fl)
{
    const RoundIn R{L.n, L.B, L.single, L.mulSH, lowmask};
    StageOut o{0, 0, 0u, 0};
#define FFS_CASE(MM) \
    case MM: o = stage_round<MM, FIRST, EMIT>(R, heap, buf, prow, genes, T, d0, cnt, M); break;
    switch (M) {
        FFS_CASE(1) FFS_CASE(2) FFS_CASE(3) FFS_CASE(4) FFS_CASE(5) FFS_CASE(6) FFS_CASE(7)
        FFS_CASE(8) FFS_CASE(9) FFS_CASE(10) FFS_CASE(11) FFS_CASE(12) FFS_CASE(13) FFS_CASE(14)
        FFS_CASE(15) FFS_CASE(16)
        default: o = stage_round<kMaxM, FIRST, EMIT>(R, heap, buf, prow, genes, T, d0, cnt, M); break;
    }
#undef FFS_CASE
    if (o.bad) bad = true;
    fl = o.flushed;
    if (!EMIT) *last = o.last_key;
    return o.w;
}

// ---------------------------------------------------------------------------
// Two stages a, b = a + 1 in one loop.  Stage a's pop at step i (its f[0]
// when the step starts) is stage b's input at the same step, so the two
// dispatch chains of a step are independent: twice the instruction-level
// parallelism per chromosome, and the key stream between a and b stays in
// registers.  Both heaps are held at the larger size M; the smaller one is
// padded with maximal keys, which never pop and never move.
//   Phase 1: a's first Ma dispatches pop initial keys (nothing reaches b).
//   Phase 2: b's first Mb dispatches pop initial keys (nothing emitted).
//   Phase 3: b's pops go to the buffer (in place: slot w <= slot i).
// When a has dispatched all n jobs its heap flows into b, and when b has,
// b's heap flows to the buffer, at most as many keys as the buffer holds
// this round (the rest in later rounds, from the saved heaps).
// ---------------------------------------------------------------------------
struct PairOut {
    int w, da1, fa1, db1, fb1;
    uint32_t last_key;
};

template <int M, bool EMIT_B>
__device__ __noinline__ PairOut pair_round(RoundIn L, uint32_t *__restrict__ heap_a, uint32_t *__restrict__ heap_b,
                                           uint32_t *__restrict__ buf, const uint16_t *prow_a, const uint16_t *prow_b,
                                           int T, int Ma, int Mb, int da0, int fa0, int db0, int fb0, int cnt)
{
    const uint32_t lowmask = L.lowmask;
    const uint32_t idmask = lowmask & ~1u, mulSH = L.mulSH;
    int da1, fa1, db1, fb1;
    uint32_t last_key_out = 0u;
    const bool chunked = !L.single;
    const int n = L.n;
    uint32_t fa[M], fb[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        fa[m] = m < Ma ? ((chunked && da0 > 0) ? heap_a[m * T] : 0u) : 0xFFFFFFFFu;
        fb[m] = m < Mb ? ((chunked && db0 > 0) ? heap_b[m * T] : 0u) : 0xFFFFFFFFu;
    }
    int w = 0, db = db0, i = 0;
    int skip_a = Ma - da0;
    skip_a = skip_a < 0 ? 0 : (skip_a > cnt ? cnt : skip_a);
    uint32_t in_a = buf[0];
    uint32_t pp_a = lds_u16(prow_a, in_a & idmask);
    for (; i < skip_a; ++i) {
        const uint32_t in_n = buf[(i + 1) * T];
        const uint32_t pp_n = lds_u16(prow_a, in_n & idmask);
        (void)dispatch_pp<M>(fa, in_a, pp_a, lowmask, mulSH);
        in_a = in_n;
        pp_a = pp_n;
    }
    uint32_t e = fa[0];
    uint32_t pp_e = lds_u16(prow_b, e & idmask);
    int end2 = i + (Mb - db > 0 ? Mb - db : 0);
    end2 = end2 > cnt ? cnt : end2;
    for (; i < end2; ++i) {
        const uint32_t in_n = buf[(i + 1) * T];
        const uint32_t pp_n = lds_u16(prow_a, in_n & idmask);
        (void)dispatch_pp<M>(fa, in_a, pp_a, lowmask, mulSH);
        (void)dispatch_pp<M>(fb, e, pp_e, lowmask, mulSH);
        ++db;
        e = fa[0];
        pp_e = lds_u16(prow_b, e & idmask);
        in_a = in_n;
        pp_a = pp_n;
    }
#pragma unroll 2
    for (; i < cnt; ++i) {
        const uint32_t in_n = buf[(i + 1) * T];
        const uint32_t pp_n = lds_u16(prow_a, in_n & idmask);
        (void)dispatch_pp<M>(fa, in_a, pp_a, lowmask, mulSH);
        const uint32_t pb = dispatch_pp<M>(fb, e, pp_e, lowmask, mulSH);
        ++db;
        if constexpr (EMIT_B) buf[(w++) * T] = pb;
        e = fa[0];
        pp_e = lds_u16(prow_b, e & idmask);
        in_a = in_n;
        pp_a = pp_n;
    }
    da1 = da0 + cnt;
    fa1 = fa0;
    if (chunked) {
#pragma unroll
        for (int m = 0; m < M; ++m)
            if (m < Ma) heap_a[m * T] = fa[m];
    }
    if (da1 == n && fa0 < Ma) {
        // a is complete: its remaining keys, in order, are b's last inputs
        if (!chunked) {
#pragma unroll
            for (int m = 0; m < M; ++m) {
                if (m < Ma) {
                    const uint32_t k = fa[m];
                    const uint32_t pb = dispatch_pp<M>(fb, k, lds_u16(prow_b, k & idmask), lowmask, mulSH);
                    if (EMIT_B && db >= Mb) buf[(w++) * T] = pb;
                    ++db;
                }
            }
            fa1 = Ma;
        } else {
            int take = Ma - fa0;
            if (EMIT_B && take > L.B - w) take = L.B - w;
            for (int t = 0; t < take; ++t) {
                const uint32_t k = heap_a[(fa0 + t) * T];
                const uint32_t pb = dispatch_pp<M>(fb, k, lds_u16(prow_b, k & idmask), lowmask, mulSH);
                if (EMIT_B && db >= Mb) buf[(w++) * T] = pb;
                ++db;
            }
            fa1 = fa0 + take;
        }
    }
    db1 = db;
    fb1 = fb0;
    if (chunked) {
#pragma unroll
        for (int m = 0; m < M; ++m)
            if (m < Mb) heap_b[m * T] = fb[m];
    }
    if constexpr (EMIT_B) {
        if (db1 == n && fb0 < Mb) {
            if (!chunked) {
#pragma unroll
                for (int m = 0; m < M; ++m)
                    if (m < Mb) buf[(w++) * T] = fb[m];
                fb1 = Mb;
            } else {
                int take = Mb - fb0;
                if (take > L.B - w) take = L.B - w;
                for (int t = 0; t < take; ++t) buf[(w + t) * T] = heap_b[(fb0 + t) * T];
                w += take;
                fb1 = fb0 + take;
            }
        }
    } else {
        uint32_t lk = fb[0];
#pragma unroll
        for (int m = 1; m < M; ++m)
            if (m == Mb - 1) lk = fb[m];
        last_key_out = lk;
    }
    return PairOut{w, da1, fa1, db1, fb1, last_key_out};
}

template <bool EMIT_B>
__device__ __forceinline__ int pair_round_dispatch(int Mp, const DecodeLayout &L, uint32_t *heap_a, uint32_t *heap_b,
                                                   uint32_t *buf, const uint16_t *prow_a, const uint16_t *prow_b,
                                                   int T, int Ma, int Mb, int da0, int fa0, int db0, int fb0, int cnt,
                                                   uint32_t lowmask, uint32_t *last_key, int &da1, int &fa1, int &db1,
                                                   int &fb1)
{
    const RoundIn R{L.n, L.B, L.single, L.mulSH, lowmask};
    PairOut o{0, da0, fa0, db0, fb0, 0u};
#define FFS_PCASE(MM)                                                                                        \
    case MM:                                                                                                 \
        o = pair_round<MM, EMIT_B>(R, heap_a, heap_b, buf, prow_a, prow_b, T, Ma, Mb, da0, fa0, db0, fb0, cnt); \
        break;
    switch (Mp) {
        FFS_PCASE(1) FFS_PCASE(2) FFS_PCASE(3) FFS_PCASE(4) FFS_PCASE(5) FFS_PCASE(6) FFS_PCASE(7)
        FFS_PCASE(8) FFS_PCASE(9) FFS_PCASE(10) FFS_PCASE(11) FFS_PCASE(12) FFS_PCASE(13) FFS_PCASE(14)
        FFS_PCASE(15) FFS_PCASE(16) FFS_PCASE(kMaxM)
        default:
            o = pair_round<kMaxM, EMIT_B>(R, heap_a, heap_b, buf, prow_a, prow_b, T, Ma, Mb, da0, fa0, db0, fb0, cnt);
            break;
    }
#undef FFS_PCASE
    da1 = o.da1;
    fa1 = o.fa1;
    db1 = o.db1;
    fb1 = o.fb1;
    if (!EMIT_B) *last_key = o.last_key;
    return o.w;
}

// Stage-0 input keys of the genes [0, cnt) of a chunk, written to buf.
__device__ __forceinline__ void genes_to_keys(const int16_t *genes, int cnt, uint32_t n, uint32_t *buf, int T,
                                              bool &bad)
{
    const int4 *g4 = reinterpret_cast<const int4 *>(genes);
    for (int i0 = 0; i0 < cnt; i0 += 8) {
        const int4 v = g4[i0 >> 3];
        const uint32_t words[4] = {(uint32_t)v.x, (uint32_t)v.y, (uint32_t)v.z, (uint32_t)v.w};
#pragma unroll
        for (int h = 0; h < 8; ++h) {
            if (i0 + h < cnt) {
                uint32_t g = (h & 1) ? (words[h >> 1] >> 16) : (words[h >> 1] & 0xFFFFu);
                g = (uint32_t)(int32_t)(int16_t)g;
                if (g >= n) { bad = true; g = 0; }
                buf[(i0 + h) * T] = (g + 1u) << 1;
            }
        }
    }
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
    if (L.pairs) {
        int s_lo = 0;   // pairs before s_lo (even) are finished
        for (int round = 0; round < max_rounds; ++round) {
            int avail = 0;
            for (int s = s_lo; s < S; s += 2) {
                const bool lastpair = s + 2 >= S;
                if (s + 1 == S) {
                    // odd stage count: the last stage alone
                    const int M = L.M[s];
                    const int d0 = wst[s].dispatched;
                    const int cnt = (s == 0) ? min(L.B, n - d0) : avail;
                    int fl = 0;
                    if (cnt > 0) {
                        if (s == 0)
                            (void)stage_round_dispatch<true, false>(M, L, region + L.heap_off[s] * T, buf,
                                                                    ptab + s * table_row_halves(n), row + d0, T, d0,
                                                                    cnt, lowmask, bad, &last_key, fl);
                        else
                            (void)stage_round_dispatch<false, false>(M, L, region + L.heap_off[s] * T, buf,
                                                                     ptab + s * table_row_halves(n), nullptr, T, d0,
                                                                     cnt, lowmask, bad, &last_key, fl);
                    }
                    __syncwarp();
                    if (lane == 0) wst[s].dispatched = d0 + cnt;
                    __syncwarp();
                    break;
                }
                const int a = s, b = s + 1;
                const int Ma = L.M[a], Mb = L.M[b];
                const int da0 = wst[a].dispatched, fa0 = wst[a].flushed;
                const int db0 = wst[b].dispatched, fb0 = wst[b].flushed;
                const int cnt = (a == 0) ? min(L.B, n - da0) : avail;
                const bool emit_b = !lastpair || (b != S - 1);
                int w = 0, da1 = da0, fa1 = fa0, db1 = db0, fb1 = fb0;
                const bool work = cnt > 0 || (da0 == n && fa0 < Ma) || (emit_b && db0 == n && fb0 < Mb);
                if (work) {
                    if (a == 0 && cnt > 0) genes_to_keys(row + da0, cnt, (uint32_t)n, buf, T, bad);
                    const int Mp = Ma > Mb ? Ma : Mb;
                    const uint16_t *pa = ptab + a * table_row_halves(n), *pb = ptab + b * table_row_halves(n);
                    uint32_t *ha = region + L.heap_off[a] * T, *hb = region + L.heap_off[b] * T;
                    if (emit_b)
                        w = pair_round_dispatch<true>(Mp, L, ha, hb, buf, pa, pb, T, Ma, Mb, da0, fa0, db0, fb0, cnt,
                                                      lowmask, &last_key, da1, fa1, db1, fb1);
                    else
                        w = pair_round_dispatch<false>(Mp, L, ha, hb, buf, pa, pb, T, Ma, Mb, da0, fa0, db0, fb0, cnt,
                                                       lowmask, &last_key, da1, fa1, db1, fb1);
                }
                __syncwarp();
                if (lane == 0) {
                    wst[a].dispatched = da1;
                    wst[a].flushed = fa1;
                    wst[b].dispatched = db1;
                    wst[b].flushed = fb1;
                }
                __syncwarp();
                avail = w;
                const bool done = da1 == n && fa1 == Ma && db1 == n && (!emit_b || fb1 == Mb);
                if (done && s == s_lo) s_lo += 2;
                if (avail == 0 && !done) break;
            }
            if (wst[S - 1].dispatched >= n) break;
        }
        __syncwarp();
        if (bad) return -1;
        if (!L.single) last_key = region[(L.heap_off[S - 1] + L.M[S - 1] - 1) * T];
        return (int32_t)(last_key >> L.SH);
    }
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
