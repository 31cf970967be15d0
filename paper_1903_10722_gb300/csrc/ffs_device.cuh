// ffs_device.cuh -- device-side building blocks of the FFS island GA for
// sm_103a: Philox4x32-10 draws, the list-scheduling decoder, and the genetic
// operators.  Included by the library's .cu files only.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "ffs_tc.cuh"

namespace fgpu {

constexpr int kMaxM = 32;        // machines per stage after clamping to n
constexpr int kMaxStages = 64;

// Device-side checks of the FFS_DEBUG_CHECKS build: FFS_DCHECK(cond, code)
// is cond; when it fails, the first failing check's code goes to the device
// error word (read with ffs_debug_check_error) and the caller skips the
// access it guards.  In the normal build it is `true` and costs nothing.
// Codes: 1 a generation's row is not a permutation of [0, n) (or its
// makespan is negative), 2 a tournament parent outside the torus, 3 a
// crossover cut outside the row, 4 a crossover write outside the row, 5 a
// migration row outside its island, 6 a surrogate ring slot outside the
// ring, 7 a surrogate pick outside the candidates, 8 a machine gene outside
// its stage.
enum : int {
    kCheckPermutation = 1, kCheckParent = 2, kCheckCut = 3, kCheckWrite = 4, kCheckMigrationRow = 5,
    kCheckRingSlot = 6, kCheckPick = 7, kCheckMachineGene = 8
};
#ifdef FFS_DEBUG_CHECKS
extern __device__ int g_ffs_check_error;
__device__ __forceinline__ bool ffs_dcheck(bool ok, int code)
{
    if (!ok) atomicCAS(&g_ffs_check_error, 0, code);
    return ok;
}
#define FFS_DCHECK(cond, code) ::fgpu::ffs_dcheck((cond), (code))
#else
#define FFS_DCHECK(cond, code) true
#endif

// Purpose codes of the Philox counter's fourth word (bits 24..31):
// surrogate candidate k of a cell uses kPurposeSurrogateBase + k (k < 16),
// candidate cut pair t of a screened pseudo pair kPurposeSurrogatePseudoBase + t,
// the surrogate's training-batch sampling kPurposeTrainSample, its weight
// initialisation kPurposeMlpInit.
constexpr uint32_t kPurposeInit = 1, kPurposeCellular = 2, kPurposePseudo = 3, kPurposeMlpInit = 14,
                   kPurposeTrainSample = 15, kPurposeSurrogateBase = 16, kPurposeSurrogatePseudoBase = 32;

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
// stage emitted this round; its heap is saved between rounds.  Per-thread
// shared words: the saved heaps (skipped when B >= n) + B (buffer) + 4
// (read-ahead slots), thread-interleaved (word w of thread t at w * T + t).
//
// Saved heaps in tensor memory: the decoder does no MMA, so the SM's 256 KB
// of TMEM (128 lanes x 512 columns of 32 bits) is free storage.  A warp may
// only touch the 32 lanes of its quarter (warp index mod 4), one lane per
// thread, so the warps of a quarter split the block's columns: warp w owns
// columns [(w / 4) * tmem_group_cols, +tmem_group_cols) of lanes 32 (w mod 4)
// .. +31.  The heaps of the first tmem_stages stages (tmem_split words)
// live there, the others in shared memory, which then holds fewer words per
// thread and more threads per SM.
// ---------------------------------------------------------------------------
struct DecodeLayout {
    int32_t n, S, SH;
    uint32_t mulSH;        // 1 << SH
    int32_t B;             // keys per round (multiple of 8)
    int32_t single;        // 1 if B >= n: one round, heaps stay in registers
    int32_t heap_words;    // saved-heap words in shared memory (0 when single)
    int32_t thread_words;  // words per thread in the interleaved region
    int32_t pairs;         // 1: stages run two at a time, interleaved (see pair_round)
    uint32_t tmem_cols;    // TMEM columns the block allocates (0: no TMEM)
    int32_t tmem_group_cols;  // columns per warp of a lane quarter
    int32_t tmem_stages;   // stages [0, tmem_stages) keep their heaps in TMEM
    int32_t tmem_split;    // their heap words (= heap_off[tmem_stages])
    uint32_t tmem_addr;    // the block's TMEM base address, written by the allocation
    int32_t obj_words;     // words of the release / due tables after the time table (0: none)
    int32_t has_rel, has_due;
    uint32_t wt;           // weight of the total tardiness in the objective
    uint32_t rel_sa, due_sa;  // shared addresses of the release / due tables (0: none), set in the kernel
    const int32_t *M;        // [S] machines per stage (clamped to n), shared memory
    const int32_t *heap_off; // [S] word offset of each stage's heap (prefix sums of M), shared memory
};

// ---------------------------------------------------------------------------
// Shared-memory access by 32-bit shared-window address.  The per-round
// functions below are out of line (one call per stage and round); passing
// them 32-bit shared addresses instead of generic pointers keeps their
// arguments few (all in registers) and their loads and stores in the shared
// space.  A warp's 32 threads own a block of 32 x thread_words words of the
// region, lane-interleaved (word k of lane l at 32 k + l), so one thread's
// words are kWordStride = 128 bytes apart: a compile-time stride, which the
// loads and stores of consecutive words take as immediate offsets.
// ---------------------------------------------------------------------------
constexpr uint32_t kWordStride = 128u;

// This thread's first word of the decoder's region.
__device__ __forceinline__ uint32_t *thread_region(uint32_t *region_base, int thread_words)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    return region_base + (size_t)warp * 32u * (uint32_t)thread_words + lane;
}

__device__ __forceinline__ uint32_t lds32(uint32_t a)
{
    uint32_t v;
    asm volatile("ld.shared.u32 %0, [%1];" : "=r"(v) : "r"(a));
    return v;
}

__device__ __forceinline__ void sts32(uint32_t a, uint32_t v)
{
    asm volatile("st.shared.u32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}

__device__ __forceinline__ uint32_t lds16(uint32_t a)
{
    uint16_t v;
    asm volatile("ld.shared.u16 %0, [%1];" : "=h"(v) : "r"(a));
    return v;
}

// A stage's saved heap as one word: bit 31 set -> TMEM address of the
// thread's first heap word (consecutive columns of its lane; TMEM addresses
// never use bit 31), else the shared address of its first word (stride
// kWordStride).
constexpr uint32_t kHeapInTmem = 0x80000000u;

__device__ __forceinline__ uint32_t heap_handle(const DecodeLayout &L, uint32_t region_sa, int T, int s)
{
    const int off = L.heap_off[s];
    if (s < L.tmem_stages) {
        const int warp = threadIdx.x >> 5;
        return kHeapInTmem | (L.tmem_addr + ((uint32_t)((warp & 3) * 32) << 16) +
                              (uint32_t)((warp >> 2) * L.tmem_group_cols + off));
    }
    (void)T;
    return region_sa + (uint32_t)(off - L.tmem_split) * kWordStride;
}

// Saved heap -> f[0, Mr) (the other slots keep their values).  TMEM loads
// are issued together and waited for once, after the thread's earlier TMEM
// stores have completed.
template <int M>
__device__ __forceinline__ void heap_load(uint32_t h, uint32_t (&f)[M], int Mr, uint32_t stride)
{
    if (h & kHeapInTmem) {
        const uint32_t ta = h & ~kHeapInTmem;
        tc::tmem_wait_st();
#pragma unroll
        for (int m = 0; m < M; ++m)
            if (m < Mr) f[m] = tc::tmem_ld1(ta + (uint32_t)m);
        tc::tmem_wait_ld();
#pragma unroll
        for (int m = 0; m < M; ++m) tc::reg_fence(f[m]);
    } else {
#pragma unroll
        for (int m = 0; m < M; ++m)
            if (m < Mr) f[m] = lds32(h + (uint32_t)m * stride);
    }
}

template <int M>
__device__ __forceinline__ void heap_store(uint32_t h, const uint32_t (&f)[M], int Mr, uint32_t stride)
{
    if (h & kHeapInTmem) {
        const uint32_t ta = h & ~kHeapInTmem;
#pragma unroll
        for (int m = 0; m < M; ++m)
            if (m < Mr) tc::tmem_st1(ta + (uint32_t)m, f[m]);
    } else {
#pragma unroll
        for (int m = 0; m < M; ++m)
            if (m < Mr) sts32(h + (uint32_t)m * stride, f[m]);
    }
}

// One word of a saved heap.
__device__ __forceinline__ uint32_t heap_read1(uint32_t h, int idx, uint32_t stride)
{
    if (h & kHeapInTmem) {
        tc::tmem_wait_st();
        uint32_t v = tc::tmem_ld1((h & ~kHeapInTmem) + (uint32_t)idx);
        tc::tmem_wait_ld();
        tc::reg_fence(v);
        return v;
    }
    return lds32(h + (uint32_t)idx * stride);
}

// f[idx] for a warp-uniform runtime idx, without indexing the register array.
template <int M>
__device__ __forceinline__ uint32_t pick_key(const uint32_t (&f)[M], int idx)
{
    uint32_t k = f[0];
#pragma unroll
    for (int m = 1; m < M; ++m) k = (idx == m) ? f[m] : k;
    return k;
}

// Tardiness of the completion key k at the last stage: max(0, time - D_j),
// D_j read from the due table (entry j + 1 = D_j at byte offset 4 (j + 1) =
// the key's low bits << 1; entry 0 = 0, so the initial keys count 0).
__device__ __forceinline__ uint32_t key_tardiness(uint32_t k, uint32_t due, uint32_t SH, uint32_t idmask)
{
    const uint32_t t = k >> SH, d = lds32(due + ((k & idmask) << 1));
    return max(t, d) - d;
}

// The block's decoding layout lives in shared memory (one copy per block,
// written by thread 0 before a barrier): the decoder reads its fields there
// again after each out-of-line per-round call instead of keeping them live
// in registers across the call.
// decode_tmem_begin: called by all threads after that barrier; warp 0
// allocates the TMEM columns for the saved heaps (the address lands in
// Lsh.tmem_addr).  decode_tmem_end frees them; every thread of the block
// must reach it.
__device__ __forceinline__ void decode_tmem_begin(DecodeLayout &Lsh)
{
    if (Lsh.tmem_cols == 0) return;
    if ((threadIdx.x >> 5) == 0) tc::tmem_alloc(&Lsh.tmem_addr, Lsh.tmem_cols);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
}

__device__ __forceinline__ void decode_tmem_end(const DecodeLayout &Lsh)
{
    if (Lsh.tmem_cols == 0) return;
    tc::tmem_wait_st();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if ((threadIdx.x >> 5) == 0) tc::tmem_dealloc(Lsh.tmem_addr, Lsh.tmem_cols);
}

// Shared-memory table of processing times (uint16): row s holds n + 1
// entries (padded to an even count), entry j + 1 = p[j][s] (entry 0 = 0), so
// the low bits of a key, (job + 1) << 1, are the byte offset of the job's entry.
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

// Two dispatches at once: jobs in1 then in2 (processing times p1, p2).
// The first pops f[0] and completes at x1; the second pops the smaller of
// f[1] and x1 (q) and completes at x2.  The heap left is f[2..M-1] with the
// larger of f[1] and x1 (y) and x2 added: a merge of the sorted f[2..] with
// the sorted pair lo <= hi of {y, x2}, whose k-th smallest is
//   max( min(f[k+2], lo), min(f[k+1], hi), f[k] )
// (terms with an index past the heap dropped) -- three operations per slot,
// one of them a three-input max, against four for two single insertions.
// Same pops and same heap as two dispatch_pp calls.
template <int M>
__device__ __forceinline__ void dispatch2_pp(uint32_t (&f)[M], uint32_t in1, uint32_t p1, uint32_t in2, uint32_t p2,
                                             uint32_t lowmask, uint32_t mulSH, uint32_t &pop1, uint32_t &pop2)
{
    const uint32_t f0 = f[0];
    const uint32_t x1 = p1 * mulSH + max((f0 & ~lowmask) | (in1 & lowmask), in1);
    if constexpr (M == 1) {
        pop1 = f0;
        pop2 = x1;
        f[0] = p2 * mulSH + max((x1 & ~lowmask) | (in2 & lowmask), in2);
    } else {
        const uint32_t q = min(f[1], x1), y = max(f[1], x1);
        const uint32_t x2 = p2 * mulSH + max((q & ~lowmask) | (in2 & lowmask), in2);
        const uint32_t lo = min(y, x2), hi = max(y, x2);
        uint32_t g[M];
#pragma unroll
        for (int k = 0; k < M; ++k) {
            const uint32_t t0 = (k + 2 < M) ? min(f[k + 2], lo) : lo;
            if (k == 0) {
                g[0] = t0;
            } else {
                const uint32_t t1 = (k + 1 < M) ? min(f[k + 1], hi) : hi;
                g[k] = (k == 1) ? max(t0, t1) : __vimax3_u32(t0, t1, f[k]);
            }
        }
#pragma unroll
        for (int k = 0; k < M; ++k) f[k] = g[k];
        pop1 = f0;
        pop2 = q;
    }
}

// Per-warp round bookkeeping lives in shared memory (identical in all lanes).
struct WarpStageState {
    int32_t dispatched;
    int32_t flushed;
};

// ---------------------------------------------------------------------------
// The per-round functions are compiled once, in ffs_decoder_stage.cu and
// ffs_decoder_pair.cu (explicit instantiations, FFS_DECODER_BODIES defined);
// every other unit sees their declarations and calls them across units
// (relocatable device code).
//
// One stage for one round, out of line.  Arguments, packed into 32-bit words:
//   nB   = n | B << 16              SH: key shift
//   heap = saved-heap handle        buf, prow: shared addresses (the buffer's
//          slot 0 of this thread, the stage's table row)
//   genes: FIRST only, the chromosome's genes [d0, d0 + cnt) (global int16)
//   dc   = d0 | cnt << 16           (jobs dispatched before; inputs this round)
//   mf   = Mr | fl0 << 8            (real heap slots; keys flushed before)
//   obj  = release table address >> 2 | due table address >> 2 << 16 (the
//          objective's shared tables, 0 = none): FIRST reads job j's release
//          time into its stage-0 key; the last stage (!EMIT) sums the
//          tardiness of its completions
// FIRST: inputs are the genes, else buf.  EMIT: popped keys go to buf (every
// stage but the last).  cnt = 0: a call that only continues the stage's
// final flush.  Once the stage has dispatched all n jobs its heap (sorted)
// follows its pops into buf, as far as the B slots allow this round.
// Returns x = keys written | flushed total << 16 | bad gene << 24, y = the
// heap's largest key (last stage), z = the tardiness summed this call (last
// stage with due times).
// The heap holds Mr <= M real entries; slots from Mr up hold maximal keys,
// which never pop and never move (used when M is the 32-slot catch-all).
// ---------------------------------------------------------------------------
template <int M, bool FIRST, bool EMIT>
__device__ __noinline__ uint4 stage_round(uint32_t nB, uint32_t SH, uint32_t heap, uint32_t buf, uint32_t prow,
                                          const int16_t *__restrict__ genes, uint32_t dc, uint32_t mf, uint32_t obj);

#ifdef FFS_DECODER_BODIES
template <int M, bool FIRST, bool EMIT>
__device__ __noinline__ uint4 stage_round(uint32_t nB, uint32_t SH, uint32_t heap, uint32_t buf, uint32_t prow,
                                          const int16_t *__restrict__ genes, uint32_t dc, uint32_t mf, uint32_t obj)
{
    const int n = (int)(nB & 0xFFFFu), B = (int)(nB >> 16);
    const int d0 = (int)(dc & 0xFFFFu), cnt = (int)(dc >> 16);
    const int Mr = (int)(mf & 0xFFu), fl0 = (int)(mf >> 8);
    // 2^SH through an opaque move: the compiler then keeps p * 2^SH + t as one
    // multiply-add (FMA pipe) instead of a shift and an add (ALU pipe, the
    // decoder's bottleneck)
    uint32_t mulSH;
    asm("mov.b32 %0, %1;" : "=r"(mulSH) : "r"(1u << SH));
    const uint32_t lowmask = mulSH - 1u, idmask = lowmask & ~1u;
    constexpr uint32_t stride = kWordStride;
    const bool single = B >= n;
    const uint32_t rel = (obj & 0xFFFFu) << 2, due = EMIT ? 0u : (obj >> 16) << 2;
    uint32_t tard = 0;
    bool bad_gene = false;
    // every slot defined before the conditional load (a partly defined
    // array here costs the whole kernel half its registers)
    uint32_t f[M];
#pragma unroll
    for (int m = 0; m < M; ++m) f[m] = m < Mr ? 0u : 0xFFFFFFFFu;
    if (d0 > 0 && !single) heap_load<M>(heap, f, Mr, stride);
    int skip = Mr - d0;
    skip = skip < 0 ? 0 : (skip > cnt ? cnt : skip);
    int w = 0;
    if constexpr (FIRST) {
        // genes arrive 8 per 16-byte load, one load ahead; cnt is a multiple of 8
        // except at the tail (rows are padded to 8 genes, so the load stays in the row)
        const int4 *g4 = reinterpret_cast<const int4 *>(genes);
        int4 vnext = cnt > 0 ? g4[0] : make_int4(0, 0, 0, 0);
        for (int i0 = 0; i0 < cnt; i0 += 8) {
            const int4 v = vnext;
            if (i0 + 8 < cnt) vnext = g4[(i0 >> 3) + 1];
            const uint32_t words[4] = {(uint32_t)v.x, (uint32_t)v.y, (uint32_t)v.z, (uint32_t)v.w};
            // the stage-1 key of gene h of the block (its release time R_j as the time)
            auto key_of = [&](int h) {
                uint32_t g = (h & 1) ? (words[h >> 1] >> 16) : (words[h >> 1] & 0xFFFFu);
                g = (uint32_t)(int32_t)(int16_t)g;
                if (g >= (uint32_t)n) { bad_gene = true; g = 0; }
                uint32_t in = (g + 1u) << 1;
                if (rel) in |= lds32(rel + (in << 1)) << SH;
                return in;
            };
            auto take = [&](int i, uint32_t popped) {
                if constexpr (EMIT) {
                    if (i >= skip) { sts32(buf + (uint32_t)w * stride, popped); ++w; }
                } else {
                    if (due) tard += key_tardiness(popped, due, SH, idmask);
                }
            };
            // two jobs per dispatch, one at the block's ragged end
#pragma unroll
            for (int h = 0; h < 8; h += 2) {
                if (i0 + h + 1 < cnt) {
                    const uint32_t ka = key_of(h), kb = key_of(h + 1);
                    uint32_t pop1, pop2;
                    dispatch2_pp<M>(f, ka, lds16(prow + (ka & idmask)), kb, lds16(prow + (kb & idmask)), lowmask,
                                    mulSH, pop1, pop2);
                    take(i0 + h, pop1);
                    take(i0 + h + 1, pop2);
                } else if (i0 + h < cnt) {
                    const uint32_t ka = key_of(h);
                    take(i0 + h, dispatch_pp<M>(f, ka, lds16(prow + (ka & idmask)), lowmask, mulSH));
                }
            }
        }
    } else if (cnt > 0) {
        // The first `skip` dispatches pop initial keys (nothing emitted): one
        // at a time.  Then two jobs per dispatch2_pp, with the keys read four
        // steps ahead and their processing times two steps ahead; the stores
        // of steps i, i + 1 go to slots i - skip, i + 1 - skip <= i + 1, never
        // to a slot still to be read.  Slots up to cnt + 3 may be read (the
        // region has four spare words per thread).
        int i = 0;
        for (; i < skip; ++i) {
            const uint32_t in = lds32(buf + (uint32_t)i * stride);
            (void)dispatch_pp<M>(f, in, lds16(prow + (in & idmask)), lowmask, mulSH);
        }
        if (i < cnt) {
            uint32_t rd = buf + (uint32_t)i * stride;
            uint32_t k0 = lds32(rd), k1 = lds32(rd + stride), k2 = lds32(rd + 2u * stride),
                     k3 = lds32(rd + 3u * stride);
            uint32_t t0 = lds16(prow + (k0 & idmask)), t1 = lds16(prow + (k1 & idmask));
            rd += 4u * stride;
            uint32_t wr = buf;
            // unrolled twice, the read-ahead registers alternate roles instead of
            // being moved at every iteration
#pragma unroll 2
            for (; i + 2 <= cnt; i += 2) {
                const uint32_t k4 = lds32(rd), k5 = lds32(rd + stride);
                const uint32_t t2 = lds16(prow + (k2 & idmask)), t3 = lds16(prow + (k3 & idmask));
                uint32_t pop1, pop2;
                dispatch2_pp<M>(f, k0, t0, k1, t1, lowmask, mulSH, pop1, pop2);
                if constexpr (EMIT) {
                    sts32(wr, pop1);
                    sts32(wr + stride, pop2);
                    wr += 2u * stride;
                } else {
                    if (due) tard += key_tardiness(pop1, due, SH, idmask) + key_tardiness(pop2, due, SH, idmask);
                }
                k0 = k2;
                k1 = k3;
                k2 = k4;
                k3 = k5;
                t0 = t2;
                t1 = t3;
                rd += 2u * stride;
            }
            if (i < cnt) {
                const uint32_t popped = dispatch_pp<M>(f, k0, t0, lowmask, mulSH);
                if constexpr (EMIT) sts32(wr, popped);
                else if (due) tard += key_tardiness(popped, due, SH, idmask);
            }
        }
        if constexpr (EMIT) w = cnt - skip;
    }
    const int d1 = d0 + cnt;
    uint4 out;
    out.y = 0u;
    out.w = 0u;
    if constexpr (EMIT) {
        int fl = fl0;
        if (d1 == n && fl < Mr) {
            // the stage is complete: its heap keys, in order, follow
            const int room = B - w;
            const int take = (Mr - fl) < room ? (Mr - fl) : room;
            for (int t = 0; t < take; ++t) sts32(buf + (uint32_t)(w + t) * stride, pick_key<M>(f, fl + t));
            w += take;
            fl += take;
        }
        if (!single && fl < Mr) heap_store<M>(heap, f, Mr, stride);
        out.x = (uint32_t)w | (uint32_t)fl << 16;
    } else {
        if (!single) heap_store<M>(heap, f, Mr, stride);
        uint32_t lk = f[0];
#pragma unroll
        for (int m = 1; m < M; ++m)
            if (m == Mr - 1) lk = f[m];
        out.y = lk;
        out.x = (uint32_t)fl0 << 16;
        // all jobs dispatched: the completions still in the heap
        if (due && d1 == n) {
#pragma unroll
            for (int m = 0; m < M; ++m)
                if (m < Mr) tard += key_tardiness(f[m], due, SH, idmask);
        }
    }
    out.z = tard;
    if (bad_gene) out.x |= 1u << 24;
    return out;
}
#endif  // FFS_DECODER_BODIES

template <bool FIRST, bool EMIT>
__device__ __forceinline__ uint4 stage_round_dispatch(int M, uint32_t nB, uint32_t SH, uint32_t heap, uint32_t buf,
                                                      uint32_t prow, const int16_t *genes, uint32_t dc, uint32_t mf,
                                                      uint32_t obj)
{
#define FFS_CASE(MM) \
    case MM: return stage_round<MM, FIRST, EMIT>(nB, SH, heap, buf, prow, genes, dc, mf, obj);
    switch (M) {
        FFS_CASE(1) FFS_CASE(2) FFS_CASE(3) FFS_CASE(4) FFS_CASE(5) FFS_CASE(6) FFS_CASE(7)
        FFS_CASE(8) FFS_CASE(9) FFS_CASE(10) FFS_CASE(11) FFS_CASE(12) FFS_CASE(13) FFS_CASE(14)
        FFS_CASE(15) FFS_CASE(16)
        default: return stage_round<kMaxM, FIRST, EMIT>(nB, SH, heap, buf, prow, genes, dc, mf, obj);
    }
#undef FFS_CASE
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
// Arguments as in stage_round, with mm = Ma | Mb << 8 | fa0 << 16 | fb0 << 24,
// dd = da0 | db0 << 16 and due = the due table's shared address when b is
// the last stage of an instance with due times (else 0).  Returns x = keys
// written | fa1 << 16 | fb1 << 24, y = da1 | db1 << 16, z = b's largest key
// (last pair), w = the tardiness of b's completions summed this call.
// ---------------------------------------------------------------------------
template <int M, bool EMIT_B>
__device__ __noinline__ uint4 pair_round(uint32_t nB, uint32_t SH, uint32_t heap_a, uint32_t heap_b, uint32_t buf,
                                         uint32_t prow_a, uint32_t prow_b, uint32_t mm, uint32_t dd, int cnt,
                                         uint32_t due);

#ifdef FFS_DECODER_BODIES
template <int M, bool EMIT_B>
__device__ __noinline__ uint4 pair_round(uint32_t nB, uint32_t SH, uint32_t heap_a, uint32_t heap_b, uint32_t buf,
                                         uint32_t prow_a, uint32_t prow_b, uint32_t mm, uint32_t dd, int cnt,
                                         uint32_t due)
{
    const int n = (int)(nB & 0xFFFFu), B = (int)(nB >> 16);
    const int Ma = (int)(mm & 0xFFu), Mb = (int)((mm >> 8) & 0xFFu);
    const int fa0 = (int)((mm >> 16) & 0xFFu), fb0 = (int)(mm >> 24);
    const int da0 = (int)(dd & 0xFFFFu), db0 = (int)(dd >> 16);
    // 2^SH through an opaque move: the compiler then keeps p * 2^SH + t as one
    // multiply-add (FMA pipe) instead of a shift and an add (ALU pipe, the
    // decoder's bottleneck)
    uint32_t mulSH;
    asm("mov.b32 %0, %1;" : "=r"(mulSH) : "r"(1u << SH));
    const uint32_t lowmask = mulSH - 1u, idmask = lowmask & ~1u;
    constexpr uint32_t stride = kWordStride;
    const bool chunked = B < n;
    if constexpr (EMIT_B) due = 0u;
    uint32_t tard = 0;
    uint32_t fa[M], fb[M];
#pragma unroll
    for (int m = 0; m < M; ++m) {
        fa[m] = m < Ma ? 0u : 0xFFFFFFFFu;
        fb[m] = m < Mb ? 0u : 0xFFFFFFFFu;
    }
    if (chunked && da0 > 0) heap_load<M>(heap_a, fa, Ma, stride);
    if (chunked && db0 > 0) heap_load<M>(heap_b, fb, Mb, stride);
    int w = 0, db = db0, i = 0;
    uint32_t wr = buf;
    if (cnt > 0) {
        int skip_a = Ma - da0;
        skip_a = skip_a < 0 ? 0 : (skip_a > cnt ? cnt : skip_a);
        // buffer keys two steps ahead, their times at a one step ahead (see
        // stage_round)
        uint32_t in_a = lds32(buf), in_n = lds32(buf + stride);
        uint32_t pp_a = lds16(prow_a + (in_a & idmask));
        uint32_t rd = buf + 2u * stride;
        for (; i < skip_a; ++i) {
            const uint32_t in_nn = lds32(rd);
            const uint32_t pp_n = lds16(prow_a + (in_n & idmask));
            (void)dispatch_pp<M>(fa, in_a, pp_a, lowmask, mulSH);
            in_a = in_n;
            in_n = in_nn;
            pp_a = pp_n;
            rd += stride;
        }
        uint32_t e = fa[0];
        uint32_t pp_e = lds16(prow_b + (e & idmask));
        int end2 = i + (Mb - db > 0 ? Mb - db : 0);
        end2 = end2 > cnt ? cnt : end2;
        // Shared loads and stores keep their source order (volatile asm), so
        // each step issues its loads first: the next buffer key and its time
        // at a, then -- right after a's dispatch -- b's next key's time, and
        // the store of b's pop last.
        for (; i < end2; ++i) {
            const uint32_t in_nn = lds32(rd);
            const uint32_t pp_n = lds16(prow_a + (in_n & idmask));
            (void)dispatch_pp<M>(fa, in_a, pp_a, lowmask, mulSH);
            const uint32_t e_n = fa[0];
            const uint32_t pp_e_n = lds16(prow_b + (e_n & idmask));
            (void)dispatch_pp<M>(fb, e, pp_e, lowmask, mulSH);
            ++db;
            e = e_n;
            pp_e = pp_e_n;
            in_a = in_n;
            in_n = in_nn;
            pp_a = pp_n;
            rd += stride;
        }
#pragma unroll 1
        for (; i < cnt; ++i) {
            const uint32_t in_nn = lds32(rd);
            const uint32_t pp_n = lds16(prow_a + (in_n & idmask));
            (void)dispatch_pp<M>(fa, in_a, pp_a, lowmask, mulSH);
            const uint32_t e_n = fa[0];
            const uint32_t pp_e_n = lds16(prow_b + (e_n & idmask));
            const uint32_t pb = dispatch_pp<M>(fb, e, pp_e, lowmask, mulSH);
            ++db;
            if constexpr (EMIT_B) {
                sts32(wr, pb);
                wr += stride;
                ++w;
            } else {
                if (due) tard += key_tardiness(pb, due, SH, idmask);
            }
            e = e_n;
            pp_e = pp_e_n;
            in_a = in_n;
            in_n = in_nn;
            pp_a = pp_n;
            rd += stride;
        }
    }
    const int da1 = da0 + cnt;
    int fa1 = fa0;
    if (da1 == n && fa0 < Ma) {
        // a is complete: its heap keys, in order, are b's last inputs (as many
        // as b's output fits in the buffer this round)
        int take = Ma - fa0;
        if (EMIT_B && take > B - w) take = B - w;
        for (int t = 0; t < take; ++t) {
            const uint32_t k = pick_key<M>(fa, fa0 + t);
            const uint32_t pb = dispatch_pp<M>(fb, k, lds16(prow_b + (k & idmask)), lowmask, mulSH);
            if (EMIT_B && db >= Mb) {
                sts32(buf + (uint32_t)w * stride, pb);
                ++w;
            }
            if (!EMIT_B && due) tard += key_tardiness(pb, due, SH, idmask);
            ++db;
        }
        fa1 = fa0 + take;
    }
    if (chunked && fa1 < Ma) heap_store<M>(heap_a, fa, Ma, stride);
    const int db1 = db;
    int fb1 = fb0;
    uint4 out;
    out.z = 0u;
    out.w = 0u;
    if constexpr (EMIT_B) {
        if (db1 == n && fb0 < Mb) {
            int take = Mb - fb0;
            if (take > B - w) take = B - w;
            for (int t = 0; t < take; ++t) sts32(buf + (uint32_t)(w + t) * stride, pick_key<M>(fb, fb0 + t));
            w += take;
            fb1 = fb0 + take;
        }
        if (chunked && fb1 < Mb) heap_store<M>(heap_b, fb, Mb, stride);
    } else {
        if (chunked) heap_store<M>(heap_b, fb, Mb, stride);
        uint32_t lk = fb[0];
#pragma unroll
        for (int m = 1; m < M; ++m)
            if (m == Mb - 1) lk = fb[m];
        out.z = lk;
        // b has dispatched all jobs: the completions still in its heap
        if (due && db1 == n) {
#pragma unroll
            for (int m = 0; m < M; ++m)
                if (m < Mb) tard += key_tardiness(fb[m], due, SH, idmask);
        }
    }
    out.w = tard;
    out.x = (uint32_t)w | (uint32_t)fa1 << 16 | (uint32_t)fb1 << 24;
    out.y = (uint32_t)da1 | (uint32_t)db1 << 16;
    return out;
}
#endif  // FFS_DECODER_BODIES

template <bool EMIT_B>
__device__ __forceinline__ uint4 pair_round_dispatch(int Mp, uint32_t nB, uint32_t SH, uint32_t heap_a,
                                                     uint32_t heap_b, uint32_t buf, uint32_t prow_a, uint32_t prow_b,
                                                     uint32_t mm, uint32_t dd, int cnt, uint32_t due)
{
#define FFS_PCASE(MM) \
    case MM: return pair_round<MM, EMIT_B>(nB, SH, heap_a, heap_b, buf, prow_a, prow_b, mm, dd, cnt, due);
    switch (Mp) {
        FFS_PCASE(1) FFS_PCASE(2) FFS_PCASE(3) FFS_PCASE(4) FFS_PCASE(5) FFS_PCASE(6) FFS_PCASE(7)
        FFS_PCASE(8) FFS_PCASE(9) FFS_PCASE(10) FFS_PCASE(11) FFS_PCASE(12) FFS_PCASE(13) FFS_PCASE(14)
        FFS_PCASE(15) FFS_PCASE(16)
        default: return pair_round<kMaxM, EMIT_B>(nB, SH, heap_a, heap_b, buf, prow_a, prow_b, mm, dd, cnt, due);
    }
#undef FFS_PCASE
}

// Stage-0 input keys of the genes [0, cnt) of a chunk, written to buf.
__device__ __forceinline__ void genes_to_keys(const int16_t *genes, int cnt, uint32_t n, uint32_t buf,
                                              uint32_t stride, uint32_t rel, uint32_t SH, bool &bad)
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
                uint32_t key = (g + 1u) << 1;
                if (rel) key |= lds32(rel + (key << 1)) << SH;   // stage-1 ready time R_j
                sts32(buf + (uint32_t)(i0 + h) * stride, key);
            }
        }
    }
}

// Decode one chromosome (row of genes in global memory, 16-byte aligned).
//   L     : the block's layout in shared memory (see decode_tmem_begin).
//   region: this thread's first shared word (thread_region), stride kWordStride.
//   ptab  : shared uint16 table, row s at ptab + s * table_row_halves(n).
//   wst   : this warp's per-stage state, S entries (shared).
// All lanes of a warp must call this together for the same instance (the
// TMEM accesses are warp-collective).
// Returns the objective -- the makespan, plus WT x total tardiness when the
// instance has due times -- or -1 if a gene is outside [0, n).
__device__ __forceinline__ int32_t decode_chromosome(const DecodeLayout &L, const int16_t *row,
                                                     uint32_t *region, int T, const uint16_t *ptab,
                                                     WarpStageState *wst)
{
    const int n = L.n, S = L.S;
    constexpr uint32_t stride = kWordStride;
    const uint32_t region_sa = tc::smem_u32(region);
    const uint32_t buf = region_sa + (uint32_t)L.heap_words * stride;
    const uint32_t tab = tc::smem_u32(ptab);
    const uint32_t row_bytes = (uint32_t)table_row_halves(n) * 2u;
    const uint32_t nB = (uint32_t)n | (uint32_t)L.B << 16, SH = (uint32_t)L.SH;
    // the objective's tables for the per-round calls (0: none)
    const uint32_t obj = (L.rel_sa >> 2) | (L.due_sa >> 2) << 16;
    uint32_t tard = 0;
    // Every buffer slot holds a valid key (or 0) before the read-ahead can
    // touch it: clear the buffer and its four spare slots.
    for (int w = 0; w < L.B + 4; ++w) sts32(buf + (uint32_t)w * stride, 0u);
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
                    if (cnt > 0) {
                        const uint32_t h = heap_handle(L, region_sa, T, s);
                        const uint32_t prow = tab + (uint32_t)s * row_bytes;
                        const uint32_t dc = (uint32_t)d0 | (uint32_t)cnt << 16, mf = (uint32_t)M;
                        const uint4 o = (s == 0)
                                            ? stage_round_dispatch<true, false>(M, nB, SH, h, buf, prow, row + d0, dc, mf, obj)
                                            : stage_round_dispatch<false, false>(M, nB, SH, h, buf, prow, nullptr, dc, mf, obj);
                        last_key = o.y;
                        tard += o.z;
                        if (o.x >> 24) bad = true;
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
                    if (a == 0 && cnt > 0) genes_to_keys(row + da0, cnt, (uint32_t)n, buf, stride, L.rel_sa, SH, bad);
                    const int Mp = Ma > Mb ? Ma : Mb;
                    const uint32_t pa = tab + (uint32_t)a * row_bytes, pb = pa + row_bytes;
                    const uint32_t ha = heap_handle(L, region_sa, T, a), hb = heap_handle(L, region_sa, T, b);
                    const uint32_t mm = (uint32_t)Ma | (uint32_t)Mb << 8 | (uint32_t)fa0 << 16 | (uint32_t)fb0 << 24;
                    const uint32_t dd = (uint32_t)da0 | (uint32_t)db0 << 16;
                    const uint4 o = emit_b ? pair_round_dispatch<true>(Mp, nB, SH, ha, hb, buf, pa, pb, mm, dd, cnt, 0u)
                                           : pair_round_dispatch<false>(Mp, nB, SH, ha, hb, buf, pa, pb, mm, dd, cnt,
                                                                        L.due_sa);
                    w = (int)(o.x & 0xFFFFu);
                    fa1 = (int)((o.x >> 16) & 0xFFu);
                    fb1 = (int)(o.x >> 24);
                    da1 = (int)(o.y & 0xFFFFu);
                    db1 = (int)(o.y >> 16);
                    if (!emit_b) {
                        last_key = o.z;
                        tard += o.w;
                    }
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
        // every lane takes part in the (warp-collective) read of the last heap,
        // a lane with a bad gene included
        if (!L.single) last_key = heap_read1(heap_handle(L, region_sa, T, S - 1), L.M[S - 1] - 1, stride);
        if (bad) return -1;
        return (int32_t)((last_key >> L.SH) + L.wt * tard);
    }
    int s_lo = 0;   // stages before s_lo have dispatched and emitted everything
    for (int round = 0; round < max_rounds; ++round) {
        int avail = 0;  // keys in buf for the next stage
        for (int s = s_lo; s < S; ++s) {
            const int M = L.M[s];
            const int d0 = wst[s].dispatched, fl0 = wst[s].flushed;
            const int cnt = (s == 0) ? min(L.B, n - d0) : avail;
            const bool last = (s == S - 1);
            int w = 0, fl = fl0;
            if (cnt > 0 || (!last && d0 == n && fl0 < M)) {
                const uint32_t h = heap_handle(L, region_sa, T, s);
                const uint32_t prow = tab + (uint32_t)s * row_bytes;
                const uint32_t dc = (uint32_t)d0 | (uint32_t)cnt << 16, mf = (uint32_t)M | (uint32_t)fl0 << 8;
                const int16_t *g = row + d0;
                uint4 o;
                if (last)
                    o = (s == 0) ? stage_round_dispatch<true, false>(M, nB, SH, h, buf, prow, g, dc, mf, obj)
                                 : stage_round_dispatch<false, false>(M, nB, SH, h, buf, prow, nullptr, dc, mf, obj);
                else
                    o = (s == 0 && cnt > 0) ? stage_round_dispatch<true, true>(M, nB, SH, h, buf, prow, g, dc, mf, obj)
                                            : stage_round_dispatch<false, true>(M, nB, SH, h, buf, prow, nullptr, dc, mf,
                                                                                obj);
                w = (int)(o.x & 0xFFFFu);
                fl = (int)((o.x >> 16) & 0xFFu);
                if (o.x >> 24) bad = true;
                if (last) {
                    last_key = o.y;
                    tard += o.z;
                }
            }
            const int d1 = d0 + cnt;
            __syncwarp();
            if (lane == 0) { wst[s].dispatched = d1; wst[s].flushed = fl; }
            __syncwarp();
            avail = w;
            const bool done = d1 == n && (last || fl == M);
            if (done && s == s_lo) ++s_lo;
            // nothing reaches later stages this round unless this one is finished
            if (avail == 0 && !done) break;
        }
        if (wst[S - 1].dispatched >= n) break;
    }
    __syncwarp();
    if (!L.single) last_key = heap_read1(heap_handle(L, region_sa, T, S - 1), L.M[S - 1] - 1, stride);
    if (bad) return -1;
    return (int32_t)((last_key >> L.SH) + L.wt * tard);
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
