// ffs_assign.cu -- exact evaluation of the paper's own genotype: strings of
// n*S genes, gene j*S + s = the machine of job j at stage s (Section 4.1,
// genotype level), on unrelated machines P_jsm (Section 3).
//
// Sequencing, which the paper leaves unstated: every machine processes the
// jobs assigned to it in order of arrival (stage 1: release time R_j, later
// stages: completion at the previous stage), ties by job index; a job starts
// at max(machine free time, arrival).  Objective: C_max, plus WT * sum_j
// max(0, C_j - D_j) with due times.
//
// One thread decodes one string.  A stage's arrivals are the machines' job
// streams of the previous stage merged in (completion, job) order: every
// stream is already in that order (a machine completes its jobs one after
// the other, processing times >= 1), so the merge takes the smallest head
// key at each step and never sorts.  Keys are completion << SH | (job+1) << 1
// as in the permutation decoder.  The streams live in a per-thread scratch of
// 2n keys in global memory; the runs' heads and the per-machine counters, and
// (when they fit) the stage's genes and table slice, in shared memory.  A call
// runs in chunks of rows: k_assign_transpose copies a chunk's genes stage-major
// (one byte each), then k_eval_assign decodes it, one row per thread.
#include <algorithm>
#include <vector>

#include "ffs_internal.cuh"

namespace fgpu {

constexpr int kAssignMaxM = 32;        // machines per stage
constexpr int kAssignThreads = 128;
constexpr size_t kAssignScratchCap = size_t(1) << 30;   // bytes of per-row scratch (streams + genes) at most

struct AssignView {
    int32_t n, S, W, SH;
    uint32_t wt;
    const int32_t *M;        // [S]
    const int32_t *off;      // [S] M_0 + ... + M_{s-1}
    const uint16_t *p;       // [n][W]
    const uint32_t *order0;  // [n] stage-1 arrival keys R_j << SH | (j+1) << 1, ascending
    const uint32_t *due;     // [n] or NULL
};

// Stage-major copy of rows [0, count) of a population chunk: the gene of job
// j at stage s goes to byte s * nstride + j of the row's output block (genes
// outside [0, 255] become 255, which no stage accepts).  Block per row; the
// row's output block stays in L2 while its scattered bytes are written.
__global__ void k_assign_transpose(const int16_t *__restrict__ pop, int ld, int n, int S, int nstride,
                                   uint8_t *__restrict__ out)
{
    const int16_t *row = pop + (int64_t)blockIdx.x * ld;
    uint8_t *o = out + (int64_t)blockIdx.x * S * nstride;
    const int total = n * S;
    for (int i = threadIdx.x; i < total; i += blockDim.x) {
        const int g = row[i];
        const int j = i / S, s = i - j * S;
        o[(int64_t)s * nstride + j] = (uint8_t)((unsigned)g > 255u ? 255 : g);
    }
}

// Per-thread arrays in shared memory, interleaved by thread (element k of
// thread t at k * T + t, so lanes indexing by their own k never conflict):
// the input runs' first two keys (hk0, hk1), position of hk1's key and end,
// and per machine of the stage its job count, fill position and free time --
// 7 * MX words.  Popping a run shifts hk1 into hk0 and refills hk1 with an
// asynchronous 4-byte copy from the run in global memory, which the next
// pop of that run waits for (one pop later at least).  With
// GENES, the stage's genes are first copied there as bytes (n per thread),
// so the dispatch reads the machine of a job from shared memory.
// PSLICE (with GENES, one row per thread): the block's threads run the
// stages in step (a barrier per stage) and share the stage's slice of the
// processing-time table, p[j][M_0 + ... + M_{s-1} + m] at pst[j * MX + m],
// copied to shared memory after the per-thread arrays and genes.
template <bool GENES, bool PSLICE>
__global__ void __launch_bounds__(kAssignThreads) k_eval_assign(AssignView V, const uint8_t *__restrict__ tpop,
                                                                int64_t N, int nstride, int32_t *__restrict__ out,
                                                                uint32_t *scratch, int MX)
{
    extern __shared__ __align__(16) uint32_t sm[];
    const int T = kAssignThreads, t = threadIdx.x;
    uint32_t *hk0 = sm + t, *hk1 = sm + MX * T + t, *freeT = sm + 2 * MX * T + t;
    int *pos = reinterpret_cast<int *>(sm) + 3 * MX * T + t, *endp = pos + MX * T, *cnt = endp + MX * T,
        *fill = cnt + MX * T;
    uint8_t *gsm = reinterpret_cast<uint8_t *>(sm + 7 * MX * T) + t;   // gene of job j at gsm[j * T]
    uint16_t *pst = reinterpret_cast<uint16_t *>(sm + 7 * MX * T + (V.n + 3) / 4 * T);
    const uint32_t hk1_sa = (uint32_t)__cvta_generic_to_shared(hk1);
    const int64_t nthreads = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + t;
    const int n = V.n, S = V.S;
    const uint32_t SH = (uint32_t)V.SH, idmask = ((1u << SH) - 1u) & ~1u;
    uint32_t *bufA = scratch + tid * 2 * (int64_t)n, *bufB = bufA + n;
    // PSLICE: one pass, rows beyond N run the stages without work (barriers)
    for (int64_t r = tid; PSLICE ? r == tid : r < N; r += nthreads) {
        const bool live = r < N;
        const uint8_t *rowt = tpop + r * (int64_t)V.S * nstride;   // stage-major genes
        bool bad = false;
        const uint32_t *in = V.order0;
        int R = 1;
        pos[0] = 1;
        endp[0] = n;
        hk0[0] = in[0];
        hk1[0] = n > 1 ? in[1] : 0xFFFFFFFFu;
        uint32_t *outb = bufA;
        uint32_t cmax = 0, tard = 0;
        for (int s = 0; s < S; ++s) {
            const int Ms = V.M[s], off = V.off[s];
            const bool last = s == S - 1;
            if constexpr (PSLICE) {
                __syncthreads();   // every thread is done with the previous slice
                for (int i = t; i < n * Ms; i += T) {
                    const int j = i / Ms, m = i - j * Ms;
                    pst[j * MX + m] = V.p[(int64_t)j * V.W + off + m];
                }
                __syncthreads();
                if (!live) continue;
            }
            for (int m = 0; m < Ms; ++m) cnt[m * T] = 0;
            const uint8_t *gs = rowt + (int64_t)s * nstride;   // 16-byte aligned
            for (int j0 = 0; j0 < n; j0 += 16) {
                const uint4 v = *reinterpret_cast<const uint4 *>(gs + j0);
                const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int u = 0; u < 16; ++u) {
                    if (j0 + u < n) {
                        int g = (int)((w[u >> 2] >> (8 * (u & 3))) & 0xFFu);
                        if (g >= Ms) {
                            bad = true;
                            g = 0;   // decoded as machine 0 (memory-safe); the row reports -1
                        }
                        ++cnt[g * T];
                        if constexpr (GENES) gsm[(j0 + u) * T] = (uint8_t)g;
                    }
                }
            }
            for (int m = 0, acc = 0; m < Ms; ++m) {
                fill[m * T] = acc;
                acc += cnt[m * T];
                freeT[m * T] = 0u;
            }
            int prev = -1;
            for (int k = 0; k < n; ++k) {
                // the next arrival: the smallest head key of the input runs
                int rb = 0;
                uint32_t kb = hk0[0];
                for (int q = 1; q < R; ++q) {
                    const uint32_t h = hk0[q * T];
                    if (h < kb) {
                        kb = h;
                        rb = q;
                    }
                }
                // hk1 of run rb: refilled by the previous pop's copy when rb was
                // popped then, else by an older one
                if (rb == prev) asm volatile("cp.async.wait_group 0;" ::: "memory");
                else asm volatile("cp.async.wait_group 1;" ::: "memory");
                hk0[rb * T] = hk1[rb * T];
                const int p1 = pos[rb * T] + 1;
                pos[rb * T] = p1;
                if (p1 < endp[rb * T])
                    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(hk1_sa + (uint32_t)(rb * T) * 4u),
                                 "l"(in + p1)
                                 : "memory");
                else
                    hk1[rb * T] = 0xFFFFFFFFu;
                asm volatile("cp.async.commit_group;" ::: "memory");
                prev = rb;
                const int j = (int)((kb & idmask) >> 1) - 1;
                int m;
                if constexpr (GENES) {
                    m = gsm[j * T];
                } else {
                    m = gs[j];
                    if (m >= Ms) m = 0;
                }
                uint32_t pj;
                if constexpr (PSLICE) pj = pst[j * MX + m];
                else pj = V.p[(int64_t)j * V.W + off + m];
                const uint32_t c = max(freeT[m * T], kb >> SH) + pj;
                freeT[m * T] = c;
                if (!last) {
                    const int f = fill[m * T];
                    fill[m * T] = f + 1;
                    outb[f] = (c << SH) | ((uint32_t)(j + 1) << 1);
                } else {
                    cmax = max(cmax, c);
                    if (V.due && c > V.due[j]) tard += c - V.due[j];
                }
            }
            // no copy in flight reads a stream the next stage overwrites
            asm volatile("cp.async.wait_all;" ::: "memory");
            if (!last) {
                // the next stage merges this stage's machine streams
                in = outb;
                R = Ms;
                for (int m = 0, acc = 0; m < Ms; ++m) {
                    const int c = cnt[m * T];
                    pos[m * T] = acc + 1;
                    endp[m * T] = acc + c;
                    hk0[m * T] = c > 0 ? in[acc] : 0xFFFFFFFFu;
                    hk1[m * T] = c > 1 ? in[acc + 1] : 0xFFFFFFFFu;
                    acc += c;
                }
                outb = outb == bufA ? bufB : bufA;
            }
        }
        if (live) out[r] = bad ? -1 : (int32_t)(cmax + V.wt * tard);
    }
}

}  // namespace fgpu

using namespace fgpu;

struct ffs_assign_instance {
    int n = 0, S = 0, W = 0, SH = 0;
    int32_t wt = 0;
    int32_t *d_M = nullptr, *d_off = nullptr;
    uint16_t *d_p = nullptr;
    uint32_t *d_order0 = nullptr, *d_due = nullptr;
    uint32_t *d_scratch = nullptr;
    uint8_t *d_tpop = nullptr;     // stage-major genes of one chunk of rows
    int nstride = 0;               // round_up(n, 16)
    int64_t scratch_threads = 0;   // rows of one chunk = threads the scratch serves (a multiple of kAssignThreads)
    int num_sms = 0;
    int MX = 0;                    // largest M_s
};

int ffs_assign_instance_create(int32_t n, int32_t S, const int32_t *M, const int32_t *p_u, const int32_t *release,
                               const int32_t *due, int32_t wt, ffs_assign_instance **out)
{
    clear_error();
    if (!out || !M || !p_u) return set_error(FFS_EINVAL, "NULL argument");
    *out = nullptr;
    if (n < 1 || n > 32767) return set_error(FFS_EINVAL, "n_jobs = %d outside [1, 32767]", n);
    if (S < 1 || S > kMaxStages) return set_error(FFS_EINVAL, "n_stages = %d outside [1, %d]", S, kMaxStages);
    if ((int64_t)n * S > (int64_t(1) << 28)) return set_error(FFS_EUNSUPPORTED, "n * S = %lld genes", (long long)n * S);
    if (due && wt < 0) return set_error(FFS_EINVAL, "tardiness weight %d < 0", wt);
    int W = 0;
    for (int s = 0; s < S; ++s) {
        if (M[s] < 1) return set_error(FFS_EINVAL, "machines_per_stage[%d] = %d < 1", s, M[s]);
        if (M[s] > kAssignMaxM) return set_error(FFS_EUNSUPPORTED, "stage %d: %d machines (> %d)", s, M[s], kAssignMaxM);
        W += M[s];
    }
    // the latest completion: max release + the sum over jobs and stages of the slowest machine
    int64_t horizon = 0, max_rel = 0;
    for (int j = 0; j < n; ++j) {
        int off = 0;
        for (int s = 0; s < S; ++s) {
            int64_t worst = 0;
            for (int m = 0; m < M[s]; ++m) {
                const int32_t v = p_u[(int64_t)j * W + off + m];
                if (v < 1) return set_error(FFS_EINVAL, "proc_time[%d][%d][%d] = %d < 1", j, s, m, v);
                if (v > 65535) return set_error(FFS_EUNSUPPORTED, "proc_time[%d][%d][%d] = %d > 65535", j, s, m, v);
                worst = std::max<int64_t>(worst, v);
            }
            horizon += worst;
            off += M[s];
        }
    }
    for (int j = 0; release && j < n; ++j) {
        if (release[j] < 0) return set_error(FFS_EINVAL, "release[%d] = %d < 0", j, release[j]);
        max_rel = std::max<int64_t>(max_rel, release[j]);
    }
    for (int j = 0; due && j < n; ++j)
        if (due[j] < 0) return set_error(FFS_EINVAL, "due[%d] = %d < 0", j, due[j]);
    horizon += max_rel;
    int bits = 0;
    while ((1 << bits) <= n) ++bits;
    const int SH = bits + 1;
    if (horizon >= (int64_t(1) << (32 - SH)))
        return set_error(FFS_EOVERFLOW, "latest completion bound %lld needs more than %d bits of key",
                         (long long)horizon, 32 - SH);
    if ((due ? (int64_t)wt * n * horizon : 0) + horizon > INT32_MAX)
        return set_error(FFS_EOVERFLOW, "objective bound exceeds int32");

    ffs_assign_instance *A = new ffs_assign_instance();
    A->n = n;
    A->S = S;
    A->W = W;
    for (int s = 0; s < S; ++s) A->MX = std::max(A->MX, M[s]);
    A->SH = SH;
    A->wt = due ? wt : 0;
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&A->num_sms, cudaDevAttrMultiProcessorCount, dev);
    std::vector<int32_t> off(S);
    for (int s = 0, acc = 0; s < S; ++s) {
        off[s] = acc;
        acc += M[s];
    }
    std::vector<uint16_t> p16((size_t)n * W);
    for (size_t i = 0; i < p16.size(); ++i) p16[i] = (uint16_t)p_u[i];
    std::vector<uint32_t> order0(n);
    for (int j = 0; j < n; ++j)
        order0[j] = ((uint32_t)(release ? release[j] : 0) << SH) | ((uint32_t)(j + 1) << 1);
    std::sort(order0.begin(), order0.end());   // (R_j, j) ascending: the stage-1 arrival order
    // scratch per thread (= per row of a chunk): 2n stream keys and the row's
    // stage-major genes; two blocks per SM, at most kAssignScratchCap bytes
    A->nstride = (n + 15) / 16 * 16;
    int64_t threads = (int64_t)A->num_sms * 2 * kAssignThreads;
    const int64_t per_keys = (int64_t)2 * n * 4, per_genes = (int64_t)S * A->nstride;
    const int64_t per = per_keys + per_genes;
    threads = std::min<int64_t>(threads, (int64_t)(kAssignScratchCap / per) / kAssignThreads * kAssignThreads);
    if (threads < kAssignThreads) threads = kAssignThreads;
    A->scratch_threads = threads;
    bool ok = cudaMalloc(&A->d_M, 4 * S) == cudaSuccess && cudaMalloc(&A->d_off, 4 * S) == cudaSuccess &&
              cudaMalloc(&A->d_p, p16.size() * 2) == cudaSuccess && cudaMalloc(&A->d_order0, 4 * n) == cudaSuccess &&
              (!due || cudaMalloc(&A->d_due, 4 * n) == cudaSuccess) &&
              cudaMalloc(&A->d_scratch, (size_t)threads * per_keys) == cudaSuccess &&
              cudaMalloc(&A->d_tpop, (size_t)threads * per_genes) == cudaSuccess;
    ok = ok && cudaMemcpy(A->d_M, M, 4 * S, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(A->d_off, off.data(), 4 * S, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(A->d_p, p16.data(), p16.size() * 2, cudaMemcpyHostToDevice) == cudaSuccess &&
         cudaMemcpy(A->d_order0, order0.data(), 4 * n, cudaMemcpyHostToDevice) == cudaSuccess &&
         (!due || cudaMemcpy(A->d_due, due, 4 * n, cudaMemcpyHostToDevice) == cudaSuccess);
    if (!ok) {
        (void)cudaGetLastError();
        ffs_assign_instance_destroy(A);
        return set_error(FFS_ENOMEM, "assignment instance device buffers");
    }
    *out = A;
    return FFS_OK;
}

int ffs_assign_instance_destroy(ffs_assign_instance *A)
{
    if (!A) return FFS_OK;
    cudaFree(A->d_M);
    cudaFree(A->d_off);
    cudaFree(A->d_p);
    cudaFree(A->d_order0);
    cudaFree(A->d_due);
    cudaFree(A->d_scratch);
    cudaFree(A->d_tpop);
    delete A;
    return FFS_OK;
}

int ffs_assign_eval(const ffs_assign_instance *A, const int16_t *pop, int64_t N, int32_t ld, int32_t *objective,
                    ffs_stream stream)
{
    clear_error();
    if (!A) return set_error(FFS_EINVAL, "NULL instance");
    if (N < 0) return set_error(FFS_EINVAL, "N = %lld < 0", (long long)N);
    if (N == 0) return FFS_OK;
    if (!pop || !objective) return set_error(FFS_EINVAL, "NULL population or output");
    if ((int64_t)ld < (int64_t)A->n * A->S || (ld & 7))
        return set_error(FFS_EINVAL, "ld = %d must be >= n * S = %lld and a multiple of 8", ld,
                         (long long)A->n * A->S);
    AssignView V;
    V.n = A->n;
    V.S = A->S;
    V.W = A->W;
    V.SH = A->SH;
    V.wt = (uint32_t)A->wt;
    V.M = A->d_M;
    V.off = A->d_off;
    V.p = A->d_p;
    V.order0 = A->d_order0;
    V.due = A->d_due;
    // shared memory: 7 * MX words per thread, plus n gene bytes and the
    // stage's table slice (shared by the block) when they still leave room
    // for two blocks per SM
    const size_t base = (size_t)7 * A->MX * 4 * kAssignThreads;
    const size_t genes = (size_t)((A->n + 3) / 4 * 4) * kAssignThreads;
    const size_t slice = ((size_t)A->n * A->MX * 2 + 15) / 16 * 16;
    const int mode = base + genes + slice <= 110 * 1024 ? 2 : base + genes <= 110 * 1024 ? 1 : 0;
    const size_t smem = base + (mode >= 1 ? genes : 0) + (mode == 2 ? slice : 0);
    const void *kern = mode == 2 ? (const void *)k_eval_assign<true, true>
                     : mode == 1 ? (const void *)k_eval_assign<true, false> : (const void *)k_eval_assign<false, false>;
    cudaStream_t st = (cudaStream_t)stream;
    FFS_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    // chunks of scratch_threads rows: stage-major copy, then one thread per row
    for (int64_t r0 = 0; r0 < N; r0 += A->scratch_threads) {
        const int64_t cnt = std::min<int64_t>(A->scratch_threads, N - r0);
        k_assign_transpose<<<(unsigned)cnt, 256, 0, st>>>(pop + r0 * ld, ld, A->n, A->S, A->nstride, A->d_tpop);
        FFS_CUDA_TRY(cudaGetLastError());
        const int grid = (int)((cnt + kAssignThreads - 1) / kAssignThreads);
        if (mode == 2)
            k_eval_assign<true, true><<<grid, kAssignThreads, smem, st>>>(V, A->d_tpop, cnt, A->nstride,
                                                                          objective + r0, A->d_scratch, A->MX);
        else if (mode == 1)
            k_eval_assign<true, false><<<grid, kAssignThreads, smem, st>>>(V, A->d_tpop, cnt, A->nstride,
                                                                           objective + r0, A->d_scratch, A->MX);
        else
            k_eval_assign<false, false><<<grid, kAssignThreads, smem, st>>>(V, A->d_tpop, cnt, A->nstride,
                                                                            objective + r0, A->d_scratch, A->MX);
        FFS_CUDA_TRY(cudaGetLastError());
    }
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

// ---------------------------------------------------------------------------
// GA on the paper's genotype (Section 4.1, genotype level): rows of L = n S
// machine genes.  The paper names no operators for it; this library reads
// them as random initial machines, complementary pairs by reflection
// (M_s - 1 - m: the binary layer's bitwise complement when M_s is a power of
// two), two-point crossover (the segment [l, r] from the first parent, the
// rest from the second) and one-gene machine reassignment, with the draws,
// tournaments and replacement rules of the job-order GA.  A generation is a
// breeding launch (children into caller scratch), the evaluator of
// ffs_assign_eval on the children, and a replacement launch.
// ---------------------------------------------------------------------------
namespace fgpu {

// Initial rows: kind 0, row r: gene i = uniform(M_{i mod S}) with draw i of
// (seed, purpose 1, island, generation 0, cell r); kind 1, pair k = rows 2k,
// 2k + 1: a drawn with cell 2k and its complement.  Thread = (row or pair,
// block of 4 genes); padding genes are 0.
__global__ void k_assign_init(uint64_t seed, uint32_t island, int kind, int64_t units, int n, int S,
                              const int32_t *__restrict__ M, int ld, int16_t *pop)
{
    const int L = n * S, blocks = ld >> 2;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= units * blocks) return;
    const int64_t u = t / blocks;
    const int b = (int)(t - u * blocks);
    const int64_t row = kind == 0 ? u : 2 * u;
    const U4 d = draw_block(seed, kPurposeInit, island, 0u, (uint32_t)row, (uint32_t)b);
    const uint32_t x[4] = {d.x, d.y, d.z, d.w};
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const int i = 4 * b + h;
        int16_t a = 0, c = 0;
        if (i < L) {
            const int Ms = M[i % S];
            a = (int16_t)uniform_below(x[h], (uint32_t)Ms);
            c = (int16_t)(Ms - 1 - a);
        }
        pop[row * ld + i] = a;
        if (kind == 1) pop[(row + 1) * ld + i] = c;
    }
}

// Machine reassignment of gene value `old` at a stage of Ms machines: u =
// uniform(x, Ms - 1), then u if u < old, else u + 1; unchanged when Ms < 2.
__device__ __forceinline__ int16_t assign_reassign(int16_t old, int Ms, uint32_t x)
{
    if (Ms < 2) return old;
    const int u = (int)uniform_below(x, (uint32_t)(Ms - 1));
    return (int16_t)(u < old ? u : u + 1);
}

// Row dst = genes [l, r] of p1 and the others of p2 (l > r: p2 alone), with
// gene `mi` (if >= 0) then reassigned with draw mx; the warp copies 8 genes
// per lane per step (16-byte loads and stores).
__device__ __forceinline__ void warp_two_point(const int16_t *p1, const int16_t *p2, int16_t *dst, int ld, int l,
                                               int r, int mi, const int32_t *M, int S, uint32_t mx)
{
    const int lane = threadIdx.x & 31;
    const int4 *a4 = reinterpret_cast<const int4 *>(p1), *b4 = reinterpret_cast<const int4 *>(p2);
    int4 *d4 = reinterpret_cast<int4 *>(dst);
    for (int q = lane; q < (ld >> 3); q += 32) {
        const int lo = 8 * q;
        if (lo >= l && lo + 7 <= r && (mi < lo || mi > lo + 7)) {
            d4[q] = a4[q];
        } else if ((lo + 7 < l || lo > r) && (mi < lo || mi > lo + 7)) {
            d4[q] = b4[q];
        } else {
            const int4 va = a4[q], vb = b4[q];
            const int16_t *ga = reinterpret_cast<const int16_t *>(&va), *gb = reinterpret_cast<const int16_t *>(&vb);
            int16_t out[8];
#pragma unroll
            for (int h = 0; h < 8; ++h) {
                const int i = lo + h;
                int16_t gv = (i >= l && i <= r) ? ga[h] : gb[h];
                if (i == mi) {
                    gv = assign_reassign(gv, M[i % S], mx);
                    if (!FFS_DCHECK(gv >= 0 && gv < M[i % S], kCheckMachineGene)) gv = 0;
                }
                out[h] = gv;
            }
            d4[q] = *reinterpret_cast<const int4 *>(out);
        }
    }
}

// Cellular children of a torus (one warp per cell): the tournaments and the
// draws of the job-order cellular step (purpose 2): crossover with draw 4,
// cut points uniform in [0, L) from draws 5-6, else a copy of the first
// winner (l > r); mutation with draw 7 reassigns gene uniform(L) (draw 8)
// with draw 9.
__global__ void k_assign_breed_cellular(GaScalars g, uint32_t island, uint32_t gen, int rows, int cols, int n, int S,
                                        const int32_t *__restrict__ M, int ld, const int16_t *__restrict__ pop,
                                        const int32_t *__restrict__ obj, int16_t *children)
{
    const int cells = rows * cols, L = n * S;
    const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (c >= cells) return;
    const U4 b0 = draw_block(g.seed, kPurposeCellular, island, gen, (uint32_t)c, 0u);
    const U4 b1 = draw_block(g.seed, kPurposeCellular, island, gen, (uint32_t)c, 1u);
    const U4 b2 = draw_block(g.seed, kPurposeCellular, island, gen, (uint32_t)c, 2u);
    const int r0 = c / cols, q0 = c - r0 * cols;
    const int up = ((r0 + rows - 1) % rows) * cols + q0, down = ((r0 + 1) % rows) * cols + q0;
    const int west = r0 * cols + (q0 + cols - 1) % cols, east = r0 * cols + (q0 + 1) % cols;
    auto slot = [&](uint32_t x) {
        const uint32_t s = uniform_below(x, 5u);
        return s == 0 ? c : s == 1 ? up : s == 2 ? down : s == 3 ? west : east;
    };
    int a = slot(b0.x), b = slot(b0.y);
    int par1 = (obj[b] < obj[a]) ? b : a;
    a = slot(b0.z);
    b = slot(b0.w);
    int par2 = (obj[b] < obj[a]) ? b : a;
    if (!FFS_DCHECK(par1 >= 0 && par1 < cells && par2 >= 0 && par2 < cells, kCheckParent)) par1 = par2 = c;
    int l = 1, r = 0;     // no crossover: everything from the first winner (passed as p2)
    const int16_t *p1 = pop + (int64_t)par1 * ld, *p2 = p1;
    if (fires(b1.x, g.cell_pc)) {
        const int u = (int)uniform_below(b1.y, (uint32_t)L), v = (int)uniform_below(b1.z, (uint32_t)L);
        l = min(u, v);
        r = max(u, v);
        p2 = pop + (int64_t)par2 * ld;
    }
    const int mi = fires(b1.w, g.cell_pm) ? (int)uniform_below(b2.x, (uint32_t)L) : -1;
    warp_two_point(p1, p2, children + (int64_t)c * ld, ld, l, r, mi, M, S, b2.y);
}

// Pseudo children (one warp per pair k): crossover with draw 0 (purpose 3),
// cut points from draws 1-2: c1 = two-point(a, b), c2 = two-point(b, a) into
// children rows 2k, 2k + 1; pairs that do not cross copy a, b there.
// cross[k] records the outcome.
__global__ void k_assign_breed_pseudo(GaScalars g, uint32_t island, uint32_t gen, int pairs, int n, int S, int ld,
                                      const int16_t *__restrict__ pop, int16_t *children, uint8_t *cross)
{
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= pairs) return;
    const int L = n * S;
    const U4 d = draw_block(g.seed, kPurposePseudo, island, gen, (uint32_t)k, 0u);
    const int16_t *A = pop + (int64_t)(2 * k) * ld, *B = A + ld;
    int16_t *c1 = children + (int64_t)(2 * k) * ld, *c2 = c1 + ld;
    const bool x = fires(d.x, g.pseudo_pc);
    int l = 1, r = 0;
    if (x) {
        const int u = (int)uniform_below(d.y, (uint32_t)L), v = (int)uniform_below(d.z, (uint32_t)L);
        l = min(u, v);
        r = max(u, v);
    }
    // no crossover: l > r copies the second argument
    warp_two_point(x ? A : B, x ? B : A, c1, ld, l, r, -1, nullptr, S, 0u);
    warp_two_point(x ? B : A, x ? A : B, c2, ld, l, r, -1, nullptr, S, 0u);
    if ((threadIdx.x & 31) == 0) cross[k] = x ? 1 : 0;
}

__device__ __forceinline__ void warp_copy_row(const int16_t *src, int16_t *dst, int ld)
{
    const int4 *s4 = reinterpret_cast<const int4 *>(src);
    int4 *d4 = reinterpret_cast<int4 *>(dst);
    for (int q = (threadIdx.x & 31); q < (ld >> 3); q += 32) d4[q] = s4[q];
}

// Cellular replacement (one warp per cell): the child iff its objective is
// lower (flag: not higher) than the cell's.
__global__ void k_assign_replace_cellular(int cells, int ld, int replace_le, const int16_t *__restrict__ pop_in,
                                          const int32_t *__restrict__ obj_in, const int16_t *__restrict__ children,
                                          const int32_t *__restrict__ child_obj, int16_t *pop_out, int32_t *obj_out)
{
    const int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (c >= cells) return;
    const int32_t mc = child_obj[c], mo = obj_in[c];
    const bool better = mc >= 0 && (replace_le ? mc <= mo : mc < mo);
    warp_copy_row(better ? children + (int64_t)c * ld : pop_in + (int64_t)c * ld, pop_out + (int64_t)c * ld, ld);
    if ((threadIdx.x & 31) == 0) obj_out[c] = better ? mc : mo;
}

// Pseudo replacement (one warp per pair): a pair that crossed keeps the two
// best of (c1, c2, a, b) ranked by (objective, that order), best first -- or
// the children with `always`; a pair that did not cross is copied.
__global__ void k_assign_replace_pseudo(int pairs, int ld, int always, const int16_t *__restrict__ pop_in,
                                        const int32_t *__restrict__ obj_in, const int16_t *__restrict__ children,
                                        const int32_t *__restrict__ child_obj, const uint8_t *__restrict__ cross,
                                        int16_t *pop_out, int32_t *obj_out)
{
    const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (k >= pairs) return;
    const int16_t *fam[4] = {children + (int64_t)(2 * k) * ld, children + (int64_t)(2 * k + 1) * ld,
                             pop_in + (int64_t)(2 * k) * ld, pop_in + (int64_t)(2 * k + 1) * ld};
    const int32_t fo[4] = {child_obj[2 * k], child_obj[2 * k + 1], obj_in[2 * k], obj_in[2 * k + 1]};
    int first = 2, second = 3;
    if (cross[k]) {
        if (always) {
            first = 0;
            second = 1;
        } else {
            first = 0;
            for (int t = 1; t < 4; ++t)
                if (fo[t] < fo[first]) first = t;
            second = -1;
            for (int t = 0; t < 4; ++t)
                if (t != first && (second < 0 || fo[t] < fo[second])) second = t;
        }
    }
    warp_copy_row(fam[first], pop_out + (int64_t)(2 * k) * ld, ld);
    warp_copy_row(fam[second], pop_out + (int64_t)(2 * k + 1) * ld, ld);
    if ((threadIdx.x & 31) == 0) {
        obj_out[2 * k] = fo[first];
        obj_out[2 * k + 1] = fo[second];
    }
}

static int64_t a256(int64_t b) { return (b + 255) / 256 * 256; }

}  // namespace fgpu

extern "C" {

int64_t ffs_assign_step_scratch_bytes(int64_t N, int32_t ld)
{
    if (N < 0 || ld < 0) return -1;
    return a256(N * ld * 2) + a256(N * 4) + a256(N / 2 + 1);
}

int ffs_assign_population_init(const ffs_assign_instance *A, uint64_t seed, uint32_t island, int32_t kind, int64_t N,
                               int32_t ld, int16_t *pop, ffs_stream stream)
{
    clear_error();
    if (!A || !pop) return set_error(FFS_EINVAL, "NULL argument");
    if (kind != 0 && kind != 1) return set_error(FFS_EINVAL, "kind %d", kind);
    if (N < 0 || (kind == 1 && (N & 1))) return set_error(FFS_EINVAL, "N = %lld (even for pseudo pairs)", (long long)N);
    int rc = validate_rows(pop, ld, A->n * A->S);
    if (rc) return rc;
    if (N == 0) return FFS_OK;
    const int64_t units = kind == 0 ? N : N / 2;
    const int64_t threads = units * (ld / 4);
    k_assign_init<<<(unsigned)((threads + 255) / 256), 256, 0, (cudaStream_t)stream>>>(seed, island, kind, units, A->n,
                                                                                        A->S, A->d_M, ld, pop);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

int ffs_assign_cellular_step(const ffs_assign_instance *A, const ffs_params *prm, uint32_t island, uint32_t generation,
                             int32_t rows, int32_t cols, int32_t ld, const int16_t *pop_in, const int32_t *obj_in,
                             int16_t *pop_out, int32_t *obj_out, void *scratch, ffs_stream stream)
{
    clear_error();
    if (!A || !prm || !pop_in || !obj_in || !pop_out || !obj_out || !scratch) return set_error(FFS_EINVAL, "NULL argument");
    if (rows < 1 || cols < 1 || (int64_t)rows * cols > (1 << 26)) return set_error(FFS_EINVAL, "bad torus %dx%d", rows, cols);
    if (pop_in == pop_out) return set_error(FFS_EINVAL, "pop_in and pop_out must differ");
    if (((uintptr_t)scratch & 255u) != 0) return set_error(FFS_EINVAL, "scratch must be 256-byte aligned");
    const int L = A->n * A->S;
    int rc = validate_rows(pop_in, ld, L);
    if (rc) return rc;
    if ((rc = validate_rows(pop_out, ld, L))) return rc;
    const int64_t cells = (int64_t)rows * cols;
    char *sp = static_cast<char *>(scratch);
    int16_t *children = reinterpret_cast<int16_t *>(sp);
    int32_t *child_obj = reinterpret_cast<int32_t *>(sp + a256(cells * ld * 2));
    cudaStream_t st = (cudaStream_t)stream;
    const GaScalars g = scalars_of(prm);
    const unsigned blocks = (unsigned)((cells * 32 + 255) / 256);
    k_assign_breed_cellular<<<blocks, 256, 0, st>>>(g, island, generation, rows, cols, A->n, A->S, A->d_M, ld, pop_in,
                                                    obj_in, children);
    FFS_CUDA_TRY(cudaGetLastError());
    if ((rc = ffs_assign_eval(A, children, cells, ld, child_obj, stream))) return rc;
    k_assign_replace_cellular<<<blocks, 256, 0, st>>>((int)cells, ld, prm->cell_replace_le, pop_in, obj_in, children,
                                                      child_obj, pop_out, obj_out);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

int ffs_assign_pseudo_step(const ffs_assign_instance *A, const ffs_params *prm, uint32_t island, uint32_t generation,
                           int32_t size, int32_t ld, const int16_t *pop_in, const int32_t *obj_in, int16_t *pop_out,
                           int32_t *obj_out, void *scratch, ffs_stream stream)
{
    clear_error();
    if (!A || !prm || !pop_in || !obj_in || !pop_out || !obj_out || !scratch) return set_error(FFS_EINVAL, "NULL argument");
    if (size < 2 || (size & 1)) return set_error(FFS_EINVAL, "pseudo island size %d must be even and >= 2", size);
    if (pop_in == pop_out) return set_error(FFS_EINVAL, "pop_in and pop_out must differ");
    if (((uintptr_t)scratch & 255u) != 0) return set_error(FFS_EINVAL, "scratch must be 256-byte aligned");
    const int L = A->n * A->S;
    int rc = validate_rows(pop_in, ld, L);
    if (rc) return rc;
    if ((rc = validate_rows(pop_out, ld, L))) return rc;
    char *sp = static_cast<char *>(scratch);
    int16_t *children = reinterpret_cast<int16_t *>(sp);
    int32_t *child_obj = reinterpret_cast<int32_t *>(sp + a256((int64_t)size * ld * 2));
    uint8_t *cross = reinterpret_cast<uint8_t *>(sp + a256((int64_t)size * ld * 2) + a256((int64_t)size * 4));
    cudaStream_t st = (cudaStream_t)stream;
    const GaScalars g = scalars_of(prm);
    const int pairs = size / 2;
    const unsigned blocks = (unsigned)(((int64_t)pairs * 32 + 255) / 256);
    k_assign_breed_pseudo<<<blocks, 256, 0, st>>>(g, island, generation, pairs, A->n, A->S, ld, pop_in, children, cross);
    FFS_CUDA_TRY(cudaGetLastError());
    if ((rc = ffs_assign_eval(A, children, size, ld, child_obj, stream))) return rc;
    k_assign_replace_pseudo<<<blocks, 256, 0, st>>>(pairs, ld, prm->pseudo_always, pop_in, obj_in, children, child_obj,
                                                    cross, pop_out, obj_out);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

}  // extern "C"
