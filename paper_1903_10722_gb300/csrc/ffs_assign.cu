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
