// ffs_probe.cu -- measurements and self-tests that keep the performance and
// failure-handling claims checkable: the integer issue rate of this GPU per
// instruction kind, and a bounded wait that is made to run out.
#include "ffs_internal.cuh"
#include "ffs_tc.cuh"

namespace fgpu {

// Eight independent chains per thread of one 32-bit operation;
// `kind` 0: min/max, 1: three-input logic, 2: three-input add, 3: multiply-add,
// 4: fp32 min/max on the same bit patterns (non-negative finite keys order as
// floats the way they order as integers), 5: packed 16-bit min/max (two
// halves per word), 6: three-input min/max, 7: add-then-max, 8: min/max and
// multiply-add alternating between chains, 9: integer and fp32 min/max
// alternating.  Kinds 8 and 9 show whether two operation kinds issue to
// separate pipes (their mixed rate then exceeds either one alone).
template <int KIND>
__global__ void __launch_bounds__(512) k_int_rate(int iters, uint32_t seed, uint32_t *sink)
{
    uint32_t a[8], b = seed ^ (threadIdx.x * 0x9E3779B9u), c = seed + blockIdx.x;
    if constexpr (KIND == 4 || KIND == 9) {
        // finite non-negative float patterns
        b &= 0x3FFFFFFFu;
        c &= 0x3FFFFFFFu;
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = (KIND == 4 || KIND == 9) ? ((b + j * 0x85EBCA6Bu) & 0x3FFFFFFFu)
                                                              : b + j * 0x85EBCA6Bu;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if constexpr (KIND == 0) a[j] = (u & 1) ? min(a[j], b) : max(a[j], c);
                else if constexpr (KIND == 1) a[j] = (a[j] ^ b) & (c | a[j]);
                else if constexpr (KIND == 2) a[j] = a[j] + a[(j + 1) & 7] + c;
                else if constexpr (KIND == 3) a[j] = a[j] * b + c;
                else if constexpr (KIND == 4)
                    a[j] = __float_as_uint((u & 1) ? fminf(__uint_as_float(a[j]), __uint_as_float(b))
                                                   : fmaxf(__uint_as_float(a[j]), __uint_as_float(c)));
                else if constexpr (KIND == 5) a[j] = (u & 1) ? __vminu2(a[j], b) : __vmaxu2(a[j], c);
                else if constexpr (KIND == 6)
                    a[j] = (u & 1) ? __vimin3_u32(a[j], b, a[(j + 1) & 7]) : __vimax3_u32(a[j], c, a[(j + 3) & 7]);
                else if constexpr (KIND == 7) a[j] = __viaddmax_u32(a[j], b, c);
                else if constexpr (KIND == 8)
                    a[j] = (j & 1) ? a[j] * b + c : ((u & 1) ? min(a[j], b) : max(a[j], c));
                else
                    a[j] = (j & 1) ? __float_as_uint((u & 1) ? fminf(__uint_as_float(a[j]), __uint_as_float(b))
                                                             : fmaxf(__uint_as_float(a[j]), __uint_as_float(c)))
                                   : ((u & 1) ? min(a[j], b) : max(a[j], c));
            }
        }
        b += 1u;
        c ^= b;
        if constexpr (KIND == 4 || KIND == 9) {
            b &= 0x3FFFFFFFu;
            c &= 0x3FFFFFFFu;
        }
    }
    uint32_t r = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) r ^= a[j];
    if (r == 0x12345678u) sink[0] = r;   // keeps the chains live
}

// One bounded wait on an mbarrier that nothing will complete: it must give
// up after limit_ns and report status 1 (0 would mean the phase completed).
__global__ void k_wait_timeout_selftest(uint64_t limit_ns, int *status)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        tc::mbar_init(&bar, 1);
        tc::mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) status[0] = tc::mbar_wait(&bar, 0, limit_ns) ? 0 : 1;
}

}  // namespace fgpu

using namespace fgpu;

extern "C" {

int ffs_measure_int_rate(int32_t kind, double *lane_ops_per_s, float *ms, ffs_stream stream)
{
    clear_error();
    if (kind < 0 || kind > 9 || !lane_ops_per_s) return set_error(FFS_EINVAL, "kind %d", kind);
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, sms = 0;
    FFS_CUDA_TRY(cudaGetDevice(&dev));
    FFS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    uint32_t *sink = nullptr;
    FFS_CUDA_TRY(cudaMallocAsync(&sink, 4, st));
    const int T = 512, blocks = sms * 4, iters = 2048;
    cudaEvent_t e0, e1;
    FFS_CUDA_TRY(cudaEventCreate(&e0));
    FFS_CUDA_TRY(cudaEventCreate(&e1));
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
        cudaEventRecord(e0, st);
        switch (kind) {
        case 0: k_int_rate<0><<<blocks, T, 0, st>>>(iters, 7u, sink); break;
        case 1: k_int_rate<1><<<blocks, T, 0, st>>>(iters, 7u, sink); break;
        case 2: k_int_rate<2><<<blocks, T, 0, st>>>(iters, 7u, sink); break;
        case 3: k_int_rate<3><<<blocks, T, 0, st>>>(iters, 7u, sink); break;
        case 4: k_int_rate<4><<<blocks, T, 0, st>>>(iters, 7u, sink); break;
        case 5: k_int_rate<5><<<blocks, T, 0, st>>>(iters, 7u, sink); break;
        case 6: k_int_rate<6><<<blocks, T, 0, st>>>(iters, 7u, sink); break;
        case 7: k_int_rate<7><<<blocks, T, 0, st>>>(iters, 7u, sink); break;
        case 8: k_int_rate<8><<<blocks, T, 0, st>>>(iters, 7u, sink); break;
        default: k_int_rate<9><<<blocks, T, 0, st>>>(iters, 7u, sink); break;
        }
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float t = 0.0f;
        cudaEventElapsedTime(&t, e0, e1);
        if (t < best) best = t;
    }
    const cudaError_t err = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(sink, st);
    if (err != cudaSuccess) return set_error(FFS_ECUDA, "int rate kernel: %s", cudaGetErrorString(err));
    // one source-level operation per chain update (kind 2's two adds and kind
    // 7's add-then-max are counted once: one instruction where the hardware has it)
    const double per_update = 1.0;
    const double ops = (double)blocks * T * iters * 16.0 * 8.0 * per_update;
    *lane_ops_per_s = ops / (best * 1e-3);
    if (ms) *ms = best;
    return FFS_OK;
}

int ffs_selftest_wait_timeout(int64_t limit_ns, int32_t *status, ffs_stream stream)
{
    clear_error();
    if (!status || limit_ns <= 0 || limit_ns > 2000000000ll) return set_error(FFS_EINVAL, "bad arguments");
    int *d = nullptr;
    cudaStream_t st = (cudaStream_t)stream;
    FFS_CUDA_TRY(cudaMallocAsync(&d, 4, st));
    FFS_CUDA_TRY(cudaMemsetAsync(d, 0xFF, 4, st));
    k_wait_timeout_selftest<<<1, 32, 0, st>>>((uint64_t)limit_ns, d);
    FFS_CUDA_TRY(cudaGetLastError());
    FFS_CUDA_TRY(cudaMemcpyAsync(status, d, 4, cudaMemcpyDeviceToHost, st));
    FFS_CUDA_TRY(cudaFreeAsync(d, st));
    FFS_CUDA_TRY(cudaStreamSynchronize(st));
    return *status == 1 ? FFS_ETIMEOUT : FFS_OK;
}

}  // extern "C"
