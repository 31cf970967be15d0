// ffs_probe.cu -- measurements and self-tests that keep the performance and
// failure-handling claims checkable: the integer issue rate of this GPU per
// instruction kind, and a bounded wait that is made to run out.
#include "ffs_internal.cuh"
#include "ffs_tc.cuh"

namespace fgpu {

// Eight independent chains per thread of one 32-bit integer operation;
// `kind` 0: min/max, 1: three-input logic, 2: three-input add, 3: multiply-add.
template <int KIND>
__global__ void __launch_bounds__(512) k_int_rate(int iters, uint32_t seed, uint32_t *sink)
{
    uint32_t a[8], b = seed ^ (threadIdx.x * 0x9E3779B9u), c = seed + blockIdx.x;
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = b + j * 0x85EBCA6Bu;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                if constexpr (KIND == 0) a[j] = (u & 1) ? min(a[j], b) : max(a[j], c);
                else if constexpr (KIND == 1) a[j] = (a[j] ^ b) & (c | a[j]);
                else if constexpr (KIND == 2) a[j] = a[j] + a[(j + 1) & 7] + c;
                else a[j] = a[j] * b + c;
            }
        }
        b += 1u;
        c ^= b;
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
    if (kind < 0 || kind > 3 || !lane_ops_per_s) return set_error(FFS_EINVAL, "kind %d", kind);
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
        default: k_int_rate<3><<<blocks, T, 0, st>>>(iters, 7u, sink); break;
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
    // source-level operations: kind 0..1 one per update, kind 2 two adds, kind 3 one multiply-add
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
