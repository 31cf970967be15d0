// ffs_noalloc.cu -- a pseudo-island generation for callers that cannot
// allocate device memory.
//
// ffs_pseudo_step needs scratch memory (the compacted children, their
// makespans, the pair-to-slot map and a counter) that its caller provides.
// Some callers cannot provide it: code running where cudaMalloc is not
// allowed or not wanted -- inside a host callback, a real-time loop that
// must not block on the allocator, or a plugin whose host framework owns
// every allocation.  ffs_pseudo_step_noalloc runs the same kernels with the
// scratch in a fixed array compiled into this library instead.
//
// The array is a file-scope __device__ variable: every GPU that loads the
// library holds its FFS_NOALLOC_SCRATCH_BYTES until the process exits, and
// every call on that GPU shares it.
#include <cstring>
#include <mutex>

#include "ffs_internal.cuh"

namespace fgpu {

static __device__ __align__(256) unsigned char g_noalloc_scratch[FFS_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch per device ordinal.  In host code the
// array's name is only a host-side stand-in, so the address comes from
// cudaGetSymbolAddress, taken once per device with that device current.
constexpr int kMaxDevices = 64;
static std::mutex g_noalloc_mutex;
static void *g_noalloc_addr[kMaxDevices] = {};

static int noalloc_scratch_address(void **out)
{
    int dev = -1;
    FFS_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return set_error(FFS_EUNSUPPORTED, "device ordinal %d", dev);
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return set_error(FFS_ECUDA, "cudaGetSymbolAddress of the fixed scratch failed: %s",
                             cudaGetErrorString(e));
        g_noalloc_addr[dev] = p;
    }
    *out = g_noalloc_addr[dev];
    return FFS_OK;
}

}  // namespace fgpu

using namespace fgpu;

extern "C" int ffs_pseudo_step_noalloc(const ffs_instance *I, const ffs_params *prm, uint32_t island,
                                       uint32_t generation, int32_t size, int32_t ld, const int16_t *pop_in,
                                       const int32_t *ms_in, int16_t *pop_out, int32_t *ms_out, ffs_stream stream)
{
    clear_error();
    if (!I || !prm || !pop_in || !ms_in || !pop_out || !ms_out) return set_error(FFS_EINVAL, "NULL argument");
    if (size < 2 || (size & 1)) return set_error(FFS_EINVAL, "pseudo island size %d must be even and >= 2", size);
    if (pop_in == pop_out) return set_error(FFS_EINVAL, "pop_in and pop_out must differ");
    int rc = validate_rows(pop_in, ld, I->n);
    if (rc) return rc;
    if ((rc = validate_rows(pop_out, ld, I->n))) return rc;
    const int64_t need = pseudo_scratch_bytes(size, ld, 1);
    if (need > (int64_t)FFS_NOALLOC_SCRATCH_BYTES)
        return set_error(FFS_EUNSUPPORTED,
                         "island of %d rows x %d genes needs %lld bytes of scratch; the fixed array holds %lld",
                         size, ld, (long long)need, (long long)FFS_NOALLOC_SCRATCH_BYTES);
    void *scratch = nullptr;
    if ((rc = noalloc_scratch_address(&scratch))) return rc;
    IslandBatch b;
    memset(&b, 0, sizeof(b));
    b.count = 1;
    IslandRef &r = b.ref[0];
    r.pop_in = pop_in;
    r.ms_in = ms_in;
    r.pop_out = pop_out;
    r.ms_out = ms_out;
    r.generation = generation;
    r.island = island;
    // launch_pseudo zeroes the slot counter on the stream before the kernels read it
    return launch_pseudo(I, scalars_of(prm), b, size, ld, scratch, prm->decode_chunk, prm->block_threads, nullptr,
                         (cudaStream_t)stream);
}
