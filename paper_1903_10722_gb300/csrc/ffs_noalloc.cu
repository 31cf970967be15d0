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
#include <utility>
#include <vector>

#include <cuda.h>

#include "ffs_internal.cuh"

namespace fgpu {

static __device__ __align__(256) unsigned char g_noalloc_scratch[FFS_NOALLOC_SCRATCH_BYTES];

// Device address of g_noalloc_scratch in the current CUDA context.  In host
// code the array's name is only a host-side stand-in, so the address comes
// from cudaGetSymbolAddress, taken with the device current.  It is cached per
// context, keyed on the driver's context ID (unique for the life of the
// process, never reused), so a call under another context -- a non-primary
// one, or the primary context created anew after cudaDeviceReset -- looks
// the address up again instead of using one that belongs to a dead or
// different context.
typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

static std::mutex g_noalloc_mutex;
static std::vector<std::pair<unsigned long long, void *>> g_noalloc_addr;   // (context ID, address)

static bool current_context_id(unsigned long long *id)
{
    static std::once_flag once;
    static CtxGetCurrentFn get_current = nullptr;
    static CtxGetIdFn get_id = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_current = reinterpret_cast<CtxGetCurrentFn>(p);
        p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            get_id = reinterpret_cast<CtxGetIdFn>(p);
        (void)cudaGetLastError();
    });
    CUcontext ctx = nullptr;
    if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx) return false;
    return get_id(ctx, id) == CUDA_SUCCESS;
}

static int noalloc_scratch_address(void **out)
{
    int dev = -1;
    FFS_CUDA_TRY(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    unsigned long long id = 0;
    const bool have_id = current_context_id(&id);
    if (have_id)
        for (const auto &e : g_noalloc_addr)
            if (e.first == id) {
                *out = e.second;
                return FFS_OK;
            }
    // first call in this context (cudaGetSymbolAddress also initialises the
    // device's primary context when no context is current yet)
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
        return set_error(FFS_ECUDA, "cudaGetSymbolAddress of the fixed scratch failed on device %d: %s", dev,
                         cudaGetErrorString(e));
    if (have_id || current_context_id(&id)) g_noalloc_addr.emplace_back(id, p);
    *out = p;
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
