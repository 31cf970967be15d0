// ffs_mlp.cu -- the surrogate network: a BF16 GEMM on the 5th-generation
// tensor cores (TMA -> shared memory -> tcgen05.mma -> TMEM -> registers)
// and the small MLP built on it (in -> h1 -> h2 -> 1, ReLU, BF16 weights and
// activations, FP32 accumulation), trained online with Adam on MSE.
//
// Every GEMM here is D[M][N] = A[M][K] * B[N][K]^T with both operands
// K-major (rows of K contiguous BF16); the backward pass transposes its
// operands into that layout with small CUDA-core kernels.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "ffs_internal.cuh"
#include "ffs_tc.cuh"

namespace fgpu {

constexpr int kGemmStages = 4;
constexpr int kBM = 128, kBK = 64;
constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s per wait

struct GemmEpi {
    float *D;                 // mode 0: FP32 output [M][ldd]
    __nv_bfloat16 *Db;        // mode 1: BF16 relu(acc + bias) [M][ldd]
    const float *bias;        // modes 1, 2: [N]
    const float *w3, *b3;     // mode 2 (persistent form, one column tile): y[row] =
    float *y;                 //   sum_c BF16(relu(acc + bias))[c] w3[c] + b3, H never stored
    // mode 3 (a hidden layer's backpropagated signal): z = acc [mask > 0],
    // FP32 into D [M][ldd] and BF16 transposed into Dt [N][ldt]
    const __nv_bfloat16 *mask;
    int ldm, ldt;
    __nv_bfloat16 *Dt;
    int ldd;
    int M_valid;
    int mode;
    int *err;                 // set to a non-zero code if a wait timed out
    int max_ctas;             // host: CTAs of the persistent form at most (0: one per SM)
    int pdl;                  // host: launch as a programmatic dependent of the stream's previous kernel
};

template <int BN>
struct GemmSmem {
    static constexpr uint32_t A_BYTES = kBM * kBK * 2;
    static constexpr uint32_t B_BYTES = BN * kBK * 2;
    static constexpr uint32_t TCOLS = BN <= 32 ? 32 : BN <= 64 ? 64 : BN <= 128 ? 128 : 256;
    static constexpr size_t BYTES = 1024 + kGemmStages * (A_BYTES + B_BYTES) + 256;
};

// 32 accumulator columns of one row (col .. col + 31 of the output) to
// memory: FP32 as they are (mode 0) or BF16 relu(acc + bias) (mode 1, the
// bias slice starting at `bias`).
__device__ __forceinline__ void gemm_store_32(const GemmEpi &epi, int row, int col, const float (&v)[32],
                                              const float *bias)
{
    if (epi.mode == 0) {
        float4 *dst = reinterpret_cast<float4 *>(epi.D + (size_t)row * epi.ldd + col);
#pragma unroll
        for (int q = 0; q < 8; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else if (epi.mode == 3) {
        const uint4 *hm = reinterpret_cast<const uint4 *>(epi.mask + (size_t)row * epi.ldm + col);
        uint32_t hw[16];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 x = hm[q];
            hw[4 * q] = x.x;
            hw[4 * q + 1] = x.y;
            hw[4 * q + 2] = x.z;
            hw[4 * q + 3] = x.w;
        }
        float z[32];
#pragma unroll
        for (int j = 0; j < 32; ++j) {
            const float h = __uint_as_float((j & 1) ? (hw[j >> 1] & 0xFFFF0000u) : (hw[j >> 1] << 16));
            z[j] = h > 0.0f ? v[j] : 0.0f;
        }
        float4 *dst = reinterpret_cast<float4 *>(epi.D + (size_t)row * epi.ldd + col);
#pragma unroll
        for (int q = 0; q < 8; ++q) dst[q] = make_float4(z[4 * q], z[4 * q + 1], z[4 * q + 2], z[4 * q + 3]);
        // column j of the warp's 32 rows: 32 consecutive BF16 of Dt's row col + j
#pragma unroll
        for (int j = 0; j < 32; ++j) epi.Dt[(size_t)(col + j) * epi.ldt + row] = __float2bfloat16_rn(z[j]);
    } else {
        uint32_t packed[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
            const float x0 = fmaxf(v[2 * q] + bias[2 * q], 0.0f);
            const float x1 = fmaxf(v[2 * q + 1] + bias[2 * q + 1], 0.0f);
            const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
            packed[q] = *reinterpret_cast<const uint32_t *>(&h);
        }
        uint4 *dst = reinterpret_cast<uint4 *>(epi.Db + (size_t)row * epi.ldd + col);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            dst[q] = make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2], packed[4 * q + 3]);
    }
}

template <int BN>
__global__ void __launch_bounds__(128, 1) k_gemm_bf16(const __grid_constant__ CUtensorMap tmA,
                                                       const __grid_constant__ CUtensorMap tmB, int K, GemmEpi epi)
{
    using SM = GemmSmem<BN>;
    extern __shared__ uint8_t smem_dyn[];
    __shared__ int s_fail;
    __shared__ float s_bias[256];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = base;
    uint8_t *sB = base + kGemmStages * SM::A_BYTES;
    uint64_t *full = reinterpret_cast<uint64_t *>(sB + kGemmStages * SM::B_BYTES);
    uint64_t *empty = full + kGemmStages;
    uint64_t *done = empty + kGemmStages;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
    const int KC = K / kBK;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kGemmStages; ++s) {
            tc::mbar_init(full + s, 1);
            tc::mbar_init(empty + s, 1);
        }
        tc::mbar_init(done, 1);
        tc::mbar_fence_init();
        s_fail = 0;
    }
    if (warp == 0) tc::tmem_alloc(tslot, SM::TCOLS);
    // what follows reads what the kernels before this one wrote
    tc::grid_dep_launch();
    tc::grid_dep_wait();
    // the epilogue's bias slice, read once per CTA
    if (epi.mode == 1)
        for (int c = threadIdx.x; c < BN; c += blockDim.x) s_bias[c] = epi.bias[n0 + c];
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;

    if (warp == 0 && lane == 0) {
        // TMA producer
        for (int kc = 0; kc < KC; ++kc) {
            const int s = kc % kGemmStages;
            if (kc >= kGemmStages && !tc::mbar_wait(empty + s, ((kc / kGemmStages) - 1) & 1, kWaitLimitNs)) {
                s_fail = 1;
                break;
            }
            tc::mbar_expect_tx(full + s, SM::A_BYTES + SM::B_BYTES);
            tc::tma_load_2d(sA + s * SM::A_BYTES, &tmA, kc * kBK, m0, full + s);
            tc::tma_load_2d(sB + s * SM::B_BYTES, &tmB, kc * kBK, n0, full + s);
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: 4 MMAs of K = 16 per 64-wide chunk
        const uint32_t idesc = tc::idesc_bf16_f32(kBM, BN);
        for (int kc = 0; kc < KC; ++kc) {
            const int s = kc % kGemmStages;
            if (!tc::mbar_wait(full + s, (kc / kGemmStages) & 1, kWaitLimitNs)) {
                s_fail = 2;
                break;
            }
            tc::fence_after_sync();
            const uint32_t a0 = tc::smem_u32(sA + s * SM::A_BYTES), b0 = tc::smem_u32(sB + s * SM::B_BYTES);
#pragma unroll
            for (int k = 0; k < kBK / 16; ++k)
                tc::mma_bf16(tmem, tc::sdesc_k_sw128(a0 + 32u * k), tc::sdesc_k_sw128(b0 + 32u * k), idesc,
                             kc > 0 || k > 0);
            tc::mma_commit(empty + s);
        }
        tc::mma_commit(done);
    }
    __syncwarp();
    const bool ok = tc::mbar_wait(done, 0, kWaitLimitNs);
    if (!ok) s_fail = 3;
    tc::fence_after_sync();

    // epilogue: warp w owns accumulator rows 32w .. 32w+31 (its TMEM lanes)
    const int row = m0 + warp * 32 + lane;
    const bool write = ok && row < epi.M_valid;
#pragma unroll 1
    for (int c = 0; c < BN; c += 32) {
        float v[32];
        tc::tmem_ld_32cols(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c, v);
        if (write) gemm_store_32(epi, row, n0 + c, v, s_bias + c);
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, SM::TCOLS);
    if (threadIdx.x == 0 && s_fail) atomicExch(epi.err, s_fail);
}

// Persistent form, for GEMMs of many row tiles (the scoring forward): at
// most one CTA per SM walks the tiles t = blockIdx.x, blockIdx.x + gridDim.x,
// ... (row tile t / Ntiles, column tile t % Ntiles, so that neighbouring
// CTAs share A rows in L2).  Warp 0 (one lane) streams A and B through the
// shared-memory ring; warp 1 allocates two BN-column accumulators in tensor
// memory and (one lane) issues the MMAs of tile i into accumulator i & 1;
// warps 2-5 read tile i's accumulator back (warp w owns TMEM lanes
// 32 (w mod 4) ..) and store it while the MMAs of tile i + 1 fill the other.
// Every wait is bounded; a timed-out wait records an error code and ends the
// role's loop, and the other roles' waits then time out in turn.
constexpr int kPersistThreads = 192;

template <int BN>
struct GemmPSmem {
    static constexpr uint32_t A_BYTES = kBM * kBK * 2;
    static constexpr uint32_t B_BYTES = BN * kBK * 2;
    static constexpr uint32_t TCOLS = 2 * BN;   // BN 128 or 256
    static constexpr size_t BYTES = 1024 + kGemmStages * (A_BYTES + B_BYTES);
};

template <int BN>
__global__ void __launch_bounds__(kPersistThreads, 1)
    k_gemm_bf16_persistent(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int K,
                           int Mtiles, int Ntiles, GemmEpi epi)
{
    static_assert(BN == 128 || BN == 256, "two accumulators must fit the 512 TMEM columns");
    using SM = GemmPSmem<BN>;
    extern __shared__ uint8_t smem_dyn[];
    __shared__ int s_fail;
    __shared__ uint32_t s_tmem;
    __shared__ float s_bias[1024];
    __shared__ float s_w3[BN];
    // each epilogue warp's 32 x 32 BF16 output chunk, rows padded to 80 bytes
    // (conflict-free 16-byte writes by row and reads by 16-byte column)
    __shared__ __align__(16) uint32_t s_stage[4][32 * 20];
    __shared__ __align__(8) uint64_t bars[2 * kGemmStages + 4];
    uint8_t *base = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_dyn) + 1023) & ~uintptr_t(1023));
    uint8_t *sA = base;
    uint8_t *sB = base + kGemmStages * SM::A_BYTES;
    uint64_t *full = bars, *empty = bars + kGemmStages;
    uint64_t *acc_full = bars + 2 * kGemmStages, *acc_empty = acc_full + 2;

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int KC = K / kBK, tiles = Mtiles * Ntiles;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kGemmStages; ++s) {
            tc::mbar_init(full + s, 1);
            tc::mbar_init(empty + s, 1);
        }
        for (int a = 0; a < 2; ++a) {
            tc::mbar_init(acc_full + a, 1);    // the MMA thread's commit
            tc::mbar_init(acc_empty + a, 4);   // one arrival per epilogue warp
        }
        tc::mbar_fence_init();
        s_fail = 0;
    }
    if (warp == 1) tc::tmem_alloc(&s_tmem, SM::TCOLS);
    if (epi.mode >= 1)
        for (int c = threadIdx.x; c < Ntiles * BN; c += blockDim.x) s_bias[c] = epi.bias[c];
    if (epi.mode == 2)
        for (int c = threadIdx.x; c < BN; c += blockDim.x) s_w3[c] = epi.w3[c];
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;

    if (warp == 0) {
        if (lane == 0) {
            // TMA producer: k-step g of this CTA uses ring stage g mod stages
            uint32_t g = 0;
            for (int t = blockIdx.x; t < tiles; t += gridDim.x) {
                const int m0 = (t / Ntiles) * kBM, n0 = (t % Ntiles) * BN;
                bool ok = true;
                for (int kc = 0; kc < KC; ++kc, ++g) {
                    const uint32_t s = g % kGemmStages;
                    if (g >= (uint32_t)kGemmStages &&
                        !tc::mbar_wait(empty + s, ((g / kGemmStages) - 1) & 1, kWaitLimitNs)) {
                        s_fail = 1;
                        ok = false;
                        break;
                    }
                    tc::mbar_expect_tx(full + s, SM::A_BYTES + SM::B_BYTES);
                    tc::tma_load_2d(sA + s * SM::A_BYTES, &tmA, kc * kBK, m0, full + s);
                    tc::tma_load_2d(sB + s * SM::B_BYTES, &tmB, kc * kBK, n0, full + s);
                }
                if (!ok) break;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            // MMA issuer: tile i of this CTA accumulates into columns (i & 1) BN
            const uint32_t idesc = tc::idesc_bf16_f32(kBM, BN);
            uint32_t g = 0;
            int i = 0;
            for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++i) {
                const uint32_t a = (uint32_t)i & 1u;
                if (i >= 2 && !tc::mbar_wait(acc_empty + a, (uint32_t)((i >> 1) - 1) & 1u, kWaitLimitNs)) {
                    s_fail = 2;
                    break;
                }
                tc::fence_after_sync();
                const uint32_t d = tmem + a * (uint32_t)BN;
                bool ok = true;
                for (int kc = 0; kc < KC; ++kc, ++g) {
                    const uint32_t s = g % kGemmStages;
                    if (!tc::mbar_wait(full + s, (g / kGemmStages) & 1, kWaitLimitNs)) {
                        s_fail = 3;
                        ok = false;
                        break;
                    }
                    tc::fence_after_sync();
                    const uint32_t a0 = tc::smem_u32(sA + s * SM::A_BYTES), b0 = tc::smem_u32(sB + s * SM::B_BYTES);
#pragma unroll
                    for (int k = 0; k < kBK / 16; ++k)
                        tc::mma_bf16(d, tc::sdesc_k_sw128(a0 + 32u * k), tc::sdesc_k_sw128(b0 + 32u * k), idesc,
                                     kc > 0 || k > 0);
                    tc::mma_commit(empty + s);
                }
                if (!ok) break;
                tc::mma_commit(acc_full + a);
            }
        }
    } else {
        // epilogue warps 2-5
        const int q = warp & 3;
        int i = 0;
        for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++i) {
            const uint32_t a = (uint32_t)i & 1u;
            const bool ok = __all_sync(0xFFFFFFFFu, tc::mbar_wait(acc_full + a, (uint32_t)(i >> 1) & 1u, kWaitLimitNs));
            if (!ok) {
                if (lane == 0) s_fail = 4;
                break;
            }
            tc::fence_after_sync();
            const int m0 = (t / Ntiles) * kBM, n0 = (t % Ntiles) * BN;
            const int row0 = m0 + q * 32, row = row0 + lane;
            const bool write = row < epi.M_valid;
            const uint32_t tacc = tmem + ((uint32_t)(q * 32) << 16) + a * (uint32_t)BN;
            uint32_t *stage = s_stage[q];
            float dot = 0.0f;   // mode 2: the output unit, columns in order
            // one 32-column chunk of this thread's row (values in u)
            auto chunk = [&](const uint32_t (&u)[32], int c) {
                if (epi.mode == 2) {
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float x = fmaxf(__uint_as_float(u[j]) + s_bias[c + j], 0.0f);
                        dot = fmaf(__bfloat162float(__float2bfloat16_rn(x)), s_w3[c + j], dot);
                    }
                } else if (epi.mode == 1) {
                    // BF16 relu(acc + bias) into the warp's staging rows, then
                    // out as 64-byte row segments, 8 rows per store
                    uint32_t packed[16];
#pragma unroll
                    for (int h = 0; h < 16; ++h) {
                        const float x0 = fmaxf(__uint_as_float(u[2 * h]) + s_bias[n0 + c + 2 * h], 0.0f);
                        const float x1 = fmaxf(__uint_as_float(u[2 * h + 1]) + s_bias[n0 + c + 2 * h + 1], 0.0f);
                        const __nv_bfloat162 b = __floats2bfloat162_rn(x0, x1);
                        packed[h] = *reinterpret_cast<const uint32_t *>(&b);
                    }
                    uint4 *srow = reinterpret_cast<uint4 *>(stage + lane * 20);
#pragma unroll
                    for (int h = 0; h < 4; ++h)
                        srow[h] = make_uint4(packed[4 * h], packed[4 * h + 1], packed[4 * h + 2], packed[4 * h + 3]);
                    __syncwarp();
#pragma unroll
                    for (int it = 0; it < 4; ++it) {
                        const int r = 8 * it + (lane >> 2), h = lane & 3;
                        const uint4 val = *reinterpret_cast<const uint4 *>(stage + r * 20 + 4 * h);
                        if (row0 + r < epi.M_valid)
                            *reinterpret_cast<uint4 *>(epi.Db + (size_t)(row0 + r) * epi.ldd + n0 + c + 8 * h) = val;
                    }
                    __syncwarp();   // the staging rows are rewritten by the next chunk
                } else if (write) {
                    float v[32];
#pragma unroll
                    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(u[j]);
                    gemm_store_32(epi, row, n0 + c, v, s_bias + n0 + c);
                }
            };
#pragma unroll 1
            for (int c = 0; c < BN; c += 64) {
                uint32_t u0[32], u1[32];
                tc::tmem_ld_32cols_async(tacc + (uint32_t)c, u0);
                tc::tmem_ld_32cols_async(tacc + (uint32_t)c + 32u, u1);
                tc::tmem_wait_ld();
                tc::reg_fence32(u0);
                tc::reg_fence32(u1);
                chunk(u0, c);
                chunk(u1, c + 32);
            }
            if (epi.mode == 2 && write) epi.y[row] = dot + epi.b3[0];
            tc::fence_before_sync();
            __syncwarp();
            if (lane == 0) tc::mbar_arrive(acc_empty + a);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 1) tc::tmem_dealloc(tmem, SM::TCOLS);
    if (threadIdx.x == 0 && s_fail) atomicExch(epi.err, s_fail);
}

// ---------------------------------------------------------------------------
// Host: tensor maps and the GEMM launcher.
// ---------------------------------------------------------------------------
typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static std::once_flag once;
    static EncodeTiledFn fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        (void)cudaGetLastError();
    });
    return fn;
}

// BF16 matrix [rows][ld] with `cols` valid columns, tiles of box_rows x 64.
static int make_map(CUtensorMap *m, const void *ptr, int rows, int cols, int ld, int box_rows)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) return set_error(FFS_ECUDA, "cuTensorMapEncodeTiled unavailable");
    if (((uintptr_t)ptr & 15u) || (ld % 8)) return set_error(FFS_EINVAL, "GEMM operand must be 16-byte aligned, ld % 8 == 0");
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(ptr), dims, strides, box, estr,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return set_error(FFS_ECUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return FFS_OK;
}

// Launch `k` as a programmatic dependent of the stream's previous kernel
// (the kernel calls grid_dep_wait before it reads that kernel's results).
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, args...);
}

template <int BN>
static int launch_gemm_bn(const CUtensorMap &ta, const CUtensorMap &tb, int Mtiles, int N, int K, const GemmEpi &epi,
                          cudaStream_t st)
{
    const size_t smem = GemmSmem<BN>::BYTES;
    FFS_CUDA_TRY(cudaFuncSetAttribute(k_gemm_bf16<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid(Mtiles, N / BN);
    if (epi.pdl) {
        FFS_CUDA_TRY(launch_pdl(k_gemm_bf16<BN>, grid, dim3(128), smem, st, ta, tb, K, epi));
        return FFS_OK;
    }
    k_gemm_bf16<BN><<<grid, 128, smem, st>>>(ta, tb, K, epi);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

template <int BN>
static int launch_gemm_persistent(const CUtensorMap &ta, const CUtensorMap &tb, int Mtiles, int N, int K,
                                  const GemmEpi &epi, int ctas, cudaStream_t st)
{
    const size_t smem = GemmPSmem<BN>::BYTES;
    FFS_CUDA_TRY(cudaFuncSetAttribute(k_gemm_bf16_persistent<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      (int)smem));
    k_gemm_bf16_persistent<BN><<<ctas, kPersistThreads, smem, st>>>(ta, tb, K, Mtiles, N / BN, epi);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

static int device_sms()
{
    static int num_sms = 0;
    if (!num_sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (num_sms <= 0) num_sms = 1;
    }
    return num_sms;
}

// The persistent form with one column tile: the output layer can be fused
// into the last hidden layer's epilogue.
static bool gemm_fused_output_ok(int M, int N)
{
    return (M + kBM - 1) / kBM >= device_sms() && (N == 128 || N == 256);
}

// D = A[M][K] * B[N][K]^T.  A rows beyond M read as zero (TMA fill); K is
// rounded up to 64 with zero columns beyond Kvalid; N a multiple of 64.
// At least one row tile per SM (and N a multiple of 128, at most 1024): the
// persistent form with two accumulators; otherwise one CTA per tile.
int gemm_bf16(const void *A, int lda, const void *B, int ldb, int M, int N, int Kvalid, GemmEpi epi, cudaStream_t st)
{
    if (M < 1 || N < 64 || N % 64 || Kvalid < 1) return set_error(FFS_EINVAL, "GEMM shape M=%d N=%d K=%d", M, N, Kvalid);
    const int K = round_up(Kvalid, kBK);
    int BN = (N % 256 == 0) ? 256 : (N % 192 == 0) ? 192 : (N % 128 == 0) ? 128 : 64;
    // few row tiles (the training batches): narrower column tiles, so that
    // more CTAs share the (latency-bound) work; wide tiles once the grid
    // covers the SMs
    const int Mt = (M + kBM - 1) / kBM;
    const int num_sms = device_sms();
    if (epi.mode == 2 && !gemm_fused_output_ok(M, N))
        return set_error(FFS_EINVAL, "fused output layer: M=%d N=%d", M, N);
    if (Mt >= num_sms && N % 128 == 0 && N <= 1024) {
        const int pbn = N % 256 == 0 ? 256 : 128;
        const int tiles = Mt * (N / pbn);
        int ctas = std::min(tiles, num_sms);
        if (epi.max_ctas > 0) ctas = std::min(ctas, epi.max_ctas);
        CUtensorMap ta, tb;
        int rc = make_map(&ta, A, M, Kvalid, lda, kBM);
        if (rc) return rc;
        if ((rc = make_map(&tb, B, N, Kvalid, ldb, pbn))) return rc;
        epi.M_valid = M;
        return pbn == 256 ? launch_gemm_persistent<256>(ta, tb, Mt, N, K, epi, ctas, st)
                          : launch_gemm_persistent<128>(ta, tb, Mt, N, K, epi, ctas, st);
    }
    while (BN > 64 && (int64_t)Mt * (N / BN) < num_sms) {
        const int nb = BN == 256 ? 128 : BN == 192 ? 64 : 64;
        if (N % nb) break;
        BN = nb;
    }
    CUtensorMap ta, tb;
    int rc = make_map(&ta, A, M, Kvalid, lda, kBM);
    if (rc) return rc;
    if ((rc = make_map(&tb, B, N, Kvalid, ldb, BN))) return rc;
    epi.M_valid = M;
    const int Mtiles = (M + kBM - 1) / kBM;
    switch (BN) {
    case 256: return launch_gemm_bn<256>(ta, tb, Mtiles, N, K, epi, st);
    case 192: return launch_gemm_bn<192>(ta, tb, Mtiles, N, K, epi, st);
    case 128: return launch_gemm_bn<128>(ta, tb, Mtiles, N, K, epi, st);
    default: return launch_gemm_bn<64>(ta, tb, Mtiles, N, K, epi, st);
    }
}

// ---------------------------------------------------------------------------
// CUDA-core kernels of the MLP (elementwise, reductions, transposes, Adam).
// ---------------------------------------------------------------------------
__global__ void k_f32_to_bf16_padded(const float *src, int rows, int cols, int ld_src, __nv_bfloat16 *dst, int ld_dst)
{
    const int r = blockIdx.y;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ld_dst; c += gridDim.x * blockDim.x)
        dst[(size_t)r * ld_dst + c] = __float2bfloat16_rn(c < cols ? src[(size_t)r * ld_src + c] : 0.0f);
}

// dst[c][r] = src[r][c] for a BF16 [rows][cols] matrix (32 x 32 tiles).
__global__ void k_transpose_bf16(const __nv_bfloat16 *src, int rows, int cols, int lds, __nv_bfloat16 *dst, int ldd)
{
    __shared__ __nv_bfloat16 tile[32][33];
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        tile[i][threadIdx.x] = (r < rows && c < cols) ? src[(size_t)r * lds + c] : __float2bfloat16_rn(0.0f);
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (c < cols && r < rows) dst[(size_t)c * ldd + r] = tile[threadIdx.x][i];
    }
}

// Layer 1's bias for inputs whose columns [P, P + nfeat) hold the same
// vector `feat` in every row (warp per output unit o): out[o] = b1[o] +
// sum_i W1b[o][P + i] BF16(feat[i]), the products as the tensor cores would
// form them (BF16 operands, FP32 sums; per-lane partials, then a fixed
// shuffle tree).
__global__ void k_fold_bias(const __nv_bfloat16 *W1b, int K1, const float *b1, int P, const float *feat, int nfeat,
                            int h1, float *out)
{
    const int o = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (o >= h1) return;
    float acc = 0.0f;
    for (int i = lane; i < nfeat; i += 32)
        acc = fmaf(__bfloat162float(W1b[(size_t)o * K1 + P + i]), __bfloat162float(__float2bfloat16_rn(feat[i])), acc);
    for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, d);
    if (lane == 0) out[o] = b1[o] + acc;
}

// y[b] = H2[b] . w3 + b3 (warp per row)
__global__ void k_out_layer(const __nv_bfloat16 *H2, int B, int h2, const float *w3, const float *b3, float *y)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= B) return;
    float acc = 0.0f;
    for (int j = lane; j < h2; j += 32) acc += __bfloat162float(H2[(size_t)warp * h2 + j]) * w3[j];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    if (lane == 0) y[warp] = acc + b3[0];
}

// Warp per row b of a training batch: y = H2[b] . w3 + b3, e = y - t[b],
// dy[b] = 2 e / B (the MSE's derivative), loss += e^2 / B, and the output
// layer's backpropagated signal dZ2[b][j] = dy[b] w3[j] [H2[b][j] > 0] as BF16,
// row-major and transposed (dZ2T[j][b]).  Same arithmetic, in the same order,
// as k_out_layer, k_loss and k_dz2 one after another.
__global__ void k_out_loss_dz2(const __nv_bfloat16 *H2, int B, int h2, const float *w3, const float *b3,
                               const float *t, float *dy, float *loss, __nv_bfloat16 *dZ2, __nv_bfloat16 *dZ2T)
{
    tc::grid_dep_launch();
    tc::grid_dep_wait();
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (b >= B) return;
    float acc = 0.0f;
    for (int j = lane; j < h2; j += 32) acc += __bfloat162float(H2[(size_t)b * h2 + j]) * w3[j];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
    const float e = (acc + b3[0]) - t[b];
    const float d = 2.0f * e / (float)B;
    if (lane == 0) {
        dy[b] = d;
        if (loss) atomicAdd(loss, e * e / (float)B);
    }
    for (int j = lane; j < h2; j += 32) {
        const float g = __bfloat162float(H2[(size_t)b * h2 + j]) > 0.0f ? d * w3[j] : 0.0f;
        const __nv_bfloat16 gb = __float2bfloat16_rn(g);
        dZ2[(size_t)b * h2 + j] = gb;
        dZ2T[(size_t)j * B + b] = gb;
    }
}

// out[j] = sum_b X[b][j] (* w[b] if w): column sums of a [B][C] matrix.
// Block (32, 32): threadIdx.x picks the column of a 32-column tile,
// threadIdx.y the rows b = y, y + 32, ...; the 32 partial sums of a column
// are then added in a fixed order, so the result does not depend on timing.
template <typename T>
__global__ void k_colsum(const T *X, const float *w, int B, int C, float *out)
{
    __shared__ float part[32][33];
    const int j = blockIdx.x * 32 + threadIdx.x;
    float acc = 0.0f;
    if (j < C) {
#pragma unroll 4
        for (int b = threadIdx.y; b < B; b += 32) {
            float x;
            if constexpr (sizeof(T) == 2) x = __bfloat162float(X[(size_t)b * C + j]);
            else x = (float)X[(size_t)b * C + j];
            acc += w ? x * w[b] : x;
        }
    }
    part[threadIdx.y][threadIdx.x] = acc;
    __syncthreads();
    if (threadIdx.y == 0 && j < C) {
        float s = 0.0f;
        for (int y = 0; y < 32; ++y) s += part[y][threadIdx.x];
        out[j] = s;
    }
}

// The output layer's parameter gradients in one launch: gw3[j] = sum_b
// H2[b][j] dy[b], gb2[j] = sum_b dZ2[b][j] (as k_colsum), and block 0 also
// gb3 = sum_b dy[b] (threads b, b + 1024, ..., then a fixed-order sum).
__global__ void k_out_grads(const __nv_bfloat16 *H2, const __nv_bfloat16 *dZ2, const float *dy, int B, int h2,
                            float *gw3, float *gb2, float *gb3)
{
    __shared__ float part[2][32][33];
    const int j = blockIdx.x * 32 + threadIdx.x;
    float a = 0.0f, c = 0.0f;
    if (j < h2) {
#pragma unroll 4
        for (int b = threadIdx.y; b < B; b += 32) {
            a += __bfloat162float(H2[(size_t)b * h2 + j]) * dy[b];
            c += __bfloat162float(dZ2[(size_t)b * h2 + j]);
        }
    }
    part[0][threadIdx.y][threadIdx.x] = a;
    part[1][threadIdx.y][threadIdx.x] = c;
    __syncthreads();
    if (threadIdx.y == 0 && j < h2) {
        float sa = 0.0f, sc = 0.0f;
        for (int y = 0; y < 32; ++y) {
            sa += part[0][y][threadIdx.x];
            sc += part[1][y][threadIdx.x];
        }
        gw3[j] = sa;
        gb2[j] = sc;
    }
    if (blockIdx.x == 0) {
        __syncthreads();
        const int tid = threadIdx.y * 32 + threadIdx.x;
        float sd = 0.0f;
        for (int b = tid; b < B; b += 1024) sd += dy[b];
        part[0][threadIdx.y][threadIdx.x] = sd;
        __syncthreads();
        if (tid == 0) {
            float t = 0.0f;
            for (int y = 0; y < 32; ++y)
                for (int x = 0; x < 32; ++x) t += part[0][y][x];
            gb3[0] = t;
        }
    }
}

// He-uniform initialisation (He et al. 2015, uniform form: limit
// sqrt(6 / fan_in)) of a [rows][ld] FP32 matrix with `cols` valid columns
// (the rest set to 0).  Element (o, i) takes word i mod 4 of the Philox block
// i / 4 of the stream (seed, kPurposeMlpInit, layer, generation 0, cell o):
// u = ((x >> 8) - 2^23) / 2^23, exactly representable in [-1, 1), and the
// value is lim * u (then * scale), each product rounded once to FP32.
__global__ void k_mlp_init(float *W, int rows, int cols, int ld, uint64_t seed, uint32_t layer, int fan_in,
                           float scale)
{
    const float lim = __fsqrt_rn(__fdiv_rn(6.0f, (float)fan_in));
    const int64_t total = (int64_t)rows * ld;
    for (int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; idx < total;
         idx += (int64_t)gridDim.x * blockDim.x) {
        const int o = (int)(idx / ld), i = (int)(idx - (int64_t)o * ld);
        float v = 0.0f;
        if (i < cols) {
            const U4 b = draw_block(seed, kPurposeMlpInit, layer, 0u, (uint32_t)o, (uint32_t)(i >> 2));
            const uint32_t x = (i & 3) == 0 ? b.x : (i & 3) == 1 ? b.y : (i & 3) == 2 ? b.z : b.w;
            const float u = (float)((int32_t)(x >> 8) - (1 << 23)) * (1.0f / 8388608.0f);
            v = __fmul_rn(lim, u);
            if (scale != 1.0f) v = __fmul_rn(v, scale);
        }
        W[idx] = v;
    }
}

// Adam (Kingma & Ba 2015) over the concatenated parameters.  The step count
// lives on the device (t_prev = steps taken so far), so a training step can
// be replayed from a CUDA graph; this step is t = t_prev + 1, with the bias
// corrections 1 - b1^t and 1 - b2^t; the last block to finish (counted in
// blocks_done, reset by it) advances the count, after every block has read it.
// It also writes the BF16 copies the GEMMs read: W1b[i] for the W1 block
// [0, nW1) and W2b[o][c] for the W2 block [w2_off, w2_off + h2 h1); the next
// training step transposes W2b into W2Tb on a side stream.
__device__ __forceinline__ float adam_one(float &p, float gi, float &m, float &v, float lr, float b1, float b2,
                                          float eps, float c1, float c2)
{
    const float mi = b1 * m + (1.0f - b1) * gi;
    const float vi = b2 * v + (1.0f - b2) * gi * gi;
    m = mi;
    v = vi;
    p = p - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    return p;
}

__global__ void k_adam_bf16(float *p, const float *g, float *m, float *v, int n, float lr, float b1, float b2,
                            float eps, long long *t_prev, unsigned int *blocks_done, int nW1, int w2_off, int h1,
                            int h2, __nv_bfloat16 *W1b, __nv_bfloat16 *W2b)
{
    tc::grid_dep_launch();
    tc::grid_dep_wait();
    const float t = (float)(*t_prev + 1);
    const float c1 = 1.0f - powf(b1, t), c2 = 1.0f - powf(b2, t);
    const int nW2 = h1 * h2;
    // four parameters per step (the blocks W1, b1, W2, ... start at multiples
    // of four), then the tail one by one
    const int nq = n >> 2;
    for (int iq = blockIdx.x * blockDim.x + threadIdx.x; iq < nq; iq += gridDim.x * blockDim.x) {
        const int i = 4 * iq;
        float4 P = reinterpret_cast<float4 *>(p)[iq];
        const float4 G = reinterpret_cast<const float4 *>(g)[iq];
        float4 Mv = reinterpret_cast<float4 *>(m)[iq];
        float4 V = reinterpret_cast<float4 *>(v)[iq];
        adam_one(P.x, G.x, Mv.x, V.x, lr, b1, b2, eps, c1, c2);
        adam_one(P.y, G.y, Mv.y, V.y, lr, b1, b2, eps, c1, c2);
        adam_one(P.z, G.z, Mv.z, V.z, lr, b1, b2, eps, c1, c2);
        adam_one(P.w, G.w, Mv.w, V.w, lr, b1, b2, eps, c1, c2);
        reinterpret_cast<float4 *>(p)[iq] = P;
        reinterpret_cast<float4 *>(m)[iq] = Mv;
        reinterpret_cast<float4 *>(v)[iq] = V;
        if (i < nW1) {
            const __nv_bfloat162 lo = __floats2bfloat162_rn(P.x, P.y), hi = __floats2bfloat162_rn(P.z, P.w);
            uint2 pk;
            pk.x = *reinterpret_cast<const uint32_t *>(&lo);
            pk.y = *reinterpret_cast<const uint32_t *>(&hi);
            *reinterpret_cast<uint2 *>(W1b + i) = pk;
        } else if (i >= w2_off && i < w2_off + nW2) {
            const int r = i - w2_off;
            const __nv_bfloat162 lo = __floats2bfloat162_rn(P.x, P.y), hi = __floats2bfloat162_rn(P.z, P.w);
            uint2 pk;
            pk.x = *reinterpret_cast<const uint32_t *>(&lo);
            pk.y = *reinterpret_cast<const uint32_t *>(&hi);
            *reinterpret_cast<uint2 *>(W2b + r) = pk;
        }
    }
    for (int i = 4 * nq + blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        // the tail lies past W1 and W2 (b2, w3, b3)
        adam_one(p[i], g[i], m[i], v[i], lr, b1, b2, eps, c1, c2);
    }
    __syncthreads();   // this block's threads have read the count
    if (threadIdx.x == 0) {
        __threadfence();
        if (atomicAdd(blocks_done, 1u) == gridDim.x - 1) {
            *t_prev += 1;
            *blocks_done = 0u;
        }
    }
}

}  // namespace fgpu

using namespace fgpu;

struct ffs_mlp {
    int in_dim = 0, K1 = 0, h1 = 0, h2 = 0, max_batch = 0;
    long long *d_adam_t = nullptr;   // Adam steps taken (device, so training steps can be graph-replayed)
    unsigned int *d_adam_done = nullptr;   // blocks of the running Adam launch that have finished
    // parameters (FP32 masters): W1 [h1][K1] (columns >= in_dim stay 0), b1, W2 [h2][h1], b2, w3 [h2], b3 [1]
    float *W1 = nullptr, *b1 = nullptr, *W2 = nullptr, *b2 = nullptr, *w3 = nullptr, *b3 = nullptr;
    float *gW1 = nullptr, *gb1 = nullptr, *gW2 = nullptr, *gb2 = nullptr, *gw3 = nullptr, *gb3 = nullptr;
    float *m = nullptr, *v = nullptr;      // Adam moments over the concatenated parameters
    float *params = nullptr, *grads = nullptr;
    size_t n_params = 0;
    __nv_bfloat16 *W1b = nullptr, *W2b = nullptr, *W2Tb = nullptr;
    // activations / scratch for max_batch rows
    __nv_bfloat16 *H1 = nullptr, *H2 = nullptr, *H1T = nullptr, *XT = nullptr, *dZ2 = nullptr, *dZ2T = nullptr,
                  *dZ1T = nullptr;
    float *y = nullptr, *dy = nullptr, *dZ1 = nullptr;
    int *err = nullptr;
    // the scoring copy (allocated on demand): what a forward pass reads (BF16
    // W1 and W2, FP32 b1, b2, w3, b3 at the parameters' offsets) and its own
    // hidden activations, so that training steps may update the network
    // while a forward pass scores with the weights of the last copy
    __nv_bfloat16 *cW1b = nullptr, *cW2b = nullptr, *cH1 = nullptr, *cH2 = nullptr;
    float *cparams = nullptr;
    float *fold = nullptr;   // [h1]: layer 1's bias with a constant input block folded in
    // a training step's side branches (forked from and joined back into the
    // caller's stream, so that a captured step keeps them in its graph)
    cudaStream_t aux[2] = {nullptr, nullptr};
    cudaEvent_t ev[8] = {};
    std::vector<void *> allocs;
};

namespace fgpu {

int mlp_in_dim(const ffs_mlp *m) { return m->in_dim; }
int mlp_max_batch(const ffs_mlp *m) { return m->max_batch; }

static void mlp_free(ffs_mlp *M)
{
    if (!M) return;
    for (void *p : M->allocs) cudaFree(p);
    for (cudaStream_t s : M->aux)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t e : M->ev)
        if (e) cudaEventDestroy(e);
    delete M;
}

static int refresh_bf16(ffs_mlp *M, cudaStream_t st)
{
    k_f32_to_bf16_padded<<<dim3(4, M->h1), 128, 0, st>>>(M->W1, M->h1, M->K1, M->K1, M->W1b, M->K1);
    k_f32_to_bf16_padded<<<dim3(4, M->h2), 128, 0, st>>>(M->W2, M->h2, M->h1, M->h1, M->W2b, M->h1);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

// What a forward pass reads and writes: the network's own weights and
// activations (training) or the scoring copy.
struct MlpFwd {
    const __nv_bfloat16 *W1b, *W2b;
    const float *b1, *b2, *w3, *b3;
    __nv_bfloat16 *H1, *H2;
};

static MlpFwd fwd_live(const ffs_mlp *M) { return {M->W1b, M->W2b, M->b1, M->b2, M->w3, M->b3, M->H1, M->H2}; }

static MlpFwd fwd_copy(const ffs_mlp *M)
{
    const float *c = M->cparams;
    return {M->cW1b, M->cW2b, c + (M->b1 - M->params), c + (M->b2 - M->params), c + (M->w3 - M->params),
            c + (M->b3 - M->params), M->cH1, M->cH2};
}

// The two hidden layers: H1 = relu(x W1^T + b1), H2 = relu(H1 W2^T + b2), BF16.
static int mlp_hidden(ffs_mlp *M, const MlpFwd &w, const void *x, int ldx, int B, cudaStream_t st, int max_ctas = 0)
{
    GemmEpi e;
    memset(&e, 0, sizeof(e));
    e.err = M->err;
    e.max_ctas = max_ctas;
    e.mode = 1;
    e.Db = w.H1;
    e.bias = w.b1;
    e.ldd = M->h1;
    int rc = gemm_bf16(x, ldx, w.W1b, M->K1, B, M->h1, M->in_dim, e, st);
    if (rc) return rc;
    e.Db = w.H2;
    e.bias = w.b2;
    e.ldd = M->h2;
    return gemm_bf16(w.H1, M->h1, w.W2b, M->h1, B, M->h2, M->h1, e, st);
}

static int mlp_forward(ffs_mlp *M, const MlpFwd &w, const void *x, int ldx, int B, float *y, cudaStream_t st,
                       int max_ctas = 0)
{
    if (gemm_fused_output_ok(B, M->h2)) {
        // large batches: the output unit in layer 2's epilogue (H2 never stored)
        GemmEpi e;
        memset(&e, 0, sizeof(e));
        e.err = M->err;
        e.max_ctas = max_ctas;
        e.mode = 1;
        e.Db = w.H1;
        e.bias = w.b1;
        e.ldd = M->h1;
        int rc = gemm_bf16(x, ldx, w.W1b, M->K1, B, M->h1, M->in_dim, e, st);
        if (rc) return rc;
        e.mode = 2;
        e.Db = nullptr;
        e.bias = w.b2;
        e.w3 = w.w3;
        e.b3 = w.b3;
        e.y = y;
        return gemm_bf16(w.H1, M->h1, w.W2b, M->h1, B, M->h2, M->h1, e, st);
    }
    int rc = mlp_hidden(M, w, x, ldx, B, st, max_ctas);
    if (rc) return rc;
    k_out_layer<<<(B * 32 + 255) / 256, 256, 0, st>>>(w.H2, B, M->h2, w.w3, w.b3, y);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

// Up to four word copies in one launch (the scoring copy's segments).
struct CopySegs {
    uint32_t *dst[4];
    const uint32_t *src[4];
    int64_t words[4];
};

__global__ void k_copy_words(CopySegs c)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int k = 0; k < 4; ++k)
        for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < c.words[k]; i += stride)
            c.dst[k][i] = c.src[k][i];
}

int mlp_enable_copy(ffs_mlp *M)
{
    if (M->cparams) return FFS_OK;
    const size_t nW1 = (size_t)M->h1 * M->K1, nW2 = (size_t)M->h2 * M->h1, Bm = (size_t)M->max_batch;
    void *p[5] = {};
    const size_t bytes[5] = {nW1 * 2, nW2 * 2, Bm * M->h1 * 2, Bm * M->h2 * 2, M->n_params * 4};
    for (int k = 0; k < 5; ++k)
        if (cudaMalloc(&p[k], bytes[k]) != cudaSuccess) {
            (void)cudaGetLastError();
            for (int j = 0; j < k; ++j) cudaFree(p[j]);
            return set_error(FFS_ENOMEM, "MLP scoring copy");
        }
    for (int k = 0; k < 5; ++k) M->allocs.push_back(p[k]);
    M->cW1b = (__nv_bfloat16 *)p[0];
    M->cW2b = (__nv_bfloat16 *)p[1];
    M->cH1 = (__nv_bfloat16 *)p[2];
    M->cH2 = (__nv_bfloat16 *)p[3];
    M->cparams = (float *)p[4];
    return FFS_OK;
}

// The scoring copy := the weights a forward pass reads, as they are now (in
// stream order).
int mlp_take_copy(ffs_mlp *M, cudaStream_t st)
{
    if (!M->cparams) return set_error(FFS_EINVAL, "the network has no scoring copy");
    const size_t nW1 = (size_t)M->h1 * M->K1, nW2 = (size_t)M->h2 * M->h1;
    const int64_t ob1 = M->b1 - M->params, ob2 = M->b2 - M->params;
    CopySegs c;
    c.dst[0] = reinterpret_cast<uint32_t *>(M->cW1b);
    c.src[0] = reinterpret_cast<const uint32_t *>(M->W1b);
    c.words[0] = (int64_t)nW1 / 2;   // h1 and K1 are multiples of 64
    c.dst[1] = reinterpret_cast<uint32_t *>(M->cW2b);
    c.src[1] = reinterpret_cast<const uint32_t *>(M->W2b);
    c.words[1] = (int64_t)nW2 / 2;
    c.dst[2] = reinterpret_cast<uint32_t *>(M->cparams + ob1);
    c.src[2] = reinterpret_cast<const uint32_t *>(M->params + ob1);
    c.words[2] = M->h1;                                    // b1
    c.dst[3] = reinterpret_cast<uint32_t *>(M->cparams + ob2);
    c.src[3] = reinterpret_cast<const uint32_t *>(M->params + ob2);
    c.words[3] = (int64_t)M->n_params - ob2;                // b2, w3, b3
    k_copy_words<<<304, 256, 0, st>>>(c);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

int mlp_fold_bias(ffs_mlp *M, bool use_copy, int P, const float *feat, int nfeat, cudaStream_t st)
{
    if (use_copy && !M->cparams) return set_error(FFS_EINVAL, "the network has no scoring copy");
    if (P < 1 || nfeat < 0 || P + nfeat > M->in_dim) return set_error(FFS_EINVAL, "fold: P %d, nfeat %d", P, nfeat);
    const MlpFwd w = use_copy ? fwd_copy(M) : fwd_live(M);
    k_fold_bias<<<(M->h1 * 32 + 255) / 256, 256, 0, st>>>(w.W1b, M->K1, w.b1, P, feat, nfeat, M->h1, M->fold);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

int mlp_forward_folded(ffs_mlp *M, bool use_copy, const void *xpos, int ldxpos, int kpos, int P, const float *feat,
                       int nfeat, int B, float *y, int max_ctas, cudaStream_t st)
{
    if (use_copy && !M->cparams) return set_error(FFS_EINVAL, "the network has no scoring copy");
    if (B < 1 || B > M->max_batch) return set_error(FFS_EINVAL, "batch %d outside [1, %d]", B, M->max_batch);
    if (kpos < 1 || kpos > P || P + nfeat > M->in_dim || ldxpos < kpos || ldxpos % 8)
        return set_error(FFS_EINVAL, "folded input: kpos %d, P %d, nfeat %d, ld %d", kpos, P, nfeat, ldxpos);
    const MlpFwd w = use_copy ? fwd_copy(M) : fwd_live(M);
    MlpFwd wf = w;
    wf.b1 = M->fold;
    // layer 1 over the kpos leading columns only (TMA reads the rest of the
    // 64-column step as zeros), with the folded bias
    GemmEpi e;
    memset(&e, 0, sizeof(e));
    e.err = M->err;
    e.max_ctas = max_ctas;
    e.mode = 1;
    e.Db = wf.H1;
    e.bias = wf.b1;
    e.ldd = M->h1;
    int rc = gemm_bf16(xpos, ldxpos, wf.W1b, M->K1, B, M->h1, kpos, e, st);
    if (rc) return rc;
    if (gemm_fused_output_ok(B, M->h2)) {
        e.mode = 2;
        e.Db = nullptr;
        e.bias = wf.b2;
        e.w3 = wf.w3;
        e.b3 = wf.b3;
        e.y = y;
        return gemm_bf16(wf.H1, M->h1, wf.W2b, M->h1, B, M->h2, M->h1, e, st);
    }
    e.Db = wf.H2;
    e.bias = wf.b2;
    e.ldd = M->h2;
    if ((rc = gemm_bf16(wf.H1, M->h1, wf.W2b, M->h1, B, M->h2, M->h1, e, st))) return rc;
    k_out_layer<<<(B * 32 + 255) / 256, 256, 0, st>>>(wf.H2, B, M->h2, wf.w3, wf.b3, y);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}


// Checkpoint blob of a network: this header, then the FP32 parameters, the
// Adam first and second moments (n_params each, the internal order: W1
// [h1][K1] with its zero columns, b1, W2, b2, w3, b3).
struct MlpBlobHeader {
    uint32_t magic, version;
    int32_t in_dim, h1, h2, K1;
    int64_t adam_t, n_params;
};
constexpr uint32_t kMlpBlobMagic = 0x4D534646u, kMlpBlobVersion = 1;

int64_t mlp_state_bytes(const ffs_mlp *M) { return (int64_t)sizeof(MlpBlobHeader) + 3 * (int64_t)M->n_params * 4; }

int mlp_save(const ffs_mlp *M, void *host, cudaStream_t st)
{
    long long t = 0;
    FFS_CUDA_TRY(cudaMemcpyAsync(&t, M->d_adam_t, 8, cudaMemcpyDeviceToHost, st));
    FFS_CUDA_TRY(cudaStreamSynchronize(st));
    MlpBlobHeader h{kMlpBlobMagic, kMlpBlobVersion, M->in_dim, M->h1, M->h2, M->K1, (int64_t)t, (int64_t)M->n_params};
    memcpy(host, &h, sizeof(h));
    float *p = reinterpret_cast<float *>(static_cast<char *>(host) + sizeof(h));
    FFS_CUDA_TRY(cudaMemcpyAsync(p, M->params, M->n_params * 4, cudaMemcpyDefault, st));
    FFS_CUDA_TRY(cudaMemcpyAsync(p + M->n_params, M->m, M->n_params * 4, cudaMemcpyDefault, st));
    FFS_CUDA_TRY(cudaMemcpyAsync(p + 2 * M->n_params, M->v, M->n_params * 4, cudaMemcpyDefault, st));
    FFS_CUDA_TRY(cudaStreamSynchronize(st));
    return FFS_OK;
}

int mlp_check_state(const ffs_mlp *M, const void *host, int64_t size)
{
    if (size < (int64_t)sizeof(MlpBlobHeader)) return set_error(FFS_EINVAL, "network state: %lld bytes", (long long)size);
    MlpBlobHeader h;
    memcpy(&h, host, sizeof(h));
    if (h.magic != kMlpBlobMagic || h.version != kMlpBlobVersion)
        return set_error(FFS_EINVAL, "network state: bad magic or version");
    if (h.in_dim != M->in_dim || h.h1 != M->h1 || h.h2 != M->h2 || h.K1 != M->K1 || h.n_params != (int64_t)M->n_params)
        return set_error(FFS_EINVAL, "network state of a %d-%d-%d network, this one is %d-%d-%d", h.in_dim, h.h1, h.h2,
                         M->in_dim, M->h1, M->h2);
    if (size < mlp_state_bytes(M)) return set_error(FFS_EINVAL, "network state truncated");
    if (h.adam_t < 0) return set_error(FFS_EINVAL, "network state: step count %lld", (long long)h.adam_t);
    return FFS_OK;
}

int mlp_load(ffs_mlp *M, const void *host, int64_t size, cudaStream_t st)
{
    if (int rc = mlp_check_state(M, host, size)) return rc;
    MlpBlobHeader h;
    memcpy(&h, host, sizeof(h));
    const float *p = reinterpret_cast<const float *>(static_cast<const char *>(host) + sizeof(h));
    FFS_CUDA_TRY(cudaMemcpyAsync(M->params, p, M->n_params * 4, cudaMemcpyDefault, st));
    FFS_CUDA_TRY(cudaMemcpyAsync(M->m, p + M->n_params, M->n_params * 4, cudaMemcpyDefault, st));
    FFS_CUDA_TRY(cudaMemcpyAsync(M->v, p + 2 * M->n_params, M->n_params * 4, cudaMemcpyDefault, st));
    const long long t = h.adam_t;
    FFS_CUDA_TRY(cudaMemcpyAsync(M->d_adam_t, &t, 8, cudaMemcpyHostToDevice, st));
    int rc = refresh_bf16(M, st);
    if (rc) return rc;
    FFS_CUDA_TRY(cudaStreamSynchronize(st));
    return FFS_OK;
}

}  // namespace fgpu

extern "C" {

int ffs_gemm_bf16(const uint16_t *A, int32_t lda, const uint16_t *B, int32_t ldb, float *D, int32_t ldd, int32_t M,
                  int32_t N, int32_t K, int32_t *err, ffs_stream stream)
{
    clear_error();
    if (!A || !B || !D || !err) return set_error(FFS_EINVAL, "NULL argument");
    if (ldd % 4 || ((uintptr_t)D & 15u)) return set_error(FFS_EINVAL, "D must be 16-byte aligned with ldd % 4 == 0");
    if (lda < K || ldb < K || ldd < N) return set_error(FFS_EINVAL, "leading dimensions too small");
    GemmEpi e;
    memset(&e, 0, sizeof(e));
    e.D = D;
    e.ldd = ldd;
    e.mode = 0;
    e.err = err;
    return gemm_bf16(A, lda, B, ldb, M, N, K, e, (cudaStream_t)stream);
}

int ffs_mlp_create(int32_t in_dim, int32_t h1, int32_t h2, int32_t max_batch, ffs_mlp **out)
{
    clear_error();
    if (!out) return set_error(FFS_EINVAL, "NULL argument");
    *out = nullptr;
    if (in_dim < 1 || in_dim > 4096) return set_error(FFS_EINVAL, "in_dim %d", in_dim);
    if (h1 < 64 || h1 % 64 || h1 > 1024 || h2 < 64 || h2 % 64 || h2 > 1024)
        return set_error(FFS_EINVAL, "hidden sizes must be multiples of 64 in [64, 1024]");
    if (max_batch < 128 || max_batch % 128) return set_error(FFS_EINVAL, "max_batch %d must be a multiple of 128", max_batch);
    ffs_mlp *M = new ffs_mlp();
    M->in_dim = in_dim;
    M->K1 = round_up(in_dim, 64);
    M->h1 = h1;
    M->h2 = h2;
    M->max_batch = max_batch;
    bool failed = false;   // an allocation failed (nothing is kept for it)
    auto alloc = [&](size_t bytes) -> void * {
        void *p = nullptr;
        if (injected_alloc_failure() || cudaMalloc(&p, bytes) != cudaSuccess) {
            (void)cudaGetLastError();
            failed = true;
            return nullptr;
        }
        M->allocs.push_back(p);
        return p;
    };
    const size_t nW1 = (size_t)h1 * M->K1, nW2 = (size_t)h2 * h1;
    M->n_params = nW1 + h1 + nW2 + h2 + h2 + 1;
    M->params = (float *)alloc(M->n_params * 4);
    M->grads = (float *)alloc(M->n_params * 4);
    M->m = (float *)alloc(M->n_params * 4);
    M->v = (float *)alloc(M->n_params * 4);
    const size_t Bm = (size_t)max_batch;
    M->W1b = (__nv_bfloat16 *)alloc(nW1 * 2);
    M->W2b = (__nv_bfloat16 *)alloc(nW2 * 2);
    M->W2Tb = (__nv_bfloat16 *)alloc(nW2 * 2);
    M->H1 = (__nv_bfloat16 *)alloc(Bm * h1 * 2);
    M->H2 = (__nv_bfloat16 *)alloc(Bm * h2 * 2);
    M->H1T = (__nv_bfloat16 *)alloc(Bm * h1 * 2);
    M->XT = (__nv_bfloat16 *)alloc(Bm * M->K1 * 2);
    M->dZ2 = (__nv_bfloat16 *)alloc(Bm * h2 * 2);
    M->dZ2T = (__nv_bfloat16 *)alloc(Bm * h2 * 2);
    M->dZ1T = (__nv_bfloat16 *)alloc(Bm * h1 * 2);
    M->y = (float *)alloc(Bm * 4);
    M->dy = (float *)alloc(Bm * 4);
    M->dZ1 = (float *)alloc(Bm * h1 * 4);
    M->err = (int *)alloc(4);
    M->d_adam_t = (long long *)alloc(8);
    M->d_adam_done = (unsigned int *)alloc(4);
    M->fold = (float *)alloc((size_t)h1 * 4);
    if (failed) {
        mlp_free(M);
        return set_error(FFS_ENOMEM, "MLP buffers");
    }
    for (cudaStream_t &s : M->aux)
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
            (void)cudaGetLastError();
            s = nullptr;
            mlp_free(M);
            return set_error(FFS_ECUDA, "MLP streams");
        }
    for (cudaEvent_t &e : M->ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            (void)cudaGetLastError();
            e = nullptr;
            mlp_free(M);
            return set_error(FFS_ECUDA, "MLP events");
        }
    float *p = M->params, *g = M->grads;
    M->W1 = p; M->gW1 = g; p += nW1; g += nW1;
    M->b1 = p; M->gb1 = g; p += h1; g += h1;
    M->W2 = p; M->gW2 = g; p += nW2; g += nW2;
    M->b2 = p; M->gb2 = g; p += h2; g += h2;
    M->w3 = p; M->gw3 = g; p += h2; g += h2;
    M->b3 = p; M->gb3 = g;
    if (cudaMemset(M->params, 0, M->n_params * 4) || cudaMemset(M->m, 0, M->n_params * 4) ||
        cudaMemset(M->v, 0, M->n_params * 4) || cudaMemset(M->grads, 0, M->n_params * 4) || cudaMemset(M->err, 0, 4) ||
        cudaMemset(M->d_adam_t, 0, 8) || cudaMemset(M->d_adam_done, 0, 4) ||
        refresh_bf16(M, 0) || cudaDeviceSynchronize()) {
        mlp_free(M);
        return set_error(FFS_ECUDA, "MLP initialisation");
    }
    *out = M;
    return FFS_OK;
}

int ffs_mlp_destroy(ffs_mlp *M)
{
    mlp_free(M);
    return FFS_OK;
}

int ffs_mlp_input_width(const ffs_mlp *M) { return M ? M->K1 : -1; }

int ffs_mlp_set_params(ffs_mlp *M, const float *W1, const float *b1, const float *W2, const float *b2, const float *w3,
                       float b3)
{
    clear_error();
    if (!M || !W1 || !b1 || !W2 || !b2 || !w3) return set_error(FFS_EINVAL, "NULL argument");
    std::vector<float> w1p((size_t)M->h1 * M->K1, 0.0f);
    for (int o = 0; o < M->h1; ++o)
        for (int i = 0; i < M->in_dim; ++i) w1p[(size_t)o * M->K1 + i] = W1[(size_t)o * M->in_dim + i];
    FFS_CUDA_TRY(cudaMemcpy(M->W1, w1p.data(), w1p.size() * 4, cudaMemcpyHostToDevice));
    FFS_CUDA_TRY(cudaMemcpy(M->b1, b1, (size_t)M->h1 * 4, cudaMemcpyHostToDevice));
    FFS_CUDA_TRY(cudaMemcpy(M->W2, W2, (size_t)M->h2 * M->h1 * 4, cudaMemcpyHostToDevice));
    FFS_CUDA_TRY(cudaMemcpy(M->b2, b2, (size_t)M->h2 * 4, cudaMemcpyHostToDevice));
    FFS_CUDA_TRY(cudaMemcpy(M->w3, w3, (size_t)M->h2 * 4, cudaMemcpyHostToDevice));
    FFS_CUDA_TRY(cudaMemcpy(M->b3, &b3, 4, cudaMemcpyHostToDevice));
    FFS_CUDA_TRY(cudaMemset(M->m, 0, M->n_params * 4));
    FFS_CUDA_TRY(cudaMemset(M->v, 0, M->n_params * 4));
    FFS_CUDA_TRY(cudaMemset(M->d_adam_t, 0, 8));
    int rc = refresh_bf16(M, 0);
    if (rc) return rc;
    FFS_CUDA_TRY(cudaDeviceSynchronize());
    return FFS_OK;
}

// Host copies of the parameters (which = 0), the last step's gradients (1),
// or Adam's first (2) or second (3) moment estimates.
int ffs_mlp_get(const ffs_mlp *M, int32_t which, float *W1, float *b1, float *W2, float *b2, float *w3, float *b3)
{
    clear_error();
    if (!M) return set_error(FFS_EINVAL, "NULL MLP");
    if (which < 0 || which > 3) return set_error(FFS_EINVAL, "which %d outside 0..3", which);
    FFS_CUDA_TRY(cudaDeviceSynchronize());
    const float *src = which == 0 ? M->params : which == 1 ? M->grads : which == 2 ? M->m : M->v;
    std::vector<float> all(M->n_params);
    FFS_CUDA_TRY(cudaMemcpy(all.data(), src, all.size() * 4, cudaMemcpyDeviceToHost));
    size_t off = 0;
    if (W1)
        for (int o = 0; o < M->h1; ++o)
            for (int i = 0; i < M->in_dim; ++i) W1[(size_t)o * M->in_dim + i] = all[off + (size_t)o * M->K1 + i];
    off += (size_t)M->h1 * M->K1;
    if (b1) memcpy(b1, &all[off], (size_t)M->h1 * 4);
    off += M->h1;
    if (W2) memcpy(W2, &all[off], (size_t)M->h2 * M->h1 * 4);
    off += (size_t)M->h2 * M->h1;
    if (b2) memcpy(b2, &all[off], (size_t)M->h2 * 4);
    off += M->h2;
    if (w3) memcpy(w3, &all[off], (size_t)M->h2 * 4);
    off += M->h2;
    if (b3) *b3 = all[off];
    return FFS_OK;
}

int ffs_mlp_init(ffs_mlp *M, uint64_t seed, ffs_stream stream)
{
    clear_error();
    if (!M) return set_error(FFS_EINVAL, "NULL MLP");
    cudaStream_t st = (cudaStream_t)stream;
    auto blocks = [](int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 4096); };
    k_mlp_init<<<blocks((int64_t)M->h1 * M->K1), 256, 0, st>>>(M->W1, M->h1, M->in_dim, M->K1, seed, 1u, M->in_dim,
                                                               1.0f);
    k_mlp_init<<<blocks((int64_t)M->h2 * M->h1), 256, 0, st>>>(M->W2, M->h2, M->h1, M->h1, seed, 2u, M->h1, 1.0f);
    k_mlp_init<<<blocks(M->h2), 256, 0, st>>>(M->w3, 1, M->h2, M->h2, seed, 3u, M->h2, 0.1f);
    FFS_CUDA_TRY(cudaGetLastError());
    FFS_CUDA_TRY(cudaMemsetAsync(M->b1, 0, (size_t)M->h1 * 4, st));
    FFS_CUDA_TRY(cudaMemsetAsync(M->b2, 0, (size_t)M->h2 * 4, st));
    FFS_CUDA_TRY(cudaMemsetAsync(M->b3, 0, 4, st));
    FFS_CUDA_TRY(cudaMemsetAsync(M->m, 0, M->n_params * 4, st));
    FFS_CUDA_TRY(cudaMemsetAsync(M->v, 0, M->n_params * 4, st));
    FFS_CUDA_TRY(cudaMemsetAsync(M->grads, 0, M->n_params * 4, st));
    FFS_CUDA_TRY(cudaMemsetAsync(M->d_adam_t, 0, 8, st));
    return refresh_bf16(M, st);
}

int ffs_mlp_adam_steps(const ffs_mlp *M, int64_t *steps)
{
    clear_error();
    if (!M || !steps) return set_error(FFS_EINVAL, "NULL argument");
    long long t = 0;
    FFS_CUDA_TRY(cudaDeviceSynchronize());
    FFS_CUDA_TRY(cudaMemcpy(&t, M->d_adam_t, 8, cudaMemcpyDeviceToHost));
    *steps = (int64_t)t;
    return FFS_OK;
}

int64_t ffs_mlp_state_bytes(const ffs_mlp *M) { return M ? mlp_state_bytes(M) : -1; }

int ffs_mlp_save(const ffs_mlp *M, void *host, int64_t capacity, ffs_stream stream)
{
    clear_error();
    if (!M || !host) return set_error(FFS_EINVAL, "NULL argument");
    if (capacity < mlp_state_bytes(M))
        return set_error(FFS_EINVAL, "capacity %lld < %lld bytes", (long long)capacity, (long long)mlp_state_bytes(M));
    return mlp_save(M, host, (cudaStream_t)stream);
}

int ffs_mlp_load(ffs_mlp *M, const void *host, int64_t size, ffs_stream stream)
{
    clear_error();
    if (!M || !host) return set_error(FFS_EINVAL, "NULL argument");
    return mlp_load(M, host, size, (cudaStream_t)stream);
}

int ffs_mlp_forward(ffs_mlp *M, const uint16_t *x, int32_t ldx, int32_t B, float *y, ffs_stream stream)
{
    clear_error();
    if (!M || !x || !y) return set_error(FFS_EINVAL, "NULL argument");
    if (B < 1 || B > M->max_batch) return set_error(FFS_EINVAL, "batch %d outside [1, %d]", B, M->max_batch);
    if (ldx < M->in_dim) return set_error(FFS_EINVAL, "ldx %d < in_dim %d", ldx, M->in_dim);
    return mlp_forward(M, fwd_live(M), x, ldx, B, y, (cudaStream_t)stream);
}

int ffs_mlp_train_step(ffs_mlp *M, const uint16_t *x, int32_t ldx, const float *target, int32_t B, float lr,
                       float *loss, ffs_stream stream)
{
    clear_error();
    if (!M || !x || !target) return set_error(FFS_EINVAL, "NULL argument");
    if (B < 128 || B % 128 || B > M->max_batch)
        return set_error(FFS_EINVAL, "training batch %d must be a multiple of 128 and <= %d", B, M->max_batch);
    if (ldx < M->in_dim) return set_error(FFS_EINVAL, "ldx %d < in_dim %d", ldx, M->in_dim);
    cudaStream_t st = (cudaStream_t)stream, s1 = M->aux[0], s2 = M->aux[1];
    cudaEvent_t e_fork = M->ev[0], e_h1 = M->ev[1], e_dz2 = M->ev[2], e_xt = M->ev[3], e_dz1 = M->ev[4],
                e_s1 = M->ev[5], e_s2 = M->ev[6], e_w2t = M->ev[7];
    const int h1 = M->h1, h2 = M->h2, K1 = M->K1;
    // The step's dependency graph on three streams; the caller's stream `st`
    // carries the critical path (forward, loss, dZ1, gW1, Adam), s1 and
    // s2 the work beside it, joined back into `st` before Adam.
    FFS_CUDA_TRY(cudaEventRecord(e_fork, st));
    FFS_CUDA_TRY(cudaStreamWaitEvent(s1, e_fork, 0));
    FFS_CUDA_TRY(cudaStreamWaitEvent(s2, e_fork, 0));
    // s2: W2^T (BF16) for dZ1 = dZ2 W2, from the weights as they are now
    k_transpose_bf16<<<dim3((h1 + 31) / 32, (h2 + 31) / 32), dim3(32, 8), 0, s2>>>(M->W2b, h2, h1, h1, M->W2Tb, h2);
    FFS_CUDA_TRY(cudaEventRecord(e_w2t, s2));
    // s1: the loss zeroed, X^T for gW1 = dZ1^T X (B = XT [K1][B], zero rows
    // beyond in_dim)
    if (loss) FFS_CUDA_TRY(cudaMemsetAsync(loss, 0, 4, s1));
    k_transpose_bf16<<<dim3((K1 + 31) / 32, (B + 31) / 32), dim3(32, 8), 0, s1>>>(
        reinterpret_cast<const __nv_bfloat16 *>(x), B, M->in_dim, ldx, M->XT, B);
    if (K1 > M->in_dim) FFS_CUDA_TRY(cudaMemsetAsync(M->XT + (size_t)M->in_dim * B, 0, (size_t)(K1 - M->in_dim) * B * 2, s1));
    FFS_CUDA_TRY(cudaEventRecord(e_xt, s1));
    // st: the forward pass's hidden layers; the kernels of the critical path
    // are launched as programmatic dependents of the one before them
    GemmEpi e;
    memset(&e, 0, sizeof(e));
    e.err = M->err;
    e.pdl = 1;
    e.mode = 1;
    e.Db = M->H1;
    e.bias = M->b1;
    e.ldd = h1;
    int rc = gemm_bf16(x, ldx, M->W1b, K1, B, h1, M->in_dim, e, st);
    if (rc) return rc;
    FFS_CUDA_TRY(cudaEventRecord(e_h1, st));
    e.Db = M->H2;
    e.bias = M->b2;
    e.ldd = h2;
    if ((rc = gemm_bf16(M->H1, h1, M->W2b, h1, B, h2, h1, e, st))) return rc;
    // s2: H1^T for gW2 = dZ2^T H1, beside layer 2
    FFS_CUDA_TRY(cudaStreamWaitEvent(s2, e_h1, 0));
    k_transpose_bf16<<<dim3((h1 + 31) / 32, (B + 31) / 32), dim3(32, 8), 0, s2>>>(M->H1, B, h1, h1, M->H1T, B);
    // st: output layer, loss and its backpropagated signal (after the loss
    // was zeroed and X^T written on s1)
    FFS_CUDA_TRY(cudaStreamWaitEvent(st, e_xt, 0));
    FFS_CUDA_TRY(launch_pdl(k_out_loss_dz2, dim3((B * 32 + 255) / 256), dim3(256), 0, st, (const __nv_bfloat16 *)M->H2,
                            B, h2, (const float *)M->w3, (const float *)M->b3, target, M->dy, loss, M->dZ2, M->dZ2T));
    FFS_CUDA_TRY(cudaEventRecord(e_dz2, st));
    // s2: the output layer's gradients and gW2 = dZ2^T H1 (A = dZ2T [h2][B], B = H1T [h1][B])
    FFS_CUDA_TRY(cudaStreamWaitEvent(s2, e_dz2, 0));
    k_out_grads<<<(h2 + 31) / 32, dim3(32, 32), 0, s2>>>(M->H2, M->dZ2, M->dy, B, h2, M->gw3, M->gb2, M->gb3);
    e.mode = 0;
    e.pdl = 0;
    e.D = M->gW2;
    e.ldd = h1;
    if ((rc = gemm_bf16(M->dZ2T, B, M->H1T, B, h2, h1, B, e, s2))) return rc;
    e.pdl = 1;
    FFS_CUDA_TRY(cudaEventRecord(e_s2, s2));
    // st: dZ1 = (dZ2 W2) [H1 > 0] (A = dZ2 [B][h2], B = W2T [h1][h2]), FP32 and
    // BF16 transposed, in the GEMM's epilogue
    FFS_CUDA_TRY(cudaStreamWaitEvent(st, e_w2t, 0));
    e.mode = 3;
    e.D = M->dZ1;
    e.ldd = h1;
    e.mask = M->H1;
    e.ldm = h1;
    e.Dt = M->dZ1T;
    e.ldt = B;
    if ((rc = gemm_bf16(M->dZ2, h2, M->W2Tb, h2, B, h1, h2, e, st))) return rc;
    e.mode = 0;
    FFS_CUDA_TRY(cudaEventRecord(e_dz1, st));
    // s1: gb1 = column sums of dZ1, beside gW1
    FFS_CUDA_TRY(cudaStreamWaitEvent(s1, e_dz1, 0));
    k_colsum<float><<<(h1 + 31) / 32, dim3(32, 32), 0, s1>>>(M->dZ1, nullptr, B, h1, M->gb1);
    FFS_CUDA_TRY(cudaEventRecord(e_s1, s1));
    // st: gW1 = dZ1^T X (A = dZ1T [h1][B], B = XT [K1][B])
    e.D = M->gW1;
    e.ldd = K1;
    if ((rc = gemm_bf16(M->dZ1T, B, M->XT, B, h1, K1, B, e, st))) return rc;
    // join, then Adam, writing the BF16 weight copies of the next forward pass as it goes
    FFS_CUDA_TRY(cudaStreamWaitEvent(st, e_s1, 0));
    FFS_CUDA_TRY(cudaStreamWaitEvent(st, e_s2, 0));
    const int nW1 = h1 * K1, w2_off = nW1 + h1;
    const int adam_blocks = std::min(1024, (int)((M->n_params / 4 + 255) / 256));
    FFS_CUDA_TRY(launch_pdl(k_adam_bf16, dim3(adam_blocks), dim3(256), 0, st, M->params, (const float *)M->grads, M->m,
                            M->v, (int)M->n_params, lr, 0.9f, 0.999f, 1e-8f, M->d_adam_t, M->d_adam_done, nW1, w2_off,
                            h1, h2, M->W1b, M->W2b));
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

// Non-zero if a tensor-core kernel of this MLP timed out waiting (then cleared).
int ffs_mlp_check(ffs_mlp *M, ffs_stream stream)
{
    clear_error();
    if (!M) return set_error(FFS_EINVAL, "NULL MLP");
    int h = 0;
    FFS_CUDA_TRY(cudaMemcpyAsync(&h, M->err, 4, cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    FFS_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    if (h) {
        cudaMemsetAsync(M->err, 0, 4, (cudaStream_t)stream);
        return set_error(FFS_ETIMEOUT, "tensor-core GEMM wait timed out (code %d)", h);
    }
    return FFS_OK;
}

}  // extern "C"
