// ffs_capi.cu -- C ABI entry points: errors, instances, the batched decoder,
// Philox draws and population initialisation.
#include <atomic>
#include <climits>
#include <cstdlib>
#include <cstdarg>
#include <cstring>
#include <mutex>

#include "ffs_internal.cuh"
#include "ffs_lanes.cuh"

namespace fgpu {

bool injected_alloc_failure()
{
    static const long long at = [] {
        const char *e = getenv("FFS_INJECT_ALLOC_FAILURE");
        return e ? atoll(e) : 0LL;
    }();
    static std::atomic<long long> count{0};
    return at > 0 && ++count == at;
}


static thread_local std::string g_err;

int set_error(int status, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return status;
}

void clear_error() { g_err.clear(); }

int validate_rows(const void *p, int ld, int n)
{
    if (ld < n || (ld & 7) != 0)
        return set_error(FFS_EINVAL, "ld = %d must be >= n = %d and a multiple of 8", ld, n);
    if (((uintptr_t)p & 15u) != 0) return set_error(FFS_EINVAL, "population base must be 16-byte aligned");
    return FFS_OK;
}

// ---------------------------------------------------------------------------
// Batched decoder kernel.  One thread per chromosome; a warp's 32 lanes
// decode 32 rows in lock step (same instance, same control flow).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(512) k_eval(DecodeLayout L, const uint32_t *__restrict__ tab_g,
                                              const int32_t *__restrict__ stage_g,
                                              const int16_t *__restrict__ pop, int64_t N, int ld,
                                              int32_t *__restrict__ out, const int32_t *count_dev,
                                              unsigned long long *decoded)
{
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ DecodeLayout s_L;
    const int T = blockDim.x;
    const SmemMap map = smem_map(L.n, L.S, T, 0, L.obj_words);
    if (count_dev) N = *count_dev;
    stage_table(smem + map.tab, tab_g, table_words(L.n, L.S) + L.obj_words);
    int32_t *st = reinterpret_cast<int32_t *>(smem + map.stage);
    for (int i = threadIdx.x; i < 2 * L.S; i += T) st[i] = stage_g[i];
    if (threadIdx.x == 0) {
        s_L = L;
        s_L.M = st;
        s_L.heap_off = st + L.S;
        const uint32_t objt = tc::smem_u32(smem + map.tab + table_words(L.n, L.S));
        s_L.rel_sa = L.has_rel ? objt : 0u;
        s_L.due_sa = L.has_due ? objt + (uint32_t)L.obj_words * 2u : 0u;
    }
    __syncthreads();
    DecodeLayout &Ls = s_L;
    decode_tmem_begin(Ls);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpStageState *wst = reinterpret_cast<WarpStageState *>(smem + map.warp) + warp * L.S;
    uint32_t *region = thread_region(smem + map.region, Ls.thread_words);
    if (decoded && blockIdx.x == 0 && threadIdx.x == 0 && N > 0) atomicAdd(decoded, (unsigned long long)N);
    for (int64_t base = (int64_t)blockIdx.x * T + warp * 32; base < N; base += (int64_t)gridDim.x * T) {
        const int64_t c = base + lane;
        const int64_t cc = c < N ? c : N - 1;
        const int32_t ms = decode_chromosome(Ls, pop + cc * ld, region, T,
                                             reinterpret_cast<const uint16_t *>(smem + map.tab), wst);
        if (c < N) out[c] = ms;
    }
    decode_tmem_end(Ls);
}

static std::mutex g_plan_mutex;

static int plan_decode_uncached(const ffs_instance *inst, const void *kernel, int B_req, int T_req,
                                int bits_per_warp, int tmem_pref, Plan *out);

int plan_decode(const ffs_instance *inst, const void *kernel, int B_req, int T_req, int bits_per_warp, Plan *out,
                int variant)
{
    std::lock_guard<std::mutex> lock(g_plan_mutex);
    for (const auto &e : inst->plan_cache) {
        if (e.first.kernel == kernel && e.first.B_req == B_req && e.first.T_req == T_req &&
            e.first.bits_per_warp == bits_per_warp && e.first.variant == variant) {
            *out = e.second;
            return FFS_OK;
        }
    }
    int rc = plan_decode_uncached(inst, kernel, B_req, T_req, bits_per_warp, tmem_of(variant), out);
    if (rc == FFS_OK) {
        out->L.pairs = pairs_of(variant);
        inst->plan_cache.push_back({ffs_instance::PlanKey{kernel, B_req, T_req, bits_per_warp, variant}, *out});
    }
    return rc;
}

// Resident blocks per SM of `kernel` at this shape, or 0.
static int occupancy(const void *kernel, int T, size_t smem)
{
    int blocks = 0;
    if (cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, T, smem) != cudaSuccess) return 0;
    return blocks;
}

// Candidate shapes: chunk B x block size T, saved heaps in shared memory
// only, or (chunked decoding) a prefix of the stages' heaps in TMEM with `tb`
// blocks per SM sharing its 512 columns; a block's warps w, w + 4, ... share
// lane quarter w mod 4 and split the block's columns in ceil(warps / 4)
// groups.  Each TMEM
// shape pads its shared memory, if needed, so that no more than tb blocks
// are resident (a further block would wait in its TMEM allocation).  Score:
// resident threads (saturating at 1024), then fewer rounds, then TMEM or not
// as tmem_pref says (0: never, 1: only if it gains on the above, 2: preferred).
static int plan_decode_uncached(const ffs_instance *inst, const void *kernel, int B_req, int T_req,
                                int bits_per_warp, int tmem_pref, Plan *out)
{
    const int n = inst->n, S = inst->S;
    const size_t smem_cap = 232448;  // 227 KB per block on sm_100-class parts
    struct Cand {
        int T = 0, B = 0, blocks = 0, tmem_blocks = 0, group_cols = 0, tstages = 0, split = 0;
        size_t smem = 0;
        long score = -1;
    } best;
    const int single_B = round_up(n, 8);
    int Bs[8];
    int nb = 0;
    if (B_req > 0) {
        if (B_req % 8) return set_error(FFS_EINVAL, "decode_chunk %d is not a multiple of 8", B_req);
        Bs[nb++] = B_req >= n ? single_B : B_req;
    } else {
        Bs[nb++] = single_B;
        for (int b : {8, 16, 32, 64, 128})
            if (b < n) Bs[nb++] = b;
    }
    int Ts[8];
    int nt = 0;
    if (T_req > 0) {
        if (T_req % 32 || T_req > 512) return set_error(FFS_EINVAL, "block_threads %d must be a multiple of 32, <= 512", T_req);
        Ts[nt++] = T_req;
    } else {
        for (int t : {64, 128, 256, 320, 384, 448, 512}) Ts[nt++] = t;
    }
    auto consider = [&](const Cand &c, bool single) {
        const long resident = (long)c.blocks * c.T;
        const long sat = resident > 1024 ? 1024 : resident;
        const long rounds_penalty = single ? 0 : (long)(16 * 64 / c.B);
        Cand k = c;
        k.score = sat * 64 - rounds_penalty * 8 + (c.T == 128 ? 1 : 0) +
                  (c.tmem_blocks ? (tmem_pref == 2 ? 2 : -2) : 0);
        if (k.score > best.score) best = k;
    };
    for (int bi = 0; bi < nb; ++bi) {
        const int B = Bs[bi];
        const bool single = B >= n;
        for (int ti = 0; ti < nt; ++ti) {
            const int T = Ts[ti];
            const SmemMap m = smem_map(n, S, T, bits_per_warp, inst->obj_words);
            {
                const int tw = (single ? 0 : inst->heap_words) + B + 4;   // +4: read-ahead slots
                Cand c;
                c.T = T;
                c.B = B;
                c.smem = (size_t)(m.region + tw * T) * 4u;
                if (c.smem <= smem_cap && (c.blocks = occupancy(kernel, T, c.smem)) > 0) consider(c, single);
            }
            if (tmem_pref == 0 || single) continue;
            for (int tb : {1, 2, 4}) {
                const int groups = (T / 32 + 3) / 4;        // warps per lane quarter (at most)
                const int cols_block = 512 / tb;
                const int gcols = cols_block / groups;
                int split = 0, ns = 0;
                while (ns < S && split + inst->M_eff[ns] <= gcols) split += inst->M_eff[ns++];
                if (ns == 0) continue;
                Cand c;
                c.T = T;
                c.B = B;
                c.tmem_blocks = tb;
                c.group_cols = gcols;
                c.tstages = ns;
                c.split = split;
                const int tw = inst->heap_words - split + B + 4;
                c.smem = (size_t)(m.region + tw * T) * 4u;
                if (c.smem > smem_cap) continue;
                c.blocks = occupancy(kernel, T, c.smem);
                while (c.blocks > tb && c.smem + 4096 <= smem_cap) {
                    c.smem += 4096;
                    c.blocks = occupancy(kernel, T, c.smem);
                }
                if (c.blocks != tb) continue;
                consider(c, false);
            }
        }
    }
    (void)cudaGetLastError();
    if (best.score < 0)
        return set_error(FFS_EUNSUPPORTED, "no decoder launch shape fits shared memory (n=%d, S=%d)", n, S);
    Plan p;
    p.T = best.T;
    p.smem = best.smem;
    p.blocks_per_sm = best.blocks;
    DecodeLayout &L = p.L;
    memset(&L, 0, sizeof(L));
    L.n = n; L.S = S; L.SH = inst->SH; L.mulSH = 1u << inst->SH;
    L.single = best.B >= n ? 1 : 0;
    L.B = L.single ? single_B : best.B;
    L.heap_words = L.single ? 0 : inst->heap_words - best.split;
    L.thread_words = L.heap_words + L.B + 4;
    if (best.tmem_blocks) {
        L.tmem_cols = (uint32_t)(512 / best.tmem_blocks);
        L.tmem_group_cols = best.group_cols;
        L.tmem_stages = best.tstages;
        L.tmem_split = best.split;
    }
    L.obj_words = inst->obj_words;
    L.has_rel = inst->has_rel;
    L.has_due = inst->has_due;
    L.wt = (uint32_t)inst->wt;
    p.smem_words_fixed = smem_map(n, S, best.T, bits_per_warp, inst->obj_words).region;
    *out = p;
    return FFS_OK;
}

const void *eval_kernel() { return (const void *)k_eval; }

// ---------------------------------------------------------------------------
// The stage-parallel decoder kernel (ffs_lanes.cuh): a warp decodes
// floor(32 / S) chromosomes at a time, lane s of each group running stage s,
// their rows staged in the warp's part of shared memory.  It serves decode
// launches too small to fill the GPU with one chromosome per lane.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) k_eval_lanes(int n, int S, uint32_t SH, int MM, int obj_words, int has_rel,
                                                    int has_due, uint32_t wt, const uint32_t *__restrict__ tab_g,
                                                    const int32_t *__restrict__ stage_g,
                                                    const int16_t *__restrict__ pop, int64_t N, int ld,
                                                    int32_t *__restrict__ out, const int32_t *count_dev,
                                                    unsigned long long *decoded)
{
    extern __shared__ __align__(16) uint32_t smem[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, W = blockDim.x >> 5;
    const LaneSetup u = lanes_block_setup(smem, n, S, obj_words, has_rel, has_due, tab_g, stage_g, ld);
    if (count_dev) N = *count_dev;
    if (decoded && blockIdx.x == 0 && threadIdx.x == 0 && N > 0) atomicAdd(decoded, (unsigned long long)N);
    const int C = u.C;
    const int64_t items = (N + C - 1) / C;
    for (int64_t it = (int64_t)blockIdx.x * W + warp; it < items; it += (int64_t)gridDim.x * W) {
        const int64_t r0 = it * C;
        const int nrows = (int)min((int64_t)C, N - r0);
        const int4 *src = reinterpret_cast<const int4 *>(pop + r0 * ld);
        int4 *dst = reinterpret_cast<int4 *>(u.rows);
        for (int k = lane; k < nrows * (ld >> 3); k += 32) dst[k] = src[k];
        __syncwarp();
        const bool active = u.g < nrows;
        const uint32_t sM = (active ? (uint32_t)u.s : 0xFFu) | (u.Ms << 8) | (SH << 16);
        const uint32_t genes = u.rows_sa + (active ? (uint32_t)(u.g * ld * 2) : 0u);
        const int32_t v = lane_decode_dispatch(MM, u.tab, u.row_bytes, genes, u.nS, sM, u.win, u.rel, u.due, wt);
        if (active && u.s == S - 1) out[r0 + u.g] = v;
        __syncwarp();   // the buffer is refilled next
    }
}

// Which decoder a launch of N chromosomes takes: variant 5 asks for the
// stage-parallel one; with the library's choice (variant 0) it is taken when
// a cost model, fitted to GB300 measurements of both decoders, predicts it
// at most 0.7x the one-lane decoder's time.  Each decoder's cycles are the
// larger of a latency term (its chain: n S dispatches at about 60 cycles /
// start_{S-1} + n steps at about 260) and an issue term (its warp
// instructions -- about 30 per dispatch per 32 chromosomes / 58 per step per
// floor(32 / S) chromosomes -- over the SMs' 4 schedulers at the issue
// rates the two kernels reach, 0.6 / 0.55 per cycle).
bool lanes_decode_pays(const ffs_instance *inst, int64_t N, int variant)
{
    if (inst->S > 32) return false;
    if (variant == kVariantLanes) return true;
    if (variant != 0 || N <= 0) return false;
    const double n = inst->n, S = inst->S, sched = 4.0 * inst->num_sms;
    double steps = n;
    for (int j = 0; j + 1 < inst->S; ++j) steps += inst->M_eff[j] + 1;
    const double C = (double)(32 / inst->S);
    const double one_lane = std::max(n * S * 60.0, (double)N / 32.0 * n * S * 30.0 / (sched * 0.6));
    const double lanes = std::max(steps * 260.0, (double)N / C * steps * 58.0 / (sched * 0.55));
    return lanes <= 0.7 * one_lane;
}

int plan_lanes(const ffs_instance *inst, int64_t N, int ld, LanesPlan *out)
{
    const int S = inst->S, n = inst->n;
    if (S > 32) return set_error(FFS_EUNSUPPORTED, "the stage-parallel decoder takes at most 32 stages, not %d", S);
    LanesPlan p;
    for (int m : inst->M_eff) p.MM = std::max(p.MM, m);
    const int W = p.T / 32;
    p.C = 32 / S;
    p.smem = ((size_t)round_up(table_words(n, S) + inst->obj_words + S, 4) + (size_t)W * p.C * ld / 2) * 4;
    if (p.smem > 232448) return set_error(FFS_EUNSUPPORTED, "stage-parallel decoder: %zu bytes of shared memory", p.smem);
    const int64_t items = (N + p.C - 1) / p.C;
    int64_t blocks = (items + W - 1) / W;
    if (blocks > (int64_t)inst->num_sms * 16) blocks = (int64_t)inst->num_sms * 16;
    p.blocks = (int)std::max<int64_t>(blocks, 1);
    *out = p;
    return FFS_OK;
}

int launch_eval_lanes(const ffs_instance *inst, const int16_t *pop, int64_t N, int ld, int32_t *out,
                      const int32_t *count_dev, unsigned long long *decoded, cudaStream_t st)
{
    LanesPlan p;
    int rc = plan_lanes(inst, N, ld, &p);
    if (rc) return rc;
    FFS_CUDA_TRY(cudaFuncSetAttribute(k_eval_lanes, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
    k_eval_lanes<<<p.blocks, p.T, p.smem, st>>>(inst->n, inst->S, (uint32_t)inst->SH, p.MM, inst->obj_words,
                                                inst->has_rel, inst->has_due, (uint32_t)inst->wt, inst->d_tab,
                                                inst->d_stage, pop, N, ld, out, count_dev, decoded);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

int launch_eval(const ffs_instance *inst, const int16_t *pop, int64_t N, int ld, int32_t *out,
                const int32_t *count_dev, int B_req, int T_req, unsigned long long *decoded,
                cudaStream_t st, int variant)
{
    // an explicit launch shape (chunk, threads) keeps the one-lane decoder
    if (lanes_decode_pays(inst, N, (B_req || T_req) && variant == 0 ? -1 : variant))
        return launch_eval_lanes(inst, pop, N, ld, out, count_dev, decoded, st);
    Plan p;
    const int T_sp = spread_threads(inst, N, T_req);
    int rc = plan_decode(inst, (const void *)k_eval, B_req, T_sp, 0, &p, variant);
    if (rc && T_sp != T_req) rc = plan_decode(inst, (const void *)k_eval, B_req, T_req, 0, &p, variant);
    if (rc) return rc;
    FFS_CUDA_TRY(cudaFuncSetAttribute(k_eval, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)p.smem));
    const int grid = grid_for(inst, p, N);
    k_eval<<<grid, p.T, p.smem, st>>>(p.L, inst->d_tab, inst->d_stage, pop, N, ld, out, count_dev, decoded);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

// ---------------------------------------------------------------------------
// Philox draws and initial populations.
// ---------------------------------------------------------------------------
__global__ void k_philox(uint64_t seed, uint32_t purpose, uint32_t island, uint32_t generation,
                         uint32_t cell0, int n_cells, int n_draws, uint32_t *out)
{
    const int64_t total_blocks = (int64_t)n_cells * ((n_draws + 3) / 4);
    const int per = (n_draws + 3) / 4;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total_blocks;
         t += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(t / per), b = (int)(t % per);
        const U4 v = draw_block(seed, purpose, island, generation, cell0 + (uint32_t)c, (uint32_t)b);
        const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int d = b * 4 + k;
            if (d < n_draws) out[(int64_t)c * n_draws + d] = w[k];
        }
    }
}

// One thread per chromosome (cellular) or per pair (pseudo): Fisher-Yates in
// the row itself (global memory, the thread's own row).
__global__ void k_init(uint64_t seed, uint32_t island, int kind, int64_t N, int n, int ld, int16_t *pop)
{
    const int64_t units = kind == 0 ? N : N / 2;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < units;
         u += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r = kind == 0 ? u : 2 * u;
        int16_t *a = pop + r * ld;
        for (int i = 0; i < ld; ++i) a[i] = (int16_t)(i < n ? i : 0);
        U4 blk{0, 0, 0, 0};
        for (int i = n - 1; i >= 1; --i) {
            const int d = n - 1 - i;
            if ((d & 3) == 0) blk = draw_block(seed, kPurposeInit, island, 0u, (uint32_t)r, (uint32_t)(d >> 2));
            const uint32_t x = (d & 3) == 0 ? blk.x : (d & 3) == 1 ? blk.y : (d & 3) == 2 ? blk.z : blk.w;
            const int j = (int)uniform_below(x, (uint32_t)(i + 1));
            const int16_t t = a[i];
            a[i] = a[j];
            a[j] = t;
        }
        if (kind == 1) {
            int16_t *b = a + ld;
            for (int i = 0; i < ld; ++i) b[i] = i < n ? a[n - 1 - i] : (int16_t)0;
        }
    }
}

int launch_init(const ffs_instance *inst, uint64_t seed, uint32_t island, int kind, int64_t N, int ld,
                int16_t *pop, cudaStream_t st)
{
    const int64_t units = kind == 0 ? N : N / 2;
    if (units <= 0) return FFS_OK;
    int64_t g = (units + 127) / 128;
    if (g > 65535) g = 65535;
    k_init<<<(int)g, 128, 0, st>>>(seed, island, kind, N, inst->n, ld, pop);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

}  // namespace fgpu

#ifdef FFS_DEBUG_CHECKS
namespace fgpu {
__device__ int g_ffs_check_error = 0;
}
#endif

namespace fgpu {
bool eager_generations()
{
    static const bool eager = [] {
        const char *v = getenv("FFS_EAGER");
        return v && v[0] && strcmp(v, "0") != 0;
    }();
    return eager;
}
}  // namespace fgpu

using namespace fgpu;

extern "C" {

const char *ffs_last_error(void) { return g_err.c_str(); }

int ffs_debug_checks(int32_t *enabled)
{
    clear_error();
    if (!enabled) return set_error(FFS_EINVAL, "NULL argument");
#ifdef FFS_DEBUG_CHECKS
    *enabled = 1;
#else
    *enabled = 0;
#endif
    return FFS_OK;
}

int ffs_debug_check_error(int32_t *code, int32_t reset, ffs_stream stream)
{
    clear_error();
    if (!code) return set_error(FFS_EINVAL, "NULL argument");
    *code = 0;
#ifdef FFS_DEBUG_CHECKS
    cudaStream_t st = (cudaStream_t)stream;
    FFS_CUDA_TRY(cudaStreamSynchronize(st));
    FFS_CUDA_TRY(cudaMemcpyFromSymbol(code, g_ffs_check_error, sizeof(int32_t)));
    if (reset) {
        const int32_t zero = 0;
        FFS_CUDA_TRY(cudaMemcpyToSymbol(g_ffs_check_error, &zero, sizeof(int32_t)));
    }
#else
    (void)reset;
    (void)stream;
#endif
    return FFS_OK;
}

void ffs_params_default(ffs_params *p)
{
    if (!p) return;
    memset(p, 0, sizeof(*p));
    p->seed = 7;
    p->cell_pc = 4294967296ull;            // 1.00
    p->cell_pm = 214748364ull;             // floor(0.05 * 2^32)
    p->pseudo_pc = 3221225472ull;          // 0.75
    p->cell_replace_le = 0;
    p->pseudo_always = 0;
    p->migration_mode = FFS_MIG_RING;
    p->migration_gap = 50;
    p->ring_num = 2;
    p->ring_den = 100;
    p->theta_num = 1;
    p->theta_den = 1;
}

int ffs_instance_create_objective(int32_t n, int32_t S, const int32_t *M, const int32_t *p, const int32_t *release,
                                  const int32_t *due, int32_t wt, ffs_instance **out)
{
    clear_error();
    if (!out || !M || !p) return set_error(FFS_EINVAL, "NULL argument");
    *out = nullptr;
    if (n < 1 || n > 32767) return set_error(FFS_EINVAL, "n_jobs = %d outside [1, 32767]", n);
    if (S < 1 || S > kMaxStages) return set_error(FFS_EINVAL, "n_stages = %d outside [1, %d]", S, kMaxStages);
    if (due && wt < 0) return set_error(FFS_EINVAL, "tardiness weight %d < 0", wt);
    int64_t total = 0;
    for (int s = 0; s < S; ++s) {
        if (M[s] < 1) return set_error(FFS_EINVAL, "machines_per_stage[%d] = %d < 1", s, M[s]);
        if ((M[s] < n ? M[s] : n) > kMaxM)
            return set_error(FFS_EUNSUPPORTED, "stage %d: %d machines (> %d) for %d jobs", s, M[s], kMaxM, n);
    }
    for (int64_t i = 0; i < (int64_t)n * S; ++i) {
        if (p[i] < 1) return set_error(FFS_EINVAL, "proc_time[%lld][%lld] = %d < 1",
                                       (long long)(i / S), (long long)(i % S), p[i]);
        if (p[i] > 65535) return set_error(FFS_EUNSUPPORTED, "proc_time[%lld][%lld] = %d > 65535",
                                           (long long)(i / S), (long long)(i % S), p[i]);
        total += p[i];
    }
    int64_t max_rel = 0;
    for (int j = 0; release && j < n; ++j) {
        if (release[j] < 0) return set_error(FFS_EINVAL, "release[%d] = %d < 0", j, release[j]);
        if (release[j] > max_rel) max_rel = release[j];
    }
    for (int j = 0; due && j < n; ++j)
        if (due[j] < 0) return set_error(FFS_EINVAL, "due[%d] = %d < 0", j, due[j]);
    int bits = 0;
    while ((1 << bits) <= n) ++bits;            // ids 1..n fit in `bits`
    const int SH = bits + 1;
    // every completion time is below max release + total processing time
    const int64_t horizon = max_rel + total;
    if (horizon >= (int64_t(1) << (32 - SH)))
        return set_error(FFS_EOVERFLOW, "latest completion bound %lld needs more than %d bits of key",
                         (long long)horizon, 32 - SH);
    if (due && (int64_t)wt * n * horizon + horizon > INT32_MAX)
        return set_error(FFS_EOVERFLOW, "objective bound WT * n * %lld + %lld exceeds int32", (long long)horizon,
                         (long long)horizon);
    ffs_instance *I = new ffs_instance();
    I->n = n; I->S = S; I->SH = SH; I->total_p = total;
    cudaGetDevice(&I->device);
    cudaDeviceGetAttribute(&I->num_sms, cudaDevAttrMultiProcessorCount, I->device);
    I->host_M.assign(M, M + S);
    I->host_p.assign(p, p + (size_t)n * S);
    I->has_rel = release ? 1 : 0;
    I->has_due = due ? 1 : 0;
    I->wt = due ? wt : 0;
    if (release) I->host_R.assign(release, release + n);
    if (due) I->host_D.assign(due, due + n);
    I->obj_words = (release || due) ? objective_words(n) : 0;
    I->M_eff.resize(S);
    I->heap_off.resize(S);
    int off = 0;
    for (int s = 0; s < S; ++s) {
        I->M_eff[s] = M[s] < n ? M[s] : n;
        I->heap_off[s] = off;
        off += I->M_eff[s];
    }
    I->heap_words = off;
    I->tab_words = table_words(n, S);
    // the time table (uint16), then the release and due tables (uint32, entry j + 1 = job j)
    std::vector<uint16_t> tab((size_t)(I->tab_words + I->obj_words) * 2, 0u);
    const int rowh = table_row_halves(n);
    for (int s = 0; s < S; ++s)
        for (int j = 0; j < n; ++j) tab[(size_t)s * rowh + j + 1] = (uint16_t)p[(size_t)j * S + s];
    if (I->obj_words) {
        uint32_t *w = reinterpret_cast<uint32_t *>(tab.data()) + I->tab_words;
        const int half = I->obj_words / 2;
        for (int j = 0; j < n; ++j) {
            w[j + 1] = release ? (uint32_t)release[j] : 0u;
            w[half + j + 1] = due ? (uint32_t)due[j] : 0u;
        }
    }
    std::vector<int32_t> stage(2 * S);
    for (int s = 0; s < S; ++s) { stage[s] = I->M_eff[s]; stage[S + s] = I->heap_off[s]; }
    // table_words and obj_words are multiples of 4: the 16-byte staging loads stay inside
    const size_t tab_bytes = (size_t)(I->tab_words + I->obj_words) * 4;
    if (cudaMalloc(&I->d_tab, tab_bytes) != cudaSuccess || cudaMalloc(&I->d_stage, 8 * S) != cudaSuccess) {
        cudaFree(I->d_tab);
        delete I;
        (void)cudaGetLastError();
        return set_error(FFS_ENOMEM, "device allocation of the instance tables failed");
    }
    if (cudaMemcpy(I->d_tab, tab.data(), tab_bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(I->d_stage, stage.data(), stage.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(I->d_tab);
        cudaFree(I->d_stage);
        delete I;
        return set_error(FFS_ECUDA, "copy of the instance tables failed");
    }
    *out = I;
    return FFS_OK;
}

int ffs_instance_create(int32_t n, int32_t S, const int32_t *M, const int32_t *p, ffs_instance **out)
{
    return ffs_instance_create_objective(n, S, M, p, nullptr, nullptr, 0, out);
}

int ffs_instance_destroy(ffs_instance *I)
{
    if (!I) return FFS_OK;
    cudaFree(I->d_tab);
    cudaFree(I->d_stage);
    cudaFree(I->d_host_pop);
    cudaFree(I->d_host_ms);
    delete I;
    return FFS_OK;
}

int ffs_population_eval(const ffs_instance *I, const int16_t *pop, int64_t N, int32_t ld, int32_t *ms,
                        ffs_stream stream)
{
    clear_error();
    if (!I) return set_error(FFS_EINVAL, "NULL instance");
    if (N < 0) return set_error(FFS_EINVAL, "N = %lld < 0", (long long)N);
    if (N == 0) return FFS_OK;
    if (!pop || !ms) return set_error(FFS_EINVAL, "NULL population or output");
    int rc = validate_rows(pop, ld, I->n);
    if (rc) return rc;
    return launch_eval(I, pop, N, ld, ms, nullptr, 0, 0, nullptr, (cudaStream_t)stream);
}

int ffs_population_eval_tuned(const ffs_instance *I, const int16_t *pop, int64_t N, int32_t ld, int32_t *ms,
                              int32_t decode_chunk, int32_t block_threads, int32_t variant, ffs_stream stream)
{
    clear_error();
    if (!I) return set_error(FFS_EINVAL, "NULL instance");
    if (N < 0) return set_error(FFS_EINVAL, "N = %lld < 0", (long long)N);
    if (decode_chunk < 0 || block_threads < 0) return set_error(FFS_EINVAL, "negative launch shape");
    if (variant < 0 || (variant > kMaxVariant && variant != kVariantLanes))
        return set_error(FFS_EINVAL, "decoder variant %d", variant);
    if (variant == kVariantLanes && I->S > 32)
        return set_error(FFS_EUNSUPPORTED, "the stage-parallel decoder takes at most 32 stages, not %d", I->S);
    if (N == 0) return FFS_OK;
    if (!pop || !ms) return set_error(FFS_EINVAL, "NULL population or output");
    int rc = validate_rows(pop, ld, I->n);
    if (rc) return rc;
    return launch_eval(I, pop, N, ld, ms, nullptr, decode_chunk, block_threads, nullptr, (cudaStream_t)stream,
                       variant);
}

int ffs_decode_plan(const ffs_instance *I, int32_t kernel, int32_t decode_chunk, int32_t block_threads,
                    int32_t variant, int32_t *chunk_out, int32_t *threads_out, int32_t *blocks_per_sm,
                    int64_t *smem_bytes, int32_t *tmem_cols)
{
    clear_error();
    if (!I) return set_error(FFS_EINVAL, "NULL instance");
    if (kernel < 0 || kernel > 2) return set_error(FFS_EINVAL, "kernel %d is not 0, 1 or 2", kernel);
    if (variant < 0 || variant > kMaxVariant) return set_error(FFS_EINVAL, "decoder variant %d", variant);
    Plan p;
    const void *k = kernel == 0 ? eval_kernel() : kernel == 1 ? cellular_kernel() : step_decode_kernel();
    int rc = plan_decode(I, k, decode_chunk, block_threads, kernel == 1 ? mark_words(I->n) : 0, &p, variant);
    if (rc) return rc;
    if (chunk_out) *chunk_out = p.L.B;
    if (threads_out) *threads_out = p.T;
    if (blocks_per_sm) *blocks_per_sm = p.blocks_per_sm;
    if (smem_bytes) *smem_bytes = (int64_t)p.smem;
    if (tmem_cols) *tmem_cols = (int32_t)p.L.tmem_cols;
    return FFS_OK;
}

int ffs_population_eval_host(const ffs_instance *I_, const int16_t *pop, int64_t N, int32_t ld,
                             int32_t *ms, ffs_stream stream)
{
    clear_error();
    ffs_instance *I = const_cast<ffs_instance *>(I_);
    if (!I) return set_error(FFS_EINVAL, "NULL instance");
    if (N < 0) return set_error(FFS_EINVAL, "N = %lld < 0", (long long)N);
    if (N == 0) return FFS_OK;
    if (!pop || !ms) return set_error(FFS_EINVAL, "NULL population or output");
    if (ld < I->n || (ld & 7)) return set_error(FFS_EINVAL, "ld = %d must be >= n and a multiple of 8", ld);
    const size_t need = (size_t)N * ld * 2;
    if (need > I->host_cap) {
        cudaFree(I->d_host_pop);
        cudaFree(I->d_host_ms);
        I->d_host_pop = nullptr;
        I->d_host_ms = nullptr;
        I->host_cap = 0;
        if (cudaMalloc(&I->d_host_pop, need) != cudaSuccess ||
            cudaMalloc(&I->d_host_ms, (size_t)N * 4) != cudaSuccess) {
            (void)cudaGetLastError();
            return set_error(FFS_ENOMEM, "device staging buffer of %zu bytes", need);
        }
        I->host_cap = need;
    }
    cudaStream_t st = (cudaStream_t)stream;
    FFS_CUDA_TRY(cudaMemcpyAsync(I->d_host_pop, pop, need, cudaMemcpyHostToDevice, st));
    int rc = launch_eval(I, I->d_host_pop, N, ld, I->d_host_ms, nullptr, 0, 0, nullptr, st);
    if (rc) return rc;
    FFS_CUDA_TRY(cudaMemcpyAsync(ms, I->d_host_ms, (size_t)N * 4, cudaMemcpyDeviceToHost, st));
    FFS_CUDA_TRY(cudaStreamSynchronize(st));
    return FFS_OK;
}

int ffs_philox_draws(uint64_t seed, uint32_t purpose, uint32_t island, uint32_t generation, uint32_t cell0,
                     int32_t n_cells, int32_t n_draws, uint32_t *out, ffs_stream stream)
{
    clear_error();
    if (n_cells < 0 || n_draws < 0) return set_error(FFS_EINVAL, "negative size");
    if (n_cells == 0 || n_draws == 0) return FFS_OK;
    if (!out) return set_error(FFS_EINVAL, "NULL output");
    if (purpose > 255) return set_error(FFS_EINVAL, "purpose %u > 255", purpose);
    const int64_t blocks = (int64_t)n_cells * ((n_draws + 3) / 4);
    int64_t g = (blocks + 255) / 256;
    if (g > 4096) g = 4096;
    k_philox<<<(int)g, 256, 0, (cudaStream_t)stream>>>(seed, purpose, island, generation, cell0, n_cells,
                                                        n_draws, out);
    FFS_CUDA_TRY(cudaGetLastError());
    return FFS_OK;
}

int ffs_population_init(const ffs_instance *I, uint64_t seed, uint32_t island, int32_t kind, int64_t N,
                        int32_t ld, int16_t *pop, ffs_stream stream)
{
    clear_error();
    if (!I) return set_error(FFS_EINVAL, "NULL instance");
    if (kind != 0 && kind != 1) return set_error(FFS_EINVAL, "kind %d is not 0 (cellular) or 1 (pseudo)", kind);
    if (N < 0 || (kind == 1 && (N & 1))) return set_error(FFS_EINVAL, "bad N = %lld", (long long)N);
    if (N == 0) return FFS_OK;
    if (!pop) return set_error(FFS_EINVAL, "NULL population");
    int rc = validate_rows(pop, ld, I->n);
    if (rc) return rc;
    return launch_init(I, seed, island, kind, N, ld, pop, (cudaStream_t)stream);
}

}  // extern "C"
