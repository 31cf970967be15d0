/*
 * sanitize_check.c -- TEST INFRASTRUCTURE ONLY: runs every entry point of
 * the CPU oracle once on small seeded cases, built with AddressSanitizer and
 * UndefinedBehaviorSanitizer (tests/test_oracle_sanitizers.py compiles it
 * together with ffs_oracle.c and runs it on the host).  Any out-of-bounds
 * access, leak, use after free, signed overflow or misaligned access in the
 * oracle aborts the run; the few invariants checked here only make sure
 * every path really executed.  Inputs come from a small LCG of this file
 * (no arithmetic of the method).
 */
#include <stdio.h>

#include "ffs_oracle.c"

static uint64_t lcg_state = 0x9E3779B97F4A7C15ull;

static uint32_t lcg(void)
{
    lcg_state = lcg_state * 6364136223846793005ull + 1442695040888963407ull;
    return (uint32_t)(lcg_state >> 33);
}

static int32_t lcg_range(int32_t lo, int32_t hi) { return lo + (int32_t)(lcg() % (uint32_t)(hi - lo + 1)); }

static int failures = 0;

#define CHECK(cond)                                                         \
    do {                                                                    \
        if (!(cond)) {                                                      \
            fprintf(stderr, "check failed at line %d: %s\n", __LINE__, #cond); \
            ++failures;                                                     \
        }                                                                   \
    } while (0)

static int is_perm(const int16_t *row, int32_t n)
{
    char *seen = (char *)calloc((size_t)n, 1);
    int ok = 1;
    for (int32_t i = 0; i < n; ++i) {
        if (row[i] < 0 || row[i] >= n || seen[row[i]]) { ok = 0; break; }
        seen[row[i]] = 1;
    }
    free(seen);
    return ok;
}

typedef struct {
    int32_t n, S;
    int32_t *M, *p, *p_u, *release, *due;
    int32_t W;
} case_t;

static case_t make_case(int32_t n, int32_t S, int32_t mlo, int32_t mhi)
{
    case_t c;
    c.n = n;
    c.S = S;
    c.M = (int32_t *)malloc((size_t)S * sizeof(int32_t));
    c.W = 0;
    for (int32_t s = 0; s < S; ++s) { c.M[s] = lcg_range(mlo, mhi); c.W += c.M[s]; }
    c.p = (int32_t *)malloc((size_t)n * S * sizeof(int32_t));
    for (int32_t i = 0; i < n * S; ++i) c.p[i] = lcg_range(1, 99);
    c.p_u = (int32_t *)malloc((size_t)n * c.W * sizeof(int32_t));
    for (int32_t i = 0; i < n * c.W; ++i) c.p_u[i] = lcg_range(1, 99);
    c.release = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    c.due = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    for (int32_t j = 0; j < n; ++j) {
        c.release[j] = lcg_range(0, 200);
        c.due[j] = c.release[j] + lcg_range(10, 400);
    }
    return c;
}

static void free_case(case_t *c)
{
    free(c->M); free(c->p); free(c->p_u); free(c->release); free(c->due);
}

static void run_decoders(case_t *c, const orc_objective *obj)
{
    const int32_t n = c->n, S = c->S;
    int16_t *perm = (int16_t *)malloc((size_t)n * sizeof(int16_t));
    int64_t *gantt = (int64_t *)malloc((size_t)n * S * 5 * sizeof(int64_t));
    for (int t = 0; t < 4; ++t) {
        orc_init_chromosome(11, 0, (uint32_t)t, n, perm);
        CHECK(is_perm(perm, n));
        const int64_t v = orc_decode_obj(n, S, c->M, c->p, obj, perm, gantt);
        CHECK(v > 0);
        CHECK(orc_decode_obj(n, S, c->M, c->p, obj, perm, NULL) == v);
        if (!obj) CHECK(orc_decode(n, S, c->M, c->p, perm, NULL) == v);
    }
    perm[0] = (int16_t)n;   /* an invalid gene */
    CHECK(orc_decode_obj(n, S, c->M, c->p, obj, perm, NULL) == -1);
    int16_t *genes = (int16_t *)malloc((size_t)n * S * sizeof(int16_t));
    for (int t = 0; t < 3; ++t) {
        orc_assign_init_row(5, 1, (uint32_t)t, n, S, c->M, genes);
        CHECK(orc_decode_assign(n, S, c->M, c->p_u, obj, genes, gantt) > 0);
    }
    genes[0] = (int16_t)c->M[0];
    CHECK(orc_decode_assign(n, S, c->M, c->p_u, obj, genes, NULL) == -1);
    if (n <= 5) {
        int16_t best[8];
        int64_t worst = 0;
        const int64_t lo = orc_bruteforce_obj(n, S, c->M, c->p, obj, &worst, best);
        CHECK(lo > 0 && lo <= worst && is_perm(best, n));
        CHECK(orc_decode_obj(n, S, c->M, c->p, obj, best, NULL) == lo);
    }
    free(perm); free(gantt); free(genes);
}

static void run_job_order_ga(case_t *c, const orc_objective *obj)
{
    const int32_t n = c->n, S = c->S, rows = 3, cols = 4, N = rows * cols, size = 8;
    const int64_t ld = (n + 7) / 8 * 8;
    orc_params prm = { 7, 0xFFFFFFFFull + 1ull, 1288490189ull, 3221225472ull, 0, 0, obj };
    int16_t *pop = (int16_t *)calloc((size_t)N * ld, sizeof(int16_t));
    int16_t *nxt = (int16_t *)calloc((size_t)N * ld, sizeof(int16_t));
    int64_t *ms = (int64_t *)calloc((size_t)N, sizeof(int64_t));
    int64_t *nms = (int64_t *)calloc((size_t)N, sizeof(int64_t));
    for (int32_t i = 0; i < N; ++i) orc_init_chromosome(7, 0, (uint32_t)i, n, pop + i * ld);
    orc_eval_population_obj(n, S, c->M, c->p, obj, pop, N, ld, ms);
    for (uint32_t g = 1; g <= 3; ++g) {
        prm.cell_replace_le = (int32_t)(g & 1u);
        CHECK(orc_cellular_generation(n, S, c->M, c->p, &prm, 0, g, rows, cols, ld, pop, ms, nxt, nms) == N);
        for (int32_t i = 0; i < N; ++i) CHECK(is_perm(nxt + i * ld, n) && nms[i] <= ms[i]);
        int16_t *t = pop; pop = nxt; nxt = t;
        int64_t *u = ms; ms = nms; nms = u;
    }
    /* screened generation, K = 3 candidates with arbitrary scores */
    float scores[3 * 12];
    for (int i = 0; i < 36; ++i) scores[i] = (float)(lcg() % 1000) * 0.01f;
    int32_t chosen[12];
    int16_t *cands = (int16_t *)malloc((size_t)N * 3 * n * sizeof(int16_t));
    CHECK(orc_screened_cellular_generation(n, S, c->M, c->p, &prm, 0, 4, rows, cols, ld, pop, ms, nxt, nms, scores,
                                           3, chosen, cands) == N);
    for (int32_t i = 0; i < N; ++i) CHECK(chosen[i] >= 0 && chosen[i] < 3);
    free(cands);
    /* pseudo island of `size` rows */
    int16_t *ppop = (int16_t *)calloc((size_t)size * ld, sizeof(int16_t));
    int16_t *pnxt = (int16_t *)calloc((size_t)size * ld, sizeof(int16_t));
    int64_t *pms = (int64_t *)calloc((size_t)size, sizeof(int64_t));
    int64_t *pnms = (int64_t *)calloc((size_t)size, sizeof(int64_t));
    for (int32_t k = 0; k < size / 2; ++k) orc_init_pseudo_pair(7, 1, k, n, ppop + 2 * k * ld, ppop + (2 * k + 1) * ld);
    orc_eval_population_obj(n, S, c->M, c->p, obj, ppop, size, ld, pms);
    for (uint32_t g = 1; g <= 3; ++g) {
        prm.pseudo_always = (int32_t)(g & 1u);
        (void)orc_pseudo_generation(n, S, c->M, c->p, &prm, 1, g, size, ld, ppop, pms, pnxt, pnms);
        for (int32_t i = 0; i < size; ++i) CHECK(is_perm(pnxt + i * ld, n));
        int16_t *t = ppop; ppop = pnxt; pnxt = t;
        int64_t *u = pms; pms = pnms; pnms = u;
    }
    /* migration: ring over the two islands, then penetration both ways */
    int32_t sizes[2] = { N, size };
    int16_t *pops[2] = { pop, ppop };
    int64_t *mss[2] = { ms, pms };
    orc_migrate_ring(2, sizes, ld, n, pops, mss, 1, 4);
    (void)orc_migrate_penetration(N, size, ld, n, pop, ms, ppop, pms, 1, 1);
    (void)orc_migrate_penetration(size, N, ld, n, ppop, pms, pop, ms, 1, 1);
    for (int32_t i = 0; i < N; ++i) CHECK(is_perm(pop + i * ld, n));
    for (int32_t i = 0; i < size; ++i) CHECK(is_perm(ppop + i * ld, n));
    int32_t order[12];
    orc_rank_island(N, ms, order);
    for (int32_t i = 1; i < N; ++i) CHECK(ms[order[i - 1]] <= ms[order[i]]);
    free(pop); free(nxt); free(ms); free(nms); free(ppop); free(pnxt); free(pms); free(pnms);
}

static void run_assign_ga(case_t *c, const orc_objective *obj)
{
    const int32_t n = c->n, S = c->S, L = n * S, rows = 2, cols = 3, N = rows * cols;
    const int64_t ld = (L + 7) / 8 * 8;
    orc_params prm = { 9, 0xFFFFFFFFull + 1ull, 2147483648ull, 3221225472ull, 0, 0, obj };
    int16_t *pop = (int16_t *)calloc((size_t)N * ld, sizeof(int16_t));
    int16_t *nxt = (int16_t *)calloc((size_t)N * ld, sizeof(int16_t));
    int64_t *ob = (int64_t *)calloc((size_t)N, sizeof(int64_t));
    int64_t *nob = (int64_t *)calloc((size_t)N, sizeof(int64_t));
    for (int32_t i = 0; i < N; ++i) orc_assign_init_row(9, 0, (uint32_t)i, n, S, c->M, pop + i * ld);
    orc_eval_population_assign(n, S, c->M, c->p_u, obj, pop, N, ld, ob);
    for (uint32_t g = 1; g <= 3; ++g) {
        CHECK(orc_assign_cellular_generation(n, S, c->M, c->p_u, &prm, 0, g, rows, cols, ld, pop, ob, nxt, nob) == N);
        for (int32_t i = 0; i < N; ++i) CHECK(nob[i] <= ob[i]);
        int16_t *t = pop; pop = nxt; nxt = t;
        int64_t *u = ob; ob = nob; nob = u;
    }
    for (int32_t k = 0; k < N / 2; ++k)
        orc_assign_init_pair(9, 1, k, n, S, c->M, pop + 2 * k * ld, pop + (2 * k + 1) * ld);
    orc_eval_population_assign(n, S, c->M, c->p_u, obj, pop, N, ld, ob);
    for (uint32_t g = 1; g <= 3; ++g) {
        (void)orc_assign_pseudo_generation(n, S, c->M, c->p_u, &prm, 1, g, N, ld, pop, ob, nxt, nob);
        int16_t *t = pop; pop = nxt; nxt = t;
        int64_t *u = ob; ob = nob; nob = u;
    }
    int16_t g1[4] = { 0, 1, 2, 0 };
    orc_assign_reassign(g1, 1, 3, lcg());
    CHECK(g1[1] != 1 && g1[1] >= 0 && g1[1] < 3);
    free(pop); free(nxt); free(ob); free(nob);
}

int main(void)
{
    uint32_t ctr[4] = { 1, 2, 3, 4 }, key[2] = { 5, 6 }, out[4];
    orc_philox4x32_10(ctr, key, out);
    CHECK(orc_uniform(0xFFFFFFFFu, 7u) == 6u && orc_bernoulli(0u, 1ull) == 1);
    {
        int16_t a[6] = { 0, 1, 2, 3, 4, 5 }, b[6] = { 5, 4, 3, 2, 1, 0 }, ch[6];
        orc_order_crossover(6, a, b, 0, 5, ch);
        CHECK(is_perm(ch, 6));
        orc_order_crossover(6, a, b, 3, 3, ch);
        CHECK(is_perm(ch, 6));
        orc_two_point(6, a, b, 2, 4, ch);
        CHECK(ch[0] == 5 && ch[2] == 2 && ch[5] == 0);
    }
    const int32_t shapes[][4] = { { 1, 1, 1, 1 }, { 5, 3, 1, 3 }, { 7, 2, 8, 8 }, { 23, 5, 2, 6 }, { 40, 4, 1, 32 } };
    for (size_t k = 0; k < sizeof(shapes) / sizeof(shapes[0]); ++k) {
        case_t c = make_case(shapes[k][0], shapes[k][1], shapes[k][2], shapes[k][3]);
        const orc_objective with_obj = { c.release, c.due, 100 };
        const orc_objective rel_only = { c.release, NULL, 0 };
        run_decoders(&c, NULL);
        run_decoders(&c, &with_obj);
        run_decoders(&c, &rel_only);
        run_job_order_ga(&c, NULL);
        run_job_order_ga(&c, &with_obj);
        run_assign_ga(&c, NULL);
        run_assign_ga(&c, &with_obj);
        free_case(&c);
    }
    if (failures) {
        fprintf(stderr, "%d checks failed\n", failures);
        return 1;
    }
    printf("oracle sanitizer run ok\n");
    return 0;
}
