/*
 * Seeded synthetic-input generators for the TREES workloads.
 *
 * This module is shared by the CUDA path's tests/benchmarks and by the CPU
 * oracle's tests.  It holds none of the task-parallel method's arithmetic:
 * it only draws random numbers and lays out inputs (keys, graphs, job mixes,
 * arrival times).  Every draw comes from one counter-based generator,
 * splitmix64 (Steele, Lea and Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014): output i of the stream seeded with s is
 * mix(s + (i + 1) * 0x9E3779B97F4A7C15), where mix is the published
 * splitmix64 finaliser.  Counter-based draws make every generator
 * deterministic regardless of thread count.
 *
 * Build: gcc -O2 -fPIC -shared -fopenmp gen.c -o libtrees_gen.so -lm
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t sm64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* Output i (0-based) of the splitmix64 stream seeded with `seed`. */
uint64_t trees_gen_splitmix64(uint64_t seed, uint64_t i) {
    return sm64_mix(seed + (i + 1) * GOLDEN);
}

/* n uint32 keys: key i = high 32 bits of splitmix64(seed, i). */
void trees_gen_keys_u32(uint64_t seed, uint64_t n, uint32_t *out) {
    int64_t nn = (int64_t)n;
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nn; i++)
        out[i] = (uint32_t)(trees_gen_splitmix64(seed, (uint64_t)i) >> 32);
}

/* ------------------------------------------------------------------ R-MAT */

typedef struct {
    int32_t nv;          /* 2^scale vertices */
    int64_t m;           /* directed CSR entries after symmetrise + dedupe */
    int64_t generated;   /* edges drawn (edge_factor * 2^scale) */
    int64_t self_loops;  /* drawn edges dropped as self loops */
    int32_t *row_ptr;    /* nv + 1 */
    int32_t *col;        /* m */
} trees_gen_graph;

/* LSD radix sort of 64-bit keys that use only the low `bits` bits. */
static void radix_sort_u64(uint64_t *a, uint64_t *tmp, int64_t n, int bits) {
    const int D = 11, R = 1 << D;
    int64_t *cnt = (int64_t *)malloc(sizeof(int64_t) * R);
    for (int shift = 0; shift < bits; shift += D) {
        memset(cnt, 0, sizeof(int64_t) * R);
        for (int64_t i = 0; i < n; i++) cnt[(a[i] >> shift) & (R - 1)]++;
        int64_t s = 0;
        for (int r = 0; r < R; r++) { int64_t c = cnt[r]; cnt[r] = s; s += c; }
        for (int64_t i = 0; i < n; i++) tmp[cnt[(a[i] >> shift) & (R - 1)]++] = a[i];
        uint64_t *t = a; a = tmp; tmp = t;
    }
    /* an odd number of passes leaves the result in the scratch array */
    int passes = (bits + D - 1) / D;
    if (passes & 1) memcpy(tmp, a, sizeof(uint64_t) * (size_t)n);
    free(cnt);
}

/*
 * R-MAT graph (Chakrabarti, Zhan, Faloutsos 2004): each of edge_factor*2^scale
 * edges descends `scale` levels of the adjacency matrix, choosing quadrant
 * (0,0),(0,1),(1,0),(1,1) with probabilities a, b, c, 1-a-b-c.  Level l uses a
 * 32-bit uniform: the high (l even) or low (l odd) half of splitmix64(seed,
 * e*ceil(scale/2) + l/2).  No noise and no vertex permutation.  Self loops are
 * dropped, every edge is stored in both directions, rows are sorted and
 * duplicates removed.  Output: int32 CSR.  Returns 0 on success.
 */
int trees_gen_rmat(int scale, int edge_factor, double a, double b, double c,
                   uint64_t seed, trees_gen_graph *g) {
    if (scale < 1 || scale > 30 || edge_factor < 1) return -1;
    const int64_t nv = (int64_t)1 << scale;
    const int64_t E = (int64_t)edge_factor * nv;
    const int draws = (scale + 1) / 2;
    const double two32 = 4294967296.0;
    const uint64_t ta = (uint64_t)(a * two32);
    const uint64_t tab = (uint64_t)((a + b) * two32);
    const uint64_t tabc = (uint64_t)((a + b + c) * two32);
    uint64_t *pairs = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(2 * E));
    uint8_t *keep = (uint8_t *)malloc((size_t)E);
    if (!pairs || !keep) { free(pairs); free(keep); return -2; }
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < E; e++) {
        uint64_t src = 0, dst = 0, r = 0;
        for (int l = 0; l < scale; l++) {
            if ((l & 1) == 0) r = trees_gen_splitmix64(seed, (uint64_t)e * draws + (l >> 1));
            uint64_t u = (l & 1) ? (r & 0xFFFFFFFFULL) : (r >> 32);
            uint64_t sb, db;
            if (u < ta) { sb = 0; db = 0; }
            else if (u < tab) { sb = 0; db = 1; }
            else if (u < tabc) { sb = 1; db = 0; }
            else { sb = 1; db = 1; }
            src = (src << 1) | sb;
            dst = (dst << 1) | db;
        }
        keep[e] = (src != dst);
        pairs[2 * e] = (src << scale) | dst;
        pairs[2 * e + 1] = (dst << scale) | src;
    }
    /* compact away self loops (both copies) */
    int64_t n = 0, loops = 0;
    for (int64_t e = 0; e < E; e++) {
        if (keep[e]) { pairs[n++] = pairs[2 * e]; pairs[n++] = pairs[2 * e + 1]; }
        else loops++;
    }
    free(keep);
    uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(n > 0 ? n : 1));
    if (!tmp) { free(pairs); return -2; }
    radix_sort_u64(pairs, tmp, n, 2 * scale);
    free(tmp);
    int64_t m = 0;
    for (int64_t i = 0; i < n; i++)
        if (m == 0 || pairs[i] != pairs[m - 1]) pairs[m++] = pairs[i];
    if (m > INT32_MAX) { free(pairs); return -3; }
    g->nv = (int32_t)nv;
    g->m = m;
    g->generated = E;
    g->self_loops = loops;
    g->row_ptr = (int32_t *)calloc((size_t)nv + 1, sizeof(int32_t));
    g->col = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m > 0 ? m : 1));
    if (!g->row_ptr || !g->col) { free(pairs); return -2; }
    const uint64_t mask = ((uint64_t)1 << scale) - 1;
    for (int64_t i = 0; i < m; i++) {
        g->row_ptr[(pairs[i] >> scale) + 1]++;
        g->col[i] = (int32_t)(pairs[i] & mask);
    }
    for (int64_t v = 0; v < nv; v++) g->row_ptr[v + 1] += g->row_ptr[v];
    free(pairs);
    return 0;
}

void trees_gen_graph_free(trees_gen_graph *g) {
    free(g->row_ptr);
    free(g->col);
    g->row_ptr = NULL;
    g->col = NULL;
}

/* ---------------------------------------------------------- job mixes */

/*
 * njobs independent jobs.  Job i draws r0 = splitmix64(seed, 2i) and
 * r1 = splitmix64(seed, 2i+1): kind = r0 mod 3 (0 fib, 1 mergesort,
 * 2 N-Queens); fib n = 10 + r1 mod 21; N-Queens n = 6 + r1 mod 6;
 * mergesort size = floor(2^(10 + 12u)), u = (r1 >> 11) * 2^-53 (log-uniform
 * in [2^10, 2^22)).  key_seed[i] seeds that job's keys (trees_gen_keys_u32).
 */
void trees_gen_jobs(uint64_t seed, int64_t njobs, int32_t *kind, int64_t *param,
                    uint64_t *key_seed) {
    for (int64_t i = 0; i < njobs; i++) {
        uint64_t r0 = trees_gen_splitmix64(seed, 2 * (uint64_t)i);
        uint64_t r1 = trees_gen_splitmix64(seed, 2 * (uint64_t)i + 1);
        int32_t k = (int32_t)(r0 % 3);
        kind[i] = k;
        if (k == 0) param[i] = 10 + (int64_t)(r1 % 21);
        else if (k == 2) param[i] = 6 + (int64_t)(r1 % 6);
        else {
            double u = (double)(r1 >> 11) * (1.0 / 9007199254740992.0);
            int64_t sz = (int64_t)floor(exp2(10.0 + 12.0 * u));
            if (sz < 1024) sz = 1024;
            if (sz > (1 << 22)) sz = 1 << 22;
            param[i] = sz;
        }
        key_seed[i] = trees_gen_splitmix64(seed ^ 0xA5A5A5A5A5A5A5A5ULL, (uint64_t)i);
    }
}

/* Poisson arrivals: n arrival times in seconds at `rate` per second,
 * inter-arrival -ln(1-u)/rate with u = (splitmix64(seed,i) >> 11) * 2^-53. */
void trees_gen_poisson_arrivals(uint64_t seed, int64_t n, double rate, double *t_out) {
    double t = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double u = (double)(trees_gen_splitmix64(seed, (uint64_t)i) >> 11) * (1.0 / 9007199254740992.0);
        t += -log1p(-u) / rate;
        t_out[i] = t;
    }
}

/* ------------------------------------------------------ binary trees */

/*
 * A random binary tree of nnodes nodes for the traversal programs: node 0 is
 * the root; node i > 0 attaches to a uniformly drawn earlier node's free child
 * slot (splitmix64(seed, i)), retrying the next node in index order when both
 * slots are taken.  left/right hold child ids or -1 (nil).
 */
void trees_gen_binary_tree(uint64_t seed, int32_t nnodes, int32_t *left, int32_t *right) {
    for (int32_t i = 0; i < nnodes; i++) { left[i] = -1; right[i] = -1; }
    for (int32_t i = 1; i < nnodes; i++) {
        uint64_t r = trees_gen_splitmix64(seed, (uint64_t)i);
        int32_t p = (int32_t)(r % (uint64_t)i);
        int side = (int)((r >> 40) & 1);
        for (;;) {
            if (side == 0 && left[p] < 0) { left[p] = i; break; }
            if (side == 1 && right[p] < 0) { right[p] = i; break; }
            if (left[p] < 0) { left[p] = i; break; }
            if (right[p] < 0) { right[p] = i; break; }
            p = (p + 1) % i;
        }
    }
}

/* Edge weights for a CSR graph, aligned with col: the weight of edge (v, u)
 * is 1 + splitmix64(seed, min(v,u) * 2^32 + max(v,u)) mod wmax, so both
 * directions of an undirected edge weigh the same.  wmax >= 1. */
void trees_gen_weights(uint64_t seed, int32_t nv, const int32_t *row_ptr, const int32_t *col, uint32_t wmax,
                       uint32_t *out) {
    for (int32_t v = 0; v < nv; v++) {
        for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; e++) {
            const uint64_t u = (uint64_t)(uint32_t)col[e], w = (uint64_t)(uint32_t)v;
            const uint64_t lo = u < w ? u : w, hi = u < w ? w : u;
            out[e] = 1u + (uint32_t)(trees_gen_splitmix64(seed, (lo << 32) | hi) % wmax);
        }
    }
}

/* n complex points as interleaved (re, im) floats: component c (0 = re,
 * 1 = im) of point i is ((splitmix64(seed, 2i + c) >> 40) - 2^23) / 2^23,
 * uniform on [-1, 1) with 24-bit resolution, so exactly a float. */
void trees_gen_signal(uint64_t seed, uint64_t n, float *out) {
    int64_t nn = (int64_t)(2 * n);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < nn; i++)
        out[i] = (float)((int64_t)(trees_gen_splitmix64(seed, (uint64_t)i) >> 40) - (1LL << 23)) *
                 (1.0f / 8388608.0f);
}
