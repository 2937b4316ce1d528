/*
 * CPU oracle for the TREES epoch step (Hechtman, Hilton, Sorin, "TREES: A
 * CPU/GPU Task-Parallel Runtime with Explicit Epoch Synchronization").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the tests, the smoke check and the benchmark's CPU
 * baseline do.  It shares no code, header, table or constant with the CUDA
 * path.  Everything here is plain, sequential and slow on purpose.
 *
 * Two parts:
 *  1. Plain definitions of what each task program computes (the method
 *     reaches these exactly, or up to rounding for the FFT): recursive
 *     Fibonacci with call counts, top-down mergesort, FIFO-queue BFS,
 *     backtracking N-Queens, Dijkstra, the discrete Fourier transform.
 *  2. A sequential Task Vector Machine simulator that runs the same programs
 *     as fork/join/emit/map tasks, one epoch at a time, in the order the paper
 *     gives: Phase 1 pops the epoch number and NDRange (Sec. 4.3.1, 5.2.2),
 *     Phase 2 runs every entry of the range whose encoded epoch matches the
 *     current one (Sec. 4.3.2, 5.2.3, footnote 2 of Sec. 5.1.2), Phase 3
 *     pushes the join range and then the fork range and runs the scheduled
 *     maps (Sec. 4.3.3, 5.2.4), and an epoch that neither forks nor joins
 *     gives its entries back by lowering nextFreeCore (Sec. 5.3).  It records
 *     a per-epoch trace (epoch number, range, valid tasks, forks, join flag,
 *     maps) that the GPU scheduler must reproduce count for count.
 *
 * Build: gcc -O2 -fPIC -shared oracle.c -o liboracle.so
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ================================================================ part 1 */

/* Fibonacci by its definition f(n) = f(n-1) + f(n-2), f(0)=0, f(1)=1
 * (Sec. 6.2 uses the naive recursive algorithm).  *calls counts every call. */
static uint64_t fib_rec(uint32_t n, uint64_t *calls) {
    (*calls)++;
    if (n < 2) return n;
    return fib_rec(n - 1, calls) + fib_rec(n - 2, calls);
}

uint64_t oracle_fib(uint32_t n, uint64_t *calls) {
    uint64_t c = 0;
    uint64_t v = fib_rec(n, &c);
    if (calls) *calls = c;
    return v;
}

/* Task counts of the fib task tree when a call with n <= cutoff (or n < 2)
 * is a leaf computed inside its task: every non-leaf call is one fib task
 * plus one join (sum) task. */
static void fib_tree(uint32_t n, uint32_t cutoff, uint64_t *tasks, uint64_t *joins) {
    (*tasks)++;
    if (n < 2 || n <= cutoff) return;
    (*joins)++;
    fib_tree(n - 1, cutoff, tasks, joins);
    fib_tree(n - 2, cutoff, tasks, joins);
}

void oracle_fib_task_counts(uint32_t n, uint32_t cutoff, uint64_t *fib_tasks, uint64_t *join_tasks) {
    uint64_t t = 0, j = 0;
    fib_tree(n, cutoff, &t, &j);
    *fib_tasks = t;
    *join_tasks = j;
}

/* Top-down mergesort (Sec. 6.4): a range of at most `leaf` keys is sorted
 * directly (insertion sort); a longer range splits at lo + (hi-lo)/2, both
 * halves are sorted, then merged taking from the left half on ties. */
static void ms_rec(uint32_t *k, uint32_t *tmp, int64_t lo, int64_t hi, int64_t leaf) {
    if (hi - lo <= leaf) {
        for (int64_t i = lo + 1; i < hi; i++) {
            uint32_t x = k[i];
            int64_t j = i - 1;
            while (j >= lo && k[j] > x) { k[j + 1] = k[j]; j--; }
            k[j + 1] = x;
        }
        return;
    }
    int64_t mid = lo + (hi - lo) / 2;
    ms_rec(k, tmp, lo, mid, leaf);
    ms_rec(k, tmp, mid, hi, leaf);
    int64_t i = lo, j = mid, o = lo;
    while (i < mid && j < hi) tmp[o++] = (k[j] < k[i]) ? k[j++] : k[i++];
    while (i < mid) tmp[o++] = k[i++];
    while (j < hi) tmp[o++] = k[j++];
    memcpy(k + lo, tmp + lo, sizeof(uint32_t) * (size_t)(hi - lo));
}

int oracle_mergesort_u32(uint32_t *keys, int64_t n, int64_t leaf) {
    if (n <= 0) return 0;
    if (leaf < 1) return -1;
    uint32_t *tmp = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)n);
    if (!tmp) return -2;
    ms_rec(keys, tmp, 0, n, leaf);
    free(tmp);
    return 0;
}

/* Breadth-first search with a FIFO queue: level[v] = hop distance from src,
 * -1 if unreachable.  Returns the number of reached vertices. */
int64_t oracle_bfs(int32_t nv, const int32_t *row_ptr, const int32_t *col, int32_t src, int32_t *level) {
    for (int32_t v = 0; v < nv; v++) level[v] = -1;
    if (src < 0 || src >= nv) return 0;
    int32_t *q = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
    if (!q) return -2;
    int64_t head = 0, tail = 0;
    level[src] = 0;
    q[tail++] = src;
    while (head < tail) {
        int32_t v = q[head++];
        for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; e++) {
            int32_t u = col[e];
            if (level[u] < 0) { level[u] = level[v] + 1; q[tail++] = u; }
        }
    }
    free(q);
    return tail;
}

/* Single-source shortest paths, Dijkstra's algorithm with a binary heap and
 * lazy deletion: the plain definition of the distances the SSSP program of
 * Sec. 6.3 reaches.  Non-negative u32 edge weights aligned with col; dist[v]
 * = length of a shortest path from src, UINT64_MAX if unreachable.  Returns
 * the number of reached vertices (-2: out of memory). */
typedef struct { uint64_t d; int32_t v; } heap_item;

static void heap_push(heap_item *h, int64_t *n, heap_item x) {
    int64_t i = (*n)++;
    while (i > 0) {
        const int64_t p = (i - 1) / 2;
        if (h[p].d <= x.d) break;
        h[i] = h[p];
        i = p;
    }
    h[i] = x;
}

static heap_item heap_pop(heap_item *h, int64_t *n) {
    const heap_item top = h[0], x = h[--(*n)];
    int64_t i = 0;
    for (;;) {
        int64_t c = 2 * i + 1;
        if (c >= *n) break;
        if (c + 1 < *n && h[c + 1].d < h[c].d) c++;
        if (x.d <= h[c].d) break;
        h[i] = h[c];
        i = c;
    }
    if (*n > 0) h[i] = x;
    return top;
}

int64_t oracle_sssp_dijkstra(int32_t nv, const int32_t *row_ptr, const int32_t *col, const uint32_t *weight,
                             int32_t src, uint64_t *dist) {
    for (int32_t v = 0; v < nv; v++) dist[v] = UINT64_MAX;
    if (src < 0 || src >= nv) return 0;
    const int64_t m = row_ptr[nv];
    heap_item *h = (heap_item *)malloc(sizeof(heap_item) * (size_t)(m + 1));
    uint8_t *done = (uint8_t *)calloc((size_t)nv, 1);
    if (!h || !done) { free(h); free(done); return -2; }
    int64_t hn = 0, reached = 0;
    dist[src] = 0;
    heap_push(h, &hn, (heap_item){0, src});
    while (hn > 0) {
        const heap_item it = heap_pop(h, &hn);
        if (done[it.v]) continue;  /* a stale entry: the vertex was settled by a shorter one */
        done[it.v] = 1;
        reached++;
        for (int32_t e = row_ptr[it.v]; e < row_ptr[it.v + 1]; e++) {
            const int32_t u = col[e];
            const uint64_t nd = it.d + weight[e];
            if (nd < dist[u]) { dist[u] = nd; heap_push(h, &hn, (heap_item){nd, u}); }
        }
    }
    free(h);
    free(done);
    return reached;
}

/* The worklist relaxation of Sec. 6.3, run sequentially: every vertex of the
 * input worklist relaxes all its out-edges (dist[u] = min(dist[u], dist[v] +
 * w)); a vertex whose distance dropped is appended to the output worklist
 * once per round; the lists swap until a round explores nothing.  Reaches
 * the same distances as Dijkstra.  *rounds and *relaxed receive the number of
 * rounds and of vertex relaxations.  Returns 0 (-2: out of memory). */
int oracle_sssp_worklist(int32_t nv, const int32_t *row_ptr, const int32_t *col, const uint32_t *weight,
                         int32_t src, uint64_t *dist, uint64_t *rounds, uint64_t *relaxed) {
    *rounds = 0;
    *relaxed = 0;
    for (int32_t v = 0; v < nv; v++) dist[v] = UINT64_MAX;
    if (src < 0 || src >= nv) return 0;
    int32_t *in = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
    int32_t *out = (int32_t *)malloc(sizeof(int32_t) * (size_t)nv);
    int64_t *queued = (int64_t *)malloc(sizeof(int64_t) * (size_t)nv);
    if (!in || !out || !queued) { free(in); free(out); free(queued); return -2; }
    for (int32_t v = 0; v < nv; v++) queued[v] = -1;
    int64_t nin = 0;
    dist[src] = 0;
    in[nin++] = src;
    while (nin > 0) {
        const int64_t r = (int64_t)(*rounds)++;
        int64_t nout = 0;
        for (int64_t i = 0; i < nin; i++) {
            const int32_t v = in[i];
            (*relaxed)++;
            for (int32_t e = row_ptr[v]; e < row_ptr[v + 1]; e++) {
                const int32_t u = col[e];
                const uint64_t nd = dist[v] + weight[e];
                if (nd < dist[u]) {
                    dist[u] = nd;
                    if (queued[u] != r) { queued[u] = r; out[nout++] = u; }
                }
            }
        }
        int32_t *t = in; in = out; out = t;
        nin = nout;
    }
    free(in);
    free(out);
    free(queued);
    return 0;
}

/* N-Queens by backtracking over rows with explicit used-column and
 * used-diagonal arrays.  Counts solutions, the nodes of the backtracking tree
 * (every consistent partial placement, root included: one row task each) and
 * the nodes that have at least one safe child (one join task each). */
typedef struct { int n; uint8_t col[32], dg1[64], dg2[64]; uint64_t nodes, internal; } nq_state;

static uint64_t nq_rec(nq_state *s, int r) {
    s->nodes++;
    if (r == s->n) return 1;
    uint64_t sum = 0;
    int any = 0;
    for (int c = 0; c < s->n; c++) {
        int a = r + c, b = r - c + s->n - 1;
        if (s->col[c] || s->dg1[a] || s->dg2[b]) continue;
        any = 1;
        s->col[c] = s->dg1[a] = s->dg2[b] = 1;
        sum += nq_rec(s, r + 1);
        s->col[c] = s->dg1[a] = s->dg2[b] = 0;
    }
    if (any) s->internal++;
    return sum;
}

uint64_t oracle_nqueens(int n, uint64_t *row_tasks, uint64_t *join_tasks) {
    nq_state s;
    memset(&s, 0, sizeof s);
    if (n < 1 || n > 16) return 0;
    s.n = n;
    uint64_t v = nq_rec(&s, 0);
    if (row_tasks) *row_tasks = s.nodes;
    if (join_tasks) *join_tasks = s.internal;
    return v;
}

/* The discrete Fourier transform by its definition (the FFT of Sec. 6.2
 * computes it):  X[k] = sum_{j<n} x[j] * exp(-2*pi*i*j*k/n),  k < n,
 * complex numbers stored as interleaved (re, im) doubles.  The angle is taken
 * from (j*k mod n), which keeps it in [0, 2*pi) without changing its value.
 * O(n^2); any n >= 1 (not only powers of two). */
static void dft_term(int64_t n, const double *x, int64_t j, int64_t k, double *re, double *im) {
    const double ang = -2.0 * M_PI * (double)((j * k) % n) / (double)n;
    const double c = cos(ang), sn = sin(ang);
    *re += x[2 * j] * c - x[2 * j + 1] * sn;
    *im += x[2 * j] * sn + x[2 * j + 1] * c;
}

void oracle_dft_at(int64_t n, const double *x, int64_t k, double *out) {
    double re = 0.0, im = 0.0;
    for (int64_t j = 0; j < n; j++) dft_term(n, x, j, k, &re, &im);
    out[0] = re;
    out[1] = im;
}

void oracle_dft(int64_t n, const double *x, double *X) {
    for (int64_t k = 0; k < n; k++) oracle_dft_at(n, x, k, X + 2 * k);
}

/* ================================================================ part 2 */

enum {
    T_FIB = 1, T_FIB_SUM, T_MS_SPLIT, T_MS_MERGE, T_NQ_ROW, T_NQ_SUM,
    T_BFS_VISIT, T_PO, T_PO_AFTER, T_PRE, T_FFT, T_FFT_COMBINE,
    NUM_TASK_TYPES = T_FFT_COMBINE
};

enum { ORACLE_FIB = 0, ORACLE_MERGESORT = 1, ORACLE_BFS = 2, ORACLE_NQUEENS = 3,
       ORACLE_POSTORDER = 4, ORACLE_PREORDER = 5, ORACLE_FFT = 6 };

enum { MAP_LEAF_SORT = 1, MAP_MERGE = 2, MAP_FFT_COMBINE = 3 };

typedef struct {
    uint32_t cen, lo, hi;   /* epoch number and NDRange [lo, hi) */
    uint32_t valid;         /* entries whose encoded epoch matched */
    uint32_t forks;         /* nextFreeCore - oldNextFreeCore */
    uint32_t joined;        /* joinScheduled */
    uint32_t maps;          /* map operations scheduled */
} oracle_epoch_t;

typedef struct {
    int program;
    uint32_t fib_n, fib_cutoff;
    uint32_t *keys; int64_t nkeys; int64_t leaf;
    int32_t nv; const int32_t *row_ptr; const int32_t *col; int32_t *level; int32_t src;
    int32_t nq_n;
    int32_t nnodes; const int32_t *left; const int32_t *right; int32_t *visit_epoch;
    uint64_t max_epochs;
    /* FFT: n points (a power of two), leaf size, largest combine run inside its
     * task (larger ones are maps), input and output as interleaved (re, im) */
    int64_t fft_n, fft_leaf, fft_cutoff;
    const double *fft_x; double *fft_X;
} oracle_tvm_params;

typedef struct {
    uint64_t epochs, tasks, forks, joins, maps, peak_slots, root_result;
    uint64_t final_slots;   /* nextFreeCore at halt: 0 when the TV emptied (Sec. 5.3) */
    int32_t err;
} oracle_tvm_stats;

typedef struct { uint32_t cen, lo, hi; } range_t;
typedef struct { int kind; int64_t a, b, c; } map_op;

typedef struct {
    /* Task Vector: one entry per abstract core (Sec. 4, 5.1.2) */
    uint32_t *code, *arg0, *arg1, *link;
    uint64_t *result;
    uint64_t cap;
    uint64_t next;                 /* nextFreeCore */
    range_t *stk; uint64_t sp, stk_cap;    /* join stack + NDRange stack */
    map_op *maps; uint64_t nmaps, maps_cap;
    uint32_t cen; uint64_t epoch_index;
    int join_scheduled, map_scheduled;
    uint64_t n_forks, n_joins, n_maps;
    const oracle_tvm_params *p;
    uint32_t *tmp;                 /* merge scratch */
    int err;
} tvm;

static int tvm_grow(tvm *m, uint64_t need) {
    if (need <= m->cap) return 0;
    uint64_t nc = m->cap ? m->cap : 1024;
    while (nc < need) nc *= 2;
    uint32_t *a = realloc(m->code, nc * 4), *b = a ? realloc(m->arg0, nc * 4) : NULL;
    if (a) m->code = a;
    if (b) m->arg0 = b;
    uint32_t *c = b ? realloc(m->arg1, nc * 4) : NULL;
    if (c) m->arg1 = c;
    uint32_t *d = c ? realloc(m->link, nc * 4) : NULL;
    if (d) m->link = d;
    uint64_t *e = d ? realloc(m->result, nc * 8) : NULL;
    if (e) m->result = e;
    if (!e) return -1;
    m->cap = nc;
    return 0;
}

static void push(tvm *m, uint32_t cen, uint32_t lo, uint32_t hi) {
    if (m->sp == m->stk_cap) {
        m->stk_cap = m->stk_cap ? 2 * m->stk_cap : 64;
        m->stk = realloc(m->stk, m->stk_cap * sizeof(range_t));
    }
    m->stk[m->sp].cen = cen; m->stk[m->sp].lo = lo; m->stk[m->sp].hi = hi;
    m->sp++;
}

/* --- the four primitives (Sec. 4.3.2) --- */

/* fork f(a0,a1): take entry nextFreeCore, write it for epoch CEN+1 */
static uint32_t prim_fork(tvm *m, uint32_t type, uint32_t a0, uint32_t a1) {
    if (tvm_grow(m, m->next + 1)) { m->err = 1; return 0; }
    uint64_t s = m->next++;
    m->code[s] = (m->cen + 1) * NUM_TASK_TYPES + type;
    m->arg0[s] = a0;
    m->arg1[s] = a1;
    m->link[s] = 0;
    m->n_forks++;
    return (uint32_t)s;
}

/* join f(a0,a1): replace own entry with f, to run in this same epoch number
 * once everything forked above it has finished; link = first child */
static void prim_join(tvm *m, uint32_t self, uint32_t type, uint32_t a0, uint32_t a1, uint32_t link) {
    m->code[self] = m->cen * NUM_TASK_TYPES + type;
    m->arg0[self] = a0;
    m->arg1[self] = a1;
    m->link[self] = link;
    m->join_scheduled = 1;
    m->n_joins++;
}

/* emit v: store the value in the task's own entry and retire the entry */
static void prim_emit(tvm *m, uint32_t self, uint64_t v) {
    m->result[self] = v;
    m->code[self] = 0;
}

/* map f(args): a data-parallel operation run before the next epoch */
static void prim_map(tvm *m, int kind, int64_t a, int64_t b, int64_t c) {
    if (m->nmaps == m->maps_cap) {
        m->maps_cap = m->maps_cap ? 2 * m->maps_cap : 256;
        m->maps = realloc(m->maps, m->maps_cap * sizeof(map_op));
    }
    m->maps[m->nmaps].kind = kind;
    m->maps[m->nmaps].a = a; m->maps[m->nmaps].b = b; m->maps[m->nmaps].c = c;
    m->nmaps++;
    m->map_scheduled = 1;
    m->n_maps++;
}

/* --- the FFT program (Sec. 6.2): radix-2 Cooley-Tukey by decimation in time.
 * Task FFT(o, d) transforms the N >> d points x[o], x[o + 2^d], x[o + 2*2^d],
 * ... (the points whose index is o modulo 2^d).  It forks FFT(o, d+1) (the
 * even-numbered of its points) and FFT(o + 2^d, d+1) (the odd-numbered) and
 * joins into COMBINE(o, d), which merges their two half-size transforms into
 * its own.  The transform of the even half occupies the first half of the
 * parent's output block and the odd half the second, so the block of FFT(o, d)
 * starts at the sum, over the bits b < d set in o, of N >> (b + 1). */
static int64_t fft_block(uint32_t o, uint32_t d, int64_t N) {
    int64_t pos = 0;
    for (uint32_t b = 0; b < d; b++)
        if ((o >> b) & 1u) pos += N >> (b + 1);
    return pos;
}

/* A leaf: the n-point DFT of its points by the definition, into its block. */
static void fft_leaf(const oracle_tvm_params *p, uint32_t o, uint32_t d, int64_t n) {
    const int64_t dst = fft_block(o, d, p->fft_n);
    for (int64_t k = 0; k < n; k++) {
        double re = 0.0, im = 0.0;
        for (int64_t j = 0; j < n; j++) {
            const int64_t src = (int64_t)o + (j << d);
            const double ang = -2.0 * M_PI * (double)((j * k) % n) / (double)n;
            re += p->fft_x[2 * src] * cos(ang) - p->fft_x[2 * src + 1] * sin(ang);
            im += p->fft_x[2 * src] * sin(ang) + p->fft_x[2 * src + 1] * cos(ang);
        }
        p->fft_X[2 * (dst + k)] = re;
        p->fft_X[2 * (dst + k) + 1] = im;
    }
}

/* The combine of a block of n points at X[dst..dst+n): its first half holds
 * E, the transform of the even points, its second half O, that of the odd
 * points; with w = exp(-2*pi*i*k/n), X[k] = E[k] + w O[k] and
 * X[k + n/2] = E[k] - w O[k] for k < n/2. */
static void fft_combine(double *X, int64_t dst, int64_t n) {
    for (int64_t k = 0; k < n / 2; k++) {
        const double ang = -2.0 * M_PI * (double)k / (double)n, wr = cos(ang), wi = sin(ang);
        double *e = X + 2 * (dst + k), *od = X + 2 * (dst + k + n / 2);
        const double tr = wr * od[0] - wi * od[1], ti = wr * od[1] + wi * od[0];
        const double er = e[0], ei = e[1];
        e[0] = er + tr;
        e[1] = ei + ti;
        od[0] = er - tr;
        od[1] = ei - ti;
    }
}

static void run_map(tvm *m, const map_op *op) {
    uint32_t *k = m->p->keys;
    if (op->kind == MAP_LEAF_SORT) {
        for (int64_t i = op->a + 1; i < op->b; i++) {
            uint32_t x = k[i];
            int64_t j = i - 1;
            while (j >= op->a && k[j] > x) { k[j + 1] = k[j]; j--; }
            k[j + 1] = x;
        }
    } else if (op->kind == MAP_MERGE) {
        int64_t i = op->a, j = op->b, o = op->a;
        while (i < op->b && j < op->c) m->tmp[o++] = (k[j] < k[i]) ? k[j++] : k[i++];
        while (i < op->b) m->tmp[o++] = k[i++];
        while (j < op->c) m->tmp[o++] = k[j++];
        memcpy(k + op->a, m->tmp + op->a, sizeof(uint32_t) * (size_t)(op->c - op->a));
    } else if (op->kind == MAP_FFT_COMBINE) {
        fft_combine(m->p->fft_X, op->a, op->b);
    }
}

/* --- task programs, written as tasks with the four primitives --- */

static uint64_t fib_plain(uint32_t n) { return n < 2 ? n : fib_plain(n - 1) + fib_plain(n - 2); }

static uint32_t nq_free(uint32_t a0, uint32_t a1, int n) {
    uint32_t cols = a0 & 0xFFFF, d1 = a1 & 0xFFFF, d2 = a1 >> 16;
    return ~(cols | d1 | d2) & ((1u << n) - 1u);
}

static void run_task(tvm *m, uint32_t s, uint32_t type) {
    const oracle_tvm_params *p = m->p;
    uint32_t a0 = m->arg0[s], a1 = m->arg1[s];
    switch (type) {
    case T_FIB: {
        uint32_t n = a0;
        if (n < 2 || n <= p->fib_cutoff) { prim_emit(m, s, fib_plain(n)); break; }
        uint32_t first = prim_fork(m, T_FIB, n - 1, 0);
        prim_fork(m, T_FIB, n - 2, 0);
        prim_join(m, s, T_FIB_SUM, n, 0, first);
        break;
    }
    case T_FIB_SUM:
        prim_emit(m, s, m->result[m->link[s]] + m->result[m->link[s] + 1]);
        break;
    case T_MS_SPLIT: {
        int64_t lo = a0, hi = a1;
        if (hi - lo <= p->leaf) {
            if (hi > lo) prim_map(m, MAP_LEAF_SORT, lo, hi, 0);
            prim_emit(m, s, 0);
            break;
        }
        int64_t mid = lo + (hi - lo) / 2;
        uint32_t first = prim_fork(m, T_MS_SPLIT, (uint32_t)lo, (uint32_t)mid);
        prim_fork(m, T_MS_SPLIT, (uint32_t)mid, (uint32_t)hi);
        prim_join(m, s, T_MS_MERGE, a0, a1, first);
        break;
    }
    case T_MS_MERGE: {
        int64_t lo = a0, hi = a1, mid = lo + (hi - lo) / 2;
        prim_map(m, MAP_MERGE, lo, mid, hi);
        prim_emit(m, s, 0);
        break;
    }
    case T_NQ_ROW: {
        int n = p->nq_n;
        uint32_t r = a0 >> 16, cols = a0 & 0xFFFF, d1 = a1 & 0xFFFF, d2 = a1 >> 16;
        uint32_t mask = (1u << n) - 1u;
        if ((int)r == n) { prim_emit(m, s, 1); break; }
        uint32_t fr = nq_free(a0, a1, n);
        if (fr == 0) { prim_emit(m, s, 0); break; }
        uint32_t first = 0;
        int k = 0;
        for (int c = 0; c < n; c++) {
            uint32_t b = 1u << c;
            if (!(fr & b)) continue;
            uint32_t nc = cols | b, nd1 = ((d1 | b) << 1) & mask, nd2 = (d2 | b) >> 1;
            uint32_t slot = prim_fork(m, T_NQ_ROW, nc | ((r + 1) << 16), nd1 | (nd2 << 16));
            if (k++ == 0) first = slot;
        }
        prim_join(m, s, T_NQ_SUM, a0, a1, first);
        break;
    }
    case T_NQ_SUM: {
        uint32_t fr = nq_free(a0, a1, p->nq_n);
        uint64_t sum = 0;
        int k = 0;
        for (uint32_t x = fr; x; x &= x - 1) k++;
        for (int i = 0; i < k; i++) sum += m->result[m->link[s] + i];
        prim_emit(m, s, sum);
        break;
    }
    case T_BFS_VISIT: {
        int32_t v = (int32_t)a0;
        for (int32_t e = p->row_ptr[v]; e < p->row_ptr[v + 1]; e++) {
            int32_t u = p->col[e];
            if (p->level[u] < 0) {
                p->level[u] = (int32_t)(m->cen + 1);
                prim_fork(m, T_BFS_VISIT, (uint32_t)u, 0);
            }
        }
        prim_emit(m, s, 0);
        break;
    }
    case T_PO: {
        int32_t node = (int32_t)a0;
        if (node < 0) { prim_emit(m, s, 0); break; }
        uint32_t first = prim_fork(m, T_PO, (uint32_t)p->right[node], 0);
        prim_fork(m, T_PO, (uint32_t)p->left[node], 0);
        prim_join(m, s, T_PO_AFTER, a0, 0, first);
        break;
    }
    case T_PO_AFTER:
        p->visit_epoch[(int32_t)a0] = (int32_t)m->epoch_index;
        prim_emit(m, s, 0);
        break;
    case T_PRE: {
        int32_t node = (int32_t)a0;
        if (node < 0) { prim_emit(m, s, 0); break; }
        p->visit_epoch[node] = (int32_t)m->epoch_index;
        prim_fork(m, T_PRE, (uint32_t)p->right[node], 0);
        prim_fork(m, T_PRE, (uint32_t)p->left[node], 0);
        prim_emit(m, s, 0);
        break;
    }
    case T_FFT: {
        const int64_t n = p->fft_n >> a1;
        if (n <= p->fft_leaf) {
            fft_leaf(p, a0, a1, n);
            prim_emit(m, s, 0);
            break;
        }
        uint32_t first = prim_fork(m, T_FFT, a0, a1 + 1);   /* even-numbered points */
        prim_fork(m, T_FFT, a0 + (1u << a1), a1 + 1);       /* odd-numbered points */
        prim_join(m, s, T_FFT_COMBINE, a0, a1, first);
        break;
    }
    case T_FFT_COMBINE: {
        const int64_t n = p->fft_n >> a1, dst = fft_block(a0, a1, p->fft_n);
        if (n <= p->fft_cutoff) fft_combine(p->fft_X, dst, n);
        else prim_map(m, MAP_FFT_COMBINE, dst, n, 0);
        prim_emit(m, s, 0);
        break;
    }
    default:
        m->err = 2;
    }
}

/* Runs one program to completion.  Returns 0, or nonzero on error
 * (1 out of memory, 2 bad task, 3 epoch limit, 4 bad arguments,
 * 5 a reclaim found nextFreeCore away from the range end). */
int oracle_tvm_run(const oracle_tvm_params *p, oracle_epoch_t *trace, uint64_t trace_cap,
                   oracle_tvm_stats *st) {
    tvm m;
    memset(&m, 0, sizeof m);
    m.p = p;
    memset(st, 0, sizeof *st);
    uint32_t root_type, r0 = 0, r1 = 0;
    switch (p->program) {
    case ORACLE_FIB: root_type = T_FIB; r0 = p->fib_n; break;
    case ORACLE_MERGESORT:
        if (p->nkeys < 0 || p->nkeys > 0xFFFFFFFFLL || p->leaf < 1) return 4;
        root_type = T_MS_SPLIT; r0 = 0; r1 = (uint32_t)p->nkeys;
        m.tmp = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(p->nkeys > 0 ? p->nkeys : 1));
        break;
    case ORACLE_BFS:
        if (p->src < 0 || p->src >= p->nv) return 4;
        for (int32_t v = 0; v < p->nv; v++) p->level[v] = -1;
        p->level[p->src] = 0;
        root_type = T_BFS_VISIT; r0 = (uint32_t)p->src; break;
    case ORACLE_NQUEENS:
        if (p->nq_n < 1 || p->nq_n > 16) return 4;
        root_type = T_NQ_ROW; break;
    case ORACLE_POSTORDER: case ORACLE_PREORDER:
        for (int32_t v = 0; v < p->nnodes; v++) p->visit_epoch[v] = -1;
        root_type = p->program == ORACLE_POSTORDER ? T_PO : T_PRE;
        r0 = p->nnodes > 0 ? 0u : 0xFFFFFFFFu; break;
    case ORACLE_FFT:
        if (p->fft_n < 1 || (p->fft_n & (p->fft_n - 1)) || p->fft_n > (1LL << 30) || p->fft_leaf < 1 ||
            !p->fft_x || !p->fft_X)
            return 4;
        root_type = T_FFT; r0 = 0; r1 = 0; break;
    default: return 4;
    }
    /* Initialisation (Sec. 4.3, 5.2.1): the root in entry 0 for epoch 0 */
    if (tvm_grow(&m, 1)) return 1;
    m.code[0] = 0 * NUM_TASK_TYPES + root_type;
    m.arg0[0] = r0; m.arg1[0] = r1; m.link[0] = 0; m.result[0] = 0;
    m.next = 1;
    push(&m, 0, 0, 1);
    uint64_t peak = 1, tasks = 0;
    while (m.sp > 0 && !m.err) {
        if (p->max_epochs && m.epoch_index >= p->max_epochs) { m.err = 3; break; }
        /* Phase 1: pop epoch number and NDRange, remember nextFreeCore,
         * clear the join and map flags */
        range_t r = m.stk[--m.sp];
        m.cen = r.cen;
        uint64_t old_next = m.next;
        m.join_scheduled = 0;
        m.map_scheduled = 0;
        m.nmaps = 0;
        /* Phase 2: every entry of the range whose code lies in
         * [CEN*NTT+1, (CEN+1)*NTT] runs; others exit at once */
        uint32_t valid = 0;
        const uint32_t lo_code = r.cen * NUM_TASK_TYPES + 1, hi_code = (r.cen + 1) * NUM_TASK_TYPES;
        for (uint32_t s = r.lo; s < r.hi && !m.err; s++) {
            uint32_t c = m.code[s];
            if (c < lo_code || c > hi_code) continue;
            valid++;
            run_task(&m, s, c - r.cen * NUM_TASK_TYPES);
        }
        if (m.err) break;
        const uint32_t forked = (uint32_t)(m.next - old_next);
        /* Phase 3: join range first, fork range on top (LIFO), then maps */
        if (m.join_scheduled) push(&m, r.cen, r.lo, r.hi);
        if (forked) push(&m, r.cen + 1, (uint32_t)old_next, (uint32_t)m.next);
        for (uint64_t i = 0; i < m.nmaps; i++) run_map(&m, &m.maps[i]);
        /* an epoch with neither forks nor joins returns its entries */
        if (!m.join_scheduled && !forked) {
            if (m.next != r.hi) { m.err = 5; break; }
            m.next = r.lo;
        }
        if (trace && m.epoch_index < trace_cap) {
            oracle_epoch_t *t = &trace[m.epoch_index];
            t->cen = r.cen; t->lo = r.lo; t->hi = r.hi; t->valid = valid;
            t->forks = forked;
            t->joined = (uint32_t)m.join_scheduled;
            t->maps = (uint32_t)m.nmaps;
        }
        if (old_next + forked > peak) peak = old_next + forked;
        tasks += valid;
        m.epoch_index++;
    }
    st->epochs = m.epoch_index;
    st->tasks = tasks;
    st->forks = m.n_forks;
    st->joins = m.n_joins;
    st->maps = m.n_maps;
    st->peak_slots = peak;
    st->root_result = m.result ? m.result[0] : 0;
    st->final_slots = m.next;
    st->err = m.err;
    free(m.code); free(m.arg0); free(m.arg1); free(m.link); free(m.result);
    free(m.stk); free(m.maps); free(m.tmp);
    return m.err;
}
