// Task programs and the per-epoch work of the TREES runtime on sm_103a.
//
// Phase 2 of an epoch (Sec. 4.3.2, 5.2.3) is processed in tiles of one slot
// per thread.  Each task is executed in two steps: `plan_task` reads the
// entry, performs emits (own-slot writes) and reports how many children it
// forks and which map it schedules; after the block-wide scan and the one
// atomic per block that hand out contiguous TV slots (the cooperative fork
// of Sec. 5.2.3, one atomic per block instead of one per wavefront),
// `commit_task` writes the children for epoch CEN+1 and rewrites its own
// entry as a join continuation (Sec. 4.3.2).
//
// Map operations (Sec. 4.2, 4.3.2, 5.2.4) are data-parallel work run by the
// whole grid after the epoch's tasks and before the next epoch: the
// mergesort leaf sort and merge-path merge, and the BFS adjacency expansion.
#pragma once

#include "trees_dev.cuh"

namespace trees {

struct Acc {
    uint32_t valid, joins, maps;
};

struct Plan {
    uint32_t type, s, a0, a1;
    uint32_t nfork;
    uint32_t mkind, ma, mb, mc, mtiles;  // tiled map request (leaf sort, merge)
    uint32_t xv, xn;                     // element map request (BFS expansion)
};

// Leaf of the fib cutoff variant: the naive recursion run inside the task
// with an explicit stack (depth <= n + 1; n <= 30 is enforced by the host).
__device__ __forceinline__ unsigned long long fib_leaf(uint32_t n) {
    uint8_t st[40];
    int sp = 0;
    unsigned long long acc = 0;
    st[sp++] = (uint8_t)n;
    while (sp) {
        const uint32_t x = st[--sp];
        if (x < 2u) {
            acc += x;
        } else {
            st[sp++] = (uint8_t)(x - 1u);
            st[sp++] = (uint8_t)(x - 2u);
        }
    }
    return acc;
}

// N-Queens row task arguments: a0 = cols | r << 16, a1 = d1 | d2 << 16, where
// d1/d2 are the diagonal masks shifted to the current row.
__device__ __forceinline__ uint32_t nq_free(uint32_t a0, uint32_t a1, uint32_t n) {
    return ~((a0 & 0xFFFFu) | (a1 & 0xFFFFu) | (a1 >> 16)) & ((1u << n) - 1u);
}

// Step 1 of a task: read it, emit if it is a leaf, count forks, request maps.
__device__ __forceinline__ void plan_task(const Conf &c, const RunParams &rp, Plan &p, uint32_t cen, uint32_t e) {
    const uint32_t s = p.s;
    switch (p.type) {
    case TREES_TASK_FIB: {
        const uint32_t n = c.a0[s];
        p.a0 = n;
        if (n < 2u || n <= rp.cutoff) {
            c.result[s] = n < 2u ? (unsigned long long)n : fib_leaf(n);
            c.code[s] = 0u;  // emit: the entry is dead (Sec. 4.3.2)
        } else {
            p.nfork = 2u;
        }
        break;
    }
    case TREES_TASK_FIB_SUM: {
        const uint32_t l = c.link[s];
        c.result[s] = c.result[l] + c.result[l + 1];
        c.code[s] = 0u;
        break;
    }
    case TREES_TASK_MS_SPLIT: {
        const uint32_t lo = c.a0[s], hi = c.a1[s];
        p.a0 = lo;
        p.a1 = hi;
        if (hi - lo <= rp.leaf) {
            if (hi > lo) {
                p.mkind = MAP_LEAF_SORT;
                p.ma = lo;
                p.mb = hi;
                p.mc = cen;
                p.mtiles = 1u;
            }
            c.code[s] = 0u;
        } else {
            p.nfork = 2u;
        }
        break;
    }
    case TREES_TASK_MS_MERGE: {
        const uint32_t lo = c.a0[s], hi = c.a1[s];
        p.mkind = MAP_MERGE;
        p.ma = lo;
        p.mb = hi;
        p.mc = cen;
        p.mtiles = (hi - lo + MERGE_TILE - 1u) / MERGE_TILE;
        c.code[s] = 0u;
        break;
    }
    case TREES_TASK_NQ_ROW: {
        const uint32_t a0 = c.a0[s], a1 = c.a1[s], n = rp.n;
        p.a0 = a0;
        p.a1 = a1;
        if ((a0 >> 16) == n) {
            c.result[s] = 1ull;
            c.code[s] = 0u;
            break;
        }
        const uint32_t fr = nq_free(a0, a1, n);
        if (fr == 0u) {
            c.result[s] = 0ull;
            c.code[s] = 0u;
        } else {
            p.nfork = (uint32_t)__popc(fr);
        }
        break;
    }
    case TREES_TASK_NQ_SUM: {
        const uint32_t k = (uint32_t)__popc(nq_free(c.a0[s], c.a1[s], rp.n));
        const uint32_t l = c.link[s];
        unsigned long long sum = 0;
        for (uint32_t i = 0; i < k; ++i) sum += c.result[l + i];
        c.result[s] = sum;
        c.code[s] = 0u;
        break;
    }
    case TREES_TASK_BFS_VISIT: {
        const uint32_t v = c.a0[s];
        const int32_t rb = __ldg(rp.row_ptr + v), re = __ldg(rp.row_ptr + v + 1);
        if (re > rb) {
            p.xv = (uint32_t)rb;
            p.xn = (uint32_t)(re - rb);
        }
        c.code[s] = 0u;
        break;
    }
    case TREES_TASK_PO: {
        const uint32_t node = c.a0[s];
        p.a0 = node;
        if ((int32_t)node < 0) c.code[s] = 0u;
        else p.nfork = 2u;
        break;
    }
    case TREES_TASK_PO_AFTER: {
        rp.visit_epoch[c.a0[s]] = (int32_t)e;
        c.code[s] = 0u;
        break;
    }
    case TREES_TASK_PRE: {
        const uint32_t node = c.a0[s];
        p.a0 = node;
        c.code[s] = 0u;
        if ((int32_t)node >= 0) {
            rp.visit_epoch[node] = (int32_t)e;
            p.nfork = 2u;
        }
        break;
    }
    default:
        break;
    }
}

// Step 2: write the children into [child, child + nfork) for epoch CEN+1 and
// turn the task into its join continuation.  Returns 1 if it joined.
__device__ __forceinline__ uint32_t commit_task(const Conf &c, const RunParams &rp, const Plan &p, uint32_t cen,
                                                 uint32_t child) {
    const uint32_t s = p.s;
    const uint32_t fe = enc(cen + 1u, 0u);
    switch (p.type) {
    case TREES_TASK_FIB:
        c.code[child] = fe + TREES_TASK_FIB;
        c.a0[child] = p.a0 - 1u;
        c.code[child + 1] = fe + TREES_TASK_FIB;
        c.a0[child + 1] = p.a0 - 2u;
        c.link[s] = child;
        c.code[s] = enc(cen, TREES_TASK_FIB_SUM);
        return 1u;
    case TREES_TASK_MS_SPLIT: {
        const uint32_t lo = p.a0, hi = p.a1, mid = lo + (hi - lo) / 2u;
        c.code[child] = fe + TREES_TASK_MS_SPLIT;
        c.a0[child] = lo;
        c.a1[child] = mid;
        c.code[child + 1] = fe + TREES_TASK_MS_SPLIT;
        c.a0[child + 1] = mid;
        c.a1[child + 1] = hi;
        c.link[s] = child;
        c.code[s] = enc(cen, TREES_TASK_MS_MERGE);
        return 1u;
    }
    case TREES_TASK_NQ_ROW: {
        const uint32_t n = rp.n, mask = (1u << n) - 1u;
        const uint32_t r = p.a0 >> 16, cols = p.a0 & 0xFFFFu, d1 = p.a1 & 0xFFFFu, d2 = p.a1 >> 16;
        uint32_t fr = nq_free(p.a0, p.a1, n);
        uint32_t slot = child;
        while (fr) {
            const uint32_t b = fr & (0u - fr);  // lowest safe column first
            fr ^= b;
            c.code[slot] = fe + TREES_TASK_NQ_ROW;
            c.a0[slot] = (cols | b) | ((r + 1u) << 16);
            c.a1[slot] = (((d1 | b) << 1) & mask) | (((d2 | b) >> 1) << 16);
            ++slot;
        }
        c.link[s] = child;
        c.code[s] = enc(cen, TREES_TASK_NQ_SUM);
        return 1u;
    }
    case TREES_TASK_PO: {
        const int32_t node = (int32_t)p.a0;
        c.code[child] = fe + TREES_TASK_PO;
        c.a0[child] = (uint32_t)__ldg(rp.right + node);
        c.code[child + 1] = fe + TREES_TASK_PO;
        c.a0[child + 1] = (uint32_t)__ldg(rp.left + node);
        c.link[s] = child;
        c.code[s] = enc(cen, TREES_TASK_PO_AFTER);
        return 1u;
    }
    case TREES_TASK_PRE: {
        const int32_t node = (int32_t)p.a0;
        c.code[child] = fe + TREES_TASK_PRE;
        c.a0[child] = (uint32_t)__ldg(rp.right + node);
        c.code[child + 1] = fe + TREES_TASK_PRE;
        c.a0[child + 1] = (uint32_t)__ldg(rp.left + node);
        return 0u;
    }
    default:
        return 0u;
    }
}

// Map allocation for one tile: one packed block scan per map list and one
// atomic per list per block, then coalesced descriptor writes.  Tiled maps
// also get a tile -> descriptor table, written cooperatively by the block.
template <int BS>
__device__ void map_alloc(const Conf &c, Ctl *ctl, Smem<BS> &sm, const Plan &p, uint32_t ep, uint32_t e,
                          uint32_t job, Acc &acc) {
    const unsigned long long qa = p.mtiles ? ((1ull << 40) | p.mtiles) : 0ull;
    const unsigned long long qb = p.xn ? ((1ull << 40) | p.xn) : 0ull;
    unsigned long long ea, eb, ta, tb;
    block_scan_u64x2<BS>(qa, qb, &ea, &eb, &ta, &tb, sm);
    if (threadIdx.x == 0) {
        sm.bc64[0] = ta ? atomicAdd(&ctl->mt_ctr[ep], ta) : 0ull;
        sm.bc64[1] = tb ? atomicAdd(&ctl->me_ctr[ep], tb) : 0ull;
    }
    __syncthreads();
    if (ta) {
        const unsigned long long g = sm.bc64[0];
        const uint32_t dbase = (uint32_t)(g >> 40), tbase = (uint32_t)(g & CTR_LOW_MASK);
        const uint32_t ndesc = (uint32_t)(ta >> 40), ntile = (uint32_t)(ta & CTR_LOW_MASK);
        const bool fits = (unsigned long long)dbase + ndesc <= c.mcap &&
                          (unsigned long long)tbase + ntile <= c.mcap;
        if (!fits) {
            if (threadIdx.x == 0) set_err(ctl, TREES_ERR_CAPACITY, e);
        } else {
            if (p.mtiles) {
                const uint32_t rank = (uint32_t)(ea >> 40), toff = (uint32_t)(ea & CTR_LOW_MASK);
                const uint32_t di = dbase + rank;
                c.mt_kind[di] = p.mkind;
                c.mt_a[di] = p.ma;
                c.mt_b[di] = p.mb;
                c.mt_c[di] = p.mc;
                c.mt_job[di] = job;
                c.mt_tilebase[di] = tbase + toff;
                sm.u.rq.toff[rank] = toff;
                sm.u.rq.di[rank] = di;
                acc.maps++;
            }
            __syncthreads();
            for (uint32_t k = threadIdx.x; k < ntile; k += BS) {
                uint32_t lo = 0, hi = ndesc;  // last request whose first tile is <= k
                while (hi - lo > 1u) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (sm.u.rq.toff[mid] <= k) lo = mid;
                    else hi = mid;
                }
                c.mt_tiledesc[tbase + k] = sm.u.rq.di[lo];
            }
        }
    }
    if (tb) {
        const unsigned long long g = sm.bc64[1];
        const uint32_t dbase = (uint32_t)(g >> 40);
        const unsigned long long ebase = g & CTR_LOW_MASK;
        const uint32_t ndesc = (uint32_t)(tb >> 40);
        const unsigned long long nel = tb & CTR_LOW_MASK;
        const unsigned long long tiles_end = (ebase + nel + EXPAND_TILE - 1) / EXPAND_TILE;
        const bool fits = (unsigned long long)dbase + ndesc <= c.mcap && ebase + nel < 0xFFFFFFFFull &&
                          tiles_end <= c.mcap;
        if (!fits) {
            if (threadIdx.x == 0) set_err(ctl, TREES_ERR_CAPACITY, e);
        } else if (p.xn) {
            const uint32_t di = dbase + (uint32_t)(eb >> 40);
            const uint32_t b = (uint32_t)(ebase + (eb & CTR_LOW_MASK));
            c.me_v[di] = p.xv;
            c.me_base[di] = b;
            c.me_job[di] = job;
            // every expansion tile whose first element falls in [b, b + xn) starts at this descriptor
            for (uint32_t t = (b + EXPAND_TILE - 1u) / EXPAND_TILE; t * EXPAND_TILE < b + p.xn; ++t) c.me_tfd[t] = di;
            acc.maps++;
        }
    }
}

// One Phase-2 tile: the slots [t0, t0 + BS) of the current range.
template <int BS>
__device__ __forceinline__ void epoch_tile(const Conf &c, Ctl *ctl, Smem<BS> &sm, uint32_t s, bool inr, uint32_t cen,
                                           uint32_t base, uint32_t ep, uint32_t e, Acc &acc) {
    Plan p;
    p.type = 0u;
    p.s = s;
    p.a0 = p.a1 = 0u;
    p.nfork = 0u;
    p.mkind = p.ma = p.mb = p.mc = p.mtiles = 0u;
    p.xv = p.xn = 0u;
    if (inr) p.type = task_type(c.code[s], cen);  // invalid or stale entries exit at once (Sec. 5.3)
    if (p.type) {
        acc.valid++;
        plan_task(c, c.rp, p, cen, e);
    }
    uint32_t ftot;
    int anymap;
    const uint32_t foff = block_scan_u32<BS>(p.nfork, (p.mtiles | p.xn) != 0u, &ftot, &anymap, sm);
    if (ftot) {
        if (threadIdx.x == 0) {
            const uint32_t b = atomicAdd(&ctl->cnt[ep], ftot);  // one atomic per block (Sec. 5.2.3)
            const bool over = (unsigned long long)base + b + ftot > c.cap;
            if (over) set_err(ctl, TREES_ERR_CAPACITY, e);
            sm.bc32[0] = b;
            sm.bc32[1] = over;
        }
        __syncthreads();
        uint32_t joined = 0u;
        if (!sm.bc32[1] && p.nfork) joined = commit_task(c, c.rp, p, cen, base + sm.bc32[0] + foff);
        acc.joins += joined;
        if (__any_sync(0xffffffffu, joined) && (threadIdx.x & 31) == 0) ctl->join[ep] = 1u;  // joinScheduled
    }
    if (anymap) map_alloc<BS>(c, ctl, sm, p, ep, e, 0u, acc);
    __syncthreads();
}

// ------------------------------------------------------------------ map operations

// Sorts keys in[lo, hi) (at most LEAF_MAX) in shared memory with a bitonic
// network and writes them to out[lo, hi).
template <int BS>
__device__ void leaf_sort(const uint32_t *in, uint32_t *out, uint32_t lo, uint32_t hi, Smem<BS> &sm) {
    const uint32_t n = hi - lo;
    uint32_t P = 1u;
    while (P < n) P <<= 1;
    for (uint32_t i = threadIdx.x; i < P; i += BS) sm.u.sortk[i] = i < n ? in[lo + i] : 0xFFFFFFFFu;
    __syncthreads();
    for (uint32_t k = 2u; k <= P; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0u; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < P / 2u; i += BS) {
                const uint32_t a = ((i & ~(j - 1u)) << 1) | (i & (j - 1u)), b = a + j;
                const uint32_t x = sm.u.sortk[a], y = sm.u.sortk[b];
                const bool up = (a & k) == 0u;
                if ((x > y) == up) {
                    sm.u.sortk[a] = y;
                    sm.u.sortk[b] = x;
                }
            }
            __syncthreads();
        }
    }
    for (uint32_t i = threadIdx.x; i < n; i += BS) out[lo + i] = sm.u.sortk[i];
    __syncthreads();
}

// Merge path (Odeh et al., "Merge Path -- parallel merging made simple",
// IPDPSW 2012): the number of A elements among the first `diag` outputs of
// the stable merge of sorted A and B.  One warp probes 32 points per step.
__device__ __forceinline__ uint32_t warp_merge_path(const uint32_t *A, uint32_t la, const uint32_t *B, uint32_t lb,
                                                    uint32_t diag) {
    uint32_t lo = diag > lb ? diag - lb : 0u, hi = diag < la ? diag : la;
    const uint32_t lane = threadIdx.x & 31u;
    while (hi > lo) {
        const uint32_t step = (hi - lo + 31u) / 32u;
        const uint32_t m = lo + lane * step;
        bool pr = false;
        if (m < hi) pr = A[m] <= B[diag - 1u - m];
        const uint32_t cnt = (uint32_t)__popc(__ballot_sync(0xffffffffu, pr));
        const uint32_t nlo = cnt ? lo + (cnt - 1u) * step + 1u : lo;
        const uint32_t cap = lo + cnt * step;
        hi = cap < hi ? cap : hi;
        lo = nlo;
    }
    return lo;
}

// One merge-path tile of the merge of in[lo, mid) and in[mid, hi) into
// out[lo, hi), mid = lo + (hi - lo) / 2: outputs [tile*T, tile*T + T).
template <int BS>
__device__ void merge_tile(const uint32_t *in, uint32_t *out, uint32_t lo, uint32_t hi, uint32_t tile, Smem<BS> &sm) {
    const uint32_t mid = lo + (hi - lo) / 2u;
    const uint32_t *A = in + lo;
    const uint32_t *B = in + mid;
    const uint32_t la = mid - lo, lb = hi - mid, L = la + lb;
    const uint32_t d0 = tile * MERGE_TILE, d1 = min(d0 + MERGE_TILE, L);
    const uint32_t wid = threadIdx.x >> 5;
    if (wid < 2u) {
        const uint32_t r = warp_merge_path(A, la, B, lb, wid == 0u ? d0 : d1);
        if ((threadIdx.x & 31u) == 0u) sm.u.mg.split[wid] = r;
    }
    __syncthreads();
    const uint32_t i0 = sm.u.mg.split[0], i1 = sm.u.mg.split[1];
    const uint32_t j0 = d0 - i0, j1 = d1 - i1;
    const uint32_t na = i1 - i0, nb = j1 - j0, nt = na + nb;
    uint32_t *sin = sm.u.mg.in;
    for (uint32_t k = threadIdx.x; k < na; k += BS) sin[k] = A[i0 + k];
    for (uint32_t k = threadIdx.x; k < nb; k += BS) sin[na + k] = B[j0 + k];
    __syncthreads();
    constexpr uint32_t MPT = MERGE_TILE / BS;
    const uint32_t dd = min(threadIdx.x * MPT, nt);
    uint32_t a = dd > nb ? dd - nb : 0u, b = dd < na ? dd : na;
    while (a < b) {
        const uint32_t m = (a + b) >> 1;
        if (sin[m] <= sin[na + dd - 1u - m]) a = m + 1u;
        else b = m;
    }
    uint32_t ia = a, ib = dd - a;
    const uint32_t dend = min(dd + MPT, nt);
    for (uint32_t o = dd; o < dend; ++o) {
        const bool takeA = ia < na && (ib >= nb || sin[ia] <= sin[na + ib]);
        sm.u.mg.out[o] = takeA ? sin[ia++] : sin[na + ib++];
    }
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < nt; k += BS) out[lo + d0 + k] = sm.u.mg.out[k];
    __syncthreads();
}

// One BFS expansion tile: EXPAND_TILE consecutive adjacency entries of the
// epoch's frontier.  Each entry's vertex is found by a binary search over the
// tile's descriptors in shared memory (load-balanced search); an unvisited
// neighbour is claimed with a CAS on its level and forked as a visit task.
template <int BS>
__device__ void expand_tile(const Conf &c, Ctl *ctl, Smem<BS> &sm, uint32_t t, uint32_t nd, uint32_t ne, uint32_t nt,
                            uint32_t cen, uint32_t base, uint32_t ep, uint32_t e) {
    constexpr uint32_t EPT = EXPAND_TILE / BS;
    const uint32_t g0 = t * EXPAND_TILE, g1 = min(g0 + EXPAND_TILE, ne);
    const uint32_t dfirst = c.me_tfd[t];
    const uint32_t dlast = (t + 1u < nt) ? c.me_tfd[t + 1u] : nd - 1u;
    const uint32_t nloc = dlast - dfirst + 1u;
    for (uint32_t k = threadIdx.x; k < nloc; k += BS) {
        sm.u.ex.base[k] = c.me_base[dfirst + k];
        sm.u.ex.v[k] = c.me_v[dfirst + k];
    }
    __syncthreads();
    uint32_t claimed[EPT];
    uint32_t nc = 0;
    const int32_t nlev = (int32_t)(cen + 1u);
#pragma unroll
    for (uint32_t j = 0; j < EPT; ++j) {
        const uint32_t g = g0 + j * BS + threadIdx.x;
        if (g < g1) {
            uint32_t lo = 0, hi = nloc;
            while (hi - lo > 1u) {
                const uint32_t mid = (lo + hi) >> 1;
                if (sm.u.ex.base[mid] <= g) lo = mid;
                else hi = mid;
            }
            const uint32_t edge = sm.u.ex.v[lo] + (g - sm.u.ex.base[lo]);
            const int32_t u = __ldg(c.rp.col + edge);
            int32_t *lv = c.rp.level + u;
            if (*(volatile int32_t *)lv < 0 && atomicCAS(lv, -1, nlev) == -1) claimed[nc++] = (uint32_t)u;
        }
    }
    uint32_t ftot;
    int any;
    const uint32_t off = block_scan_u32<BS>(nc, 0, &ftot, &any, sm);
    if (ftot) {
        if (threadIdx.x == 0) {
            const uint32_t b = atomicAdd(&ctl->cnt[ep], ftot);
            const bool over = (unsigned long long)base + b + ftot > c.cap;
            if (over) set_err(ctl, TREES_ERR_CAPACITY, e);
            sm.bc32[0] = b;
            sm.bc32[1] = over;
        }
        __syncthreads();
        if (!sm.bc32[1]) {
            const uint32_t code = enc(cen + 1u, TREES_TASK_BFS_VISIT);
            const uint32_t slot0 = base + sm.bc32[0] + off;
            for (uint32_t i = 0; i < nc; ++i) {
                c.code[slot0 + i] = code;
                c.a0[slot0 + i] = claimed[i];
            }
        }
    }
    __syncthreads();
}

// The map phase of epoch e: every block takes tiles grid-stride over the
// tiled list (leaf sorts, merge tiles) followed by the expansion tiles.
template <int BS>
__device__ void map_phase(const Conf &c, Ctl *ctl, Smem<BS> &sm, uint32_t ep, uint32_t e, uint32_t cen, uint32_t base,
                          unsigned long long mt, unsigned long long me, const RunParams *job_params = nullptr,
                          uint32_t job_stride = 0) {
    const uint32_t nt1 = (uint32_t)(mt & CTR_LOW_MASK);
    const uint32_t nd2 = (uint32_t)(me >> 40), ne2 = (uint32_t)(me & CTR_LOW_MASK);
    const uint32_t nt2 = (ne2 + EXPAND_TILE - 1u) / EXPAND_TILE;
    uint32_t *keys = c.rp.keys, *scratch = c.rp.scratch;
    for (uint32_t t = blockIdx.x; t < nt1 + nt2; t += gridDim.x) {
        if (t < nt1) {
            const uint32_t di = c.mt_tiledesc[t];
            const uint32_t kind = c.mt_kind[di], a = c.mt_a[di], b = c.mt_b[di], cc = c.mt_c[di];
            if (job_params) {  // batched runs: the descriptor names its job
                const RunParams *jp = reinterpret_cast<const RunParams *>(
                    reinterpret_cast<const char *>(job_params) + (size_t)c.mt_job[di] * job_stride);
                keys = jp->keys;
                scratch = jp->scratch;
            }
            // a node at depth d writes its sorted run to keys (d even) or scratch (d odd)
            uint32_t *outb = (cc & 1u) ? scratch : keys;
            if (kind == MAP_LEAF_SORT) {
                leaf_sort<BS>(keys, outb, a, b, sm);
            } else {
                const uint32_t *inb = (cc & 1u) ? keys : scratch;
                merge_tile<BS>(inb, outb, a, b, t - c.mt_tilebase[di], sm);
            }
        } else {
            expand_tile<BS>(c, ctl, sm, t - nt1, nd2, ne2, nt2, cen, base, ep, e);
        }
    }
}

}  // namespace trees
