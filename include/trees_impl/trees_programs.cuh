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
// mergesort leaf sort and merge-path merge, the BFS and SSSP adjacency
// expansions and the FFT's combine butterflies.
#pragma once

#include "trees_dev.cuh"

namespace trees {

struct Acc {
    uint32_t valid, joins, maps;
};

// Program masks: which task types (and maps) a kernel is compiled for.  A
// kernel built for one program carries only that program's dispatch cases,
// as the paper's compiler emits one kernel per program (Sec. 5).
constexpr uint32_t PM_FIB = 1u, PM_MS = 2u, PM_NQ = 4u, PM_BFS = 8u, PM_TRAV = 16u, PM_SSSP = 32u, PM_FFT = 64u;
constexpr uint32_t PM_USER = 128u;  // a user program (trees_program.cuh), compiled into its own kernel
constexpr uint32_t PM_ALL = PM_FIB | PM_MS | PM_NQ | PM_BFS | PM_TRAV | PM_SSSP | PM_FFT;  // the built-in programs
constexpr uint32_t PM_MAPS = PM_MS | PM_BFS | PM_SSSP | PM_FFT | PM_USER;  // programs that may schedule maps

// The program type a kernel built for built-in programs carries (none).
struct NoUserProgram {};

__device__ __forceinline__ trees_user_env user_env(const Conf &c) {
    trees_user_env env;
#pragma unroll
    for (int i = 0; i < TREES_USER_PARAMS; ++i) {
        env.ptr[i] = c.rp.up[i];
        env.val[i] = c.rp.uv[i];
    }
    env.result = reinterpret_cast<uint64_t *>(c.result);
    return env;
}

__host__ __device__ constexpr uint32_t program_mask(int program) {
    return program == TREES_PROG_FIB         ? PM_FIB
           : program == TREES_PROG_MERGESORT ? PM_MS
           : program == TREES_PROG_NQUEENS   ? PM_NQ
           : program == TREES_PROG_BFS       ? PM_BFS
           : program == TREES_PROG_SSSP      ? PM_SSSP
           : program == TREES_PROG_FFT       ? PM_FFT
                                             : PM_TRAV;
}

// What one task decided in step 1: its slot, its type, how many children it
// forks (or how many map units it schedules when m != 0) and the arguments
// step 2 needs.
struct Plan {
    uint32_t s, t, n, m, a0, a1;
};

// SSSP relax records pack (epoch + 1) above the low SSSP_USED_SHIFT bits of
// a distance; distances of 2^40 or more are never recorded (their vertices
// are simply relaxed again when forked).
constexpr uint32_t SSSP_USED_SHIFT = 40;

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

// Which TV columns a task type reads besides its code.
__device__ __forceinline__ bool needs_a0(uint32_t t) { return t != 0u && t != TREES_TASK_FIB_SUM; }
__device__ __forceinline__ bool needs_a1(uint32_t t) {
    return t == TREES_TASK_MS_SPLIT || t == TREES_TASK_MS_MERGE || t == TREES_TASK_NQ_ROW || t == TREES_TASK_NQ_SUM ||
           t == TREES_TASK_FFT || t == TREES_TASK_FFT_COMBINE;
}

// ------------------------------------------------------------------ FFT (Sec. 6.2)
// Radix-2 Cooley-Tukey by decimation in time.  Task FFT(o, d) (a0 = o,
// a1 = d) transforms the M = N >> d points x[o + j 2^d], j < M.  Its even-
// numbered points are the points of FFT(o, d+1), its odd-numbered ones those
// of FFT(o + 2^d, d+1); their transforms E and O land in the first and second
// half of its own output block, which the combine turns into its transform:
// X[k] = E[k] + w^k O[k], X[k + M/2] = E[k] - w^k O[k], w = exp(-2 pi i / M).
// So the block of FFT(o, d) starts at the d low bits of o reversed, times M.
__device__ __forceinline__ uint32_t fft_block(uint32_t o, uint32_t d, uint32_t lgn) {
    return d ? (__brev(o) >> (32u - d)) << (lgn - d) : 0u;
}

// exp(-2 pi i k / 2^lgm), k < 2^(lgm-1): sincospif of 2k / 2^lgm, a quotient
// that is exact in fp32 for k < 2^24.
__device__ __forceinline__ float2 fft_twiddle(uint32_t k, uint32_t lgm) {
    float sn, cs;
    sincospif(ldexpf((float)k, 1 - (int)lgm), &sn, &cs);
    return make_float2(cs, -sn);
}

// One butterfly, e <- e + w o, o <- e - w o, with the roundings spelled out
// so that every caller (leaf, combine task, combine map) computes
// bit-identical values.
__device__ __forceinline__ void fft_bfly(float2 &e, float2 &o, float2 w) {
    const float tr = __fmaf_rn(w.x, o.x, -__fmul_rn(w.y, o.y));
    const float ti = __fmaf_rn(w.x, o.y, __fmul_rn(w.y, o.x));
    const float2 a = e;
    e = make_float2(__fadd_rn(a.x, tr), __fadd_rn(a.y, ti));
    o = make_float2(__fsub_rn(a.x, tr), __fsub_rn(a.y, ti));
}

__host__ __device__ constexpr int fft_rev(int j, int bits) {
    return bits == 0 ? 0 : ((j & 1) << (bits - 1)) | fft_rev(j >> 1, bits - 1);
}

// The leaves among one thread's TPT slots of a tile, K = 2^LK points each,
// in registers: the points of G leaves are loaded together (their loads in
// flight at once), then each leaf is transformed and stored.  Register r of
// a leaf holds its point of index rev(r) (LK-bit reversal), so the LK
// butterfly stages (the combines of its 2-, 4-, ..., K-point
// sub-transforms, in the same arithmetic as the combine tasks) leave the
// transform in natural order.
template <int LK, int TPT>
__device__ __forceinline__ void fft_leaves_k(const float2 *__restrict__ x, float2 *__restrict__ X, uint32_t lgn,
                                             const Plan (&p)[TPT], uint32_t d) {
    constexpr int K = 1 << LK, G = LK >= 4 ? 1 : (TPT < 2 ? TPT : 2);  // at most 16 points in flight per thread
#pragma unroll
    for (int k0 = 0; k0 < TPT; k0 += G) {
        float2 a[G][K];
        bool lf[G];
#pragma unroll
        for (int g = 0; g < G; ++g) {
            lf[g] = p[k0 + g].t == TREES_TASK_FFT && p[k0 + g].n == 0u;
            if (lf[g]) {
#pragma unroll
                for (int r = 0; r < K; ++r) a[g][r] = x[p[k0 + g].a0 + ((uint32_t)fft_rev(r, LK) << d)];
            }
        }
#pragma unroll
        for (int g = 0; g < G; ++g) {
            if (!lf[g]) continue;
#pragma unroll
            for (int lm = 1; lm <= LK; ++lm) {
                const int h = 1 << (lm - 1);
#pragma unroll
                for (int k = 0; k < h; ++k) {
                    const float2 w = fft_twiddle((uint32_t)k, (uint32_t)lm);
#pragma unroll
                    for (int q = 0; q < K; q += 2 * h) fft_bfly(a[g][q + k], a[g][q + k + h], w);
                }
            }
            const uint32_t dst = fft_block(p[k0 + g].a0, d, lgn);
#pragma unroll
            for (int k = 0; k < K; ++k) X[dst + k] = a[g][k];
        }
    }
}

// All leaves of an epoch have the same depth d, so one leaf size serves the thread.
template <int TPT>
__device__ __forceinline__ void fft_leaves(const float2 *x, float2 *X, uint32_t lgn, const Plan (&p)[TPT]) {
    uint32_t d = 0xFFFFFFFFu;
#pragma unroll
    for (int k = 0; k < TPT; ++k)
        if (p[k].t == TREES_TASK_FFT && p[k].n == 0u) d = p[k].a1;
    if (d == 0xFFFFFFFFu) return;
    switch (lgn - d) {
    case 0:  // one point: the transform is the point
#pragma unroll
        for (int k = 0; k < TPT; ++k)
            if (p[k].t == TREES_TASK_FFT && p[k].n == 0u) X[fft_block(p[k].a0, d, lgn)] = x[p[k].a0];
        break;
    case 1: fft_leaves_k<1, TPT>(x, X, lgn, p, d); break;
    case 2: fft_leaves_k<2, TPT>(x, X, lgn, p, d); break;
    case 3: fft_leaves_k<3, TPT>(x, X, lgn, p, d); break;
    default: fft_leaves_k<4, TPT>(x, X, lgn, p, d); break;
    }
}

// One leaf, out of line (see fft_task_bodies).
static __device__ __noinline__ void fft_leaf_slot(const float2 *x, float2 *X, uint32_t o, uint32_t d, uint32_t lgn) {
    Plan q[1];
    q[0].t = TREES_TASK_FFT;
    q[0].n = 0u;
    q[0].a0 = o;
    q[0].a1 = d;
    fft_leaves<1>(x, X, lgn, q);
}

// A combine of 2^lgm points done by its own task (the paper's FFT).
static __device__ __noinline__ void fft_combine_task(float2 *X, uint32_t dst, uint32_t lgm) {
    const uint32_t h = 1u << (lgm - 1u);
    uint32_t k = 0;
    for (; k + 4u <= h; k += 4u) {
        float2 e[4], o[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            e[q] = X[dst + k + q];
            o[q] = X[dst + h + k + q];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            fft_bfly(e[q], o[q], fft_twiddle(k + q, lgm));
            X[dst + k + q] = e[q];
            X[dst + h + k + q] = o[q];
        }
    }
    for (; k < h; ++k) {
        float2 e = X[dst + k], o = X[dst + h + k];
        fft_bfly(e, o, fft_twiddle(k, lgm));
        X[dst + k] = e;
        X[dst + h + k] = o;
    }
}
__device__ __forceinline__ bool needs_link(uint32_t t) { return t == TREES_TASK_FIB_SUM || t == TREES_TASK_NQ_SUM; }

// Step 1 of a task: given its arguments, emit if it is a leaf (own-slot
// writes, Sec. 4.3.2), count its forks, or request a map.  Only the task
// types of the programs in PM are compiled in.
template <uint32_t PM, uint32_t MT, typename UP = NoUserProgram>
__device__ __forceinline__ void plan_task(const Conf &c, const RunParams &rp, Plan &p, uint32_t cen, uint32_t e,
                                          uint32_t a0, uint32_t a1, uint32_t lk) {
    const uint32_t s = p.s;
    p.a0 = a0;
    p.a1 = a1;
    if constexpr ((PM & PM_USER) != 0u) {  // the user program decides (trees_user.h)
        const trees_user_task t = {s, p.t, a0, a1, lk, cen};
        const trees_user_plan q = UP::plan(t, user_env(c));
        if (q.map_units) {
            p.m = MAP_USER;
            p.n = q.map_units;
            p.a0 = q.map_a;
            p.a1 = q.map_b;
        } else {
            p.n = q.forks;
        }
        if (q.emit) c.result[s] = q.value;
        if (!q.forks || q.map_units) c.code[s] = 0u;
        return;
    }
    if constexpr ((PM & PM_FIB) != 0u) {
        if (p.t == TREES_TASK_FIB) {
            if (a0 < 2u || a0 <= rp.cutoff) {
                c.result[s] = a0 < 2u ? (unsigned long long)a0 : fib_leaf(a0);
                c.code[s] = 0u;  // emit: the entry is dead
            } else {
                p.n = 2u;
            }
            return;
        }
        if (p.t == TREES_TASK_FIB_SUM) {
            c.result[s] = c.result[lk] + c.result[lk + 1];
            c.code[s] = 0u;
            return;
        }
    }
    if constexpr ((PM & PM_MS) != 0u) {
        if (p.t == TREES_TASK_MS_SPLIT) {
            if (a1 - a0 <= rp.leaf) {
                if (a1 > a0) {
                    p.m = MAP_LEAF_SORT;
                    p.n = 1u;
                }
                c.code[s] = 0u;
            } else {
                p.n = 2u;
            }
            return;
        }
        if (p.t == TREES_TASK_MS_MERGE) {
            p.m = MAP_MERGE;
            p.n = (a1 - a0 + MT - 1u) / MT;  // merge tiles of MT outputs
            c.code[s] = 0u;
            return;
        }
    }
    if constexpr ((PM & PM_NQ) != 0u) {
        if (p.t == TREES_TASK_NQ_ROW) {
            if ((a0 >> 16) == rp.n) {
                c.result[s] = 1ull;
                c.code[s] = 0u;
                return;
            }
            const uint32_t fr = nq_free(a0, a1, rp.n);
            if (fr == 0u) {
                c.result[s] = 0ull;
                c.code[s] = 0u;
            } else {
                p.n = (uint32_t)__popc(fr);
            }
            return;
        }
        if (p.t == TREES_TASK_NQ_SUM) {
            const uint32_t k = (uint32_t)__popc(nq_free(a0, a1, rp.n));
            unsigned long long sum = 0;
            for (uint32_t i = 0; i < k; ++i) sum += c.result[lk + i];
            c.result[s] = sum;
            c.code[s] = 0u;
            return;
        }
    }
    if constexpr ((PM & PM_BFS) != 0u) {
        if (p.t == TREES_TASK_BFS_VISIT) {
            const int32_t rb = __ldg(rp.row_ptr + a0), re = __ldg(rp.row_ptr + a0 + 1);
            if (re > rb) {
                p.m = MAP_EXPAND;
                p.a0 = (uint32_t)rb;
                p.n = (uint32_t)(re - rb);
            }
            c.code[s] = 0u;
            return;
        }
    }
    if constexpr ((PM & PM_SSSP) != 0u) {
        if (p.t == TREES_TASK_SSSP_RELAX) {  // relax(v): a map over v's out-edges (Sec. 6.3)
            const int32_t rb = __ldg(rp.row_ptr + a0), re = __ldg(rp.row_ptr + a0 + 1);
            // v's relaxation in the previous epoch already propagated its current distance along
            // every out-edge: nothing is left to relax, the task ends at once
            const unsigned long long dv = rp.dist[a0];
            const bool done = cen > 0u && dv < (1ull << SSSP_USED_SHIFT) &&  // record 0 = never relaxed
                              rp.used[a0] == ((unsigned long long)cen << SSSP_USED_SHIFT | dv);
            if (re > rb && !done) {
                p.m = MAP_EXPAND;
                p.a0 = (uint32_t)rb;
                p.a1 = a0;
                p.n = (uint32_t)(re - rb);
            }
            c.code[s] = 0u;
            return;
        }
    }
    if constexpr ((PM & PM_FFT) != 0u) {
        // a leaf's transform and a combine done in its task run at the end of
        // the tile (fft_task_bodies), out of this unrolled loop
        if (p.t == TREES_TASK_FFT) {
            if ((1u << (rp.lgn - a1)) <= rp.leaf) c.code[s] = 0u;
            else p.n = 2u;
            return;
        }
        if (p.t == TREES_TASK_FFT_COMBINE) {
            const uint32_t lgm = rp.lgn - a1;
            if ((1u << lgm) > rp.cutoff) {  // a map over its 2^(lgm-1) butterflies
                p.m = MAP_FFT;
                p.n = 1u << (lgm - 1u);
            }
            c.code[s] = 0u;
            return;
        }
    }
    if constexpr ((PM & PM_TRAV) != 0u) {
        if (p.t == TREES_TASK_PO) {
            if ((int32_t)a0 < 0) c.code[s] = 0u;
            else p.n = 2u;
            return;
        }
        if (p.t == TREES_TASK_PO_AFTER) {
            rp.visit_epoch[a0] = (int32_t)e;
            c.code[s] = 0u;
            return;
        }
        if (p.t == TREES_TASK_PRE) {
            c.code[s] = 0u;
            if ((int32_t)a0 >= 0) {
                rp.visit_epoch[a0] = (int32_t)e;
                p.n = 2u;
            }
            return;
        }
    }
}

__device__ __forceinline__ uint32_t forks_of(const Plan &p) { return p.m ? 0u : p.n; }

// The work of FFT leaves and of combines below the cutoff (both emit and
// fork nothing, so it can follow the tile's forks).  The FFT's own kernel
// with one slot per thread runs its leaf inline (spill-free at 128
// registers); the others call the leaves out of line, so that the leaf's
// registers do not weigh on the rest of the kernel.
template <uint32_t PM, int TPT>
__device__ __forceinline__ void fft_task_bodies(const RunParams &rp, const Plan (&p)[TPT]) {
    if constexpr (PM == PM_FFT && TPT == 1) {
        fft_leaves<TPT>(rp.fx, rp.fX, rp.lgn, p);
    } else {
#pragma unroll 1
        for (int k = 0; k < TPT; ++k)
            if (p[k].t == TREES_TASK_FFT && p[k].n == 0u) fft_leaf_slot(rp.fx, rp.fX, p[k].a0, p[k].a1, rp.lgn);
    }
#pragma unroll
    for (int k = 0; k < TPT; ++k)
        if (p[k].t == TREES_TASK_FFT_COMBINE && p[k].m == 0u)
            fft_combine_task(rp.fX, fft_block(p[k].a0, p[k].a1, rp.lgn), rp.lgn - p[k].a1);
}

// The FFT's leaf epoch (16-point leaves): every task of a fresh FFT range
// has depth CEN (the root is task (0, 0) of epoch 0 and a fork's children
// have the next depth in the next epoch), so when 2^(lgn - CEN) = 16 points
// is the leaf size every task of the range is a leaf: it reads its entry,
// transforms its 16 points and emits them into their output block, forks
// nothing and joins nothing.  With no forks there is no scan and no block
// barrier, so each thread streams through its slots of the block's tiles on
// its own, its next entries in flight while a slot is transformed (the
// generic tile path waits for each tile's loads after its block scan).  Slot
// order is point order (task o is at slot lo + o), so a warp's loads stay
// coalesced.  lb holds LCAP bytes of shared memory for two buffers
// (fft_leaf_dyn_bytes).  With room for 16 points a thread, the next slot's
// points are copied there (cp.async, point r of every thread contiguous)
// while this slot is transformed, so a slot no longer waits a round trip for
// its inputs and no register holds them (2^24 points, 256 x 1: 1.19 -> 1.105
// ms, output bit-identical; holding them in registers spilled).  With room
// for 32, each warp also stages its 32 leaves' outputs (row per lane,
// columns XOR-swizzled against bank conflicts) and stores them as whole
// 128-byte blocks, two per instruction, instead of 16 scattered 8-byte
// stores per lane (128 x 1: 1.15 -> 1.12 ms; 512 x 1 with both buffers in
// dynamic shared memory 1.198 -> 1.094 ms).
template <int BS, int TPT, size_t LCAP>
__device__ __forceinline__ void fft_leaf_epoch(const Conf &c, float2 *lb, unsigned long long t0, unsigned long long step,
                                               uint32_t hi, uint32_t cen, Acc &acc) {
    const float2 *__restrict__ x = c.rp.fx;
    float2 *__restrict__ X = c.rp.fX;
    const uint32_t lgn = c.rp.lgn, d = cen;
    const uint32_t ntile = t0 < hi ? (uint32_t)((hi - t0 + step - 1ull) / step) : 0u, n = ntile * (uint32_t)TPT;
    const auto slot = [&](uint32_t i) {
        return t0 + (unsigned long long)(i / (uint32_t)TPT) * step + (unsigned long long)(i % (uint32_t)TPT) * BS +
               threadIdx.x;
    };
    // slot i's task: its code (0: none or not this thread's) and offset o
    const auto entry = [&](uint32_t i, uint32_t &cd, uint32_t &o) {
        cd = 0u;
        o = 0u;
        if (i < n) {
            const unsigned long long s = slot(i);
            if (s < hi) {
                cd = c.code[s];
                o = c.a0[s];
            }
        }
    };
    const auto inputs = [&](uint32_t cd, uint32_t o, float2 (&a)[16]) {
        if (task_type(cd, cen) == TREES_TASK_FFT) {
#pragma unroll
            for (int r = 0; r < 16; ++r) a[r] = x[o + ((uint32_t)fft_rev(r, 4) << d)];
        }
    };
    uint32_t c0, o0, c1, o1, c2, o2;
    entry(0u, c0, o0);
    entry(1u, c1, o1);
    if constexpr ((size_t)BS * 16u * sizeof(float2) <= LCAP) {
        float2 *pb = lb + threadIdx.x;  // point r at pb[r * BS]
        constexpr bool STAGE = (size_t)BS * 32u * sizeof(float2) <= LCAP;
        const auto issue = [&](uint32_t cd, uint32_t o) {
            if (task_type(cd, cen) == TREES_TASK_FFT) {
#pragma unroll
                for (int r = 0; r < 16; ++r) cp_async_8(pb + r * BS, x + o + ((uint32_t)fft_rev(r, 4) << d));
            }
            cp_async_commit();
        };
        // the leaf's 15 twiddles, once per block from the same function the combines use (bit-identical):
        // with the inputs prefetched the slots are bound by their instructions (2^24 points, 512 x 2:
        // 1.073 -> 1.058 ms; before the prefetch the same table changed nothing)
        __shared__ float2 tw[15];  // stage lm's twiddle k at tw[2^(lm-1) - 1 + k]
        for (uint32_t q = threadIdx.x; q < 15u; q += BS) {
            const uint32_t h = 1u << (31 - __clz(q + 1u));
            tw[q] = fft_twiddle(q + 1u - h, (uint32_t)(32 - __clz(h)));
        }
        __syncthreads();
        issue(c0, o0);
        for (uint32_t i = 0; i < n; ++i) {
            entry(i + 2u, c2, o2);
            cp_async_wait_all();  // this slot's points
            if (task_type(c0, cen) == TREES_TASK_FFT) {
                float2 a[16];
#pragma unroll
                for (int r = 0; r < 16; ++r) a[r] = pb[r * BS];
                acc.valid++;
#pragma unroll
                for (int q = 0; q < 16; q += 2) fft_bfly(a[q], a[q + 1], tw[0]);
                issue(c1, o1);  // every point has been used: the next slot's copies may overwrite them
#pragma unroll
                for (int lm = 2; lm <= 4; ++lm) {
                    const int h = 1 << (lm - 1);
#pragma unroll
                    for (int k = 0; k < h; ++k) {
                        const float2 w = tw[h - 1 + k];
#pragma unroll
                        for (int q = 0; q < 16; q += 2 * h) fft_bfly(a[q + k], a[q + k + h], w);
                    }
                }
                if constexpr (STAGE) {
                    float2 *ob = lb + BS * 16 + (threadIdx.x & ~31u) * 16u;
                    const uint32_t ln = threadIdx.x & 31u;
#pragma unroll
                    for (int k = 0; k < 16; ++k) ob[ln * 16u + ((uint32_t)k ^ (ln & 15u))] = a[k];
                } else {
                    const uint32_t dst = fft_block(o0, d, lgn);
#pragma unroll
                    for (int k = 0; k < 16; ++k) X[dst + k] = a[k];
                }
                c.code[(uint32_t)slot(i)] = 0u;
            } else {
                issue(c1, o1);
            }
            if constexpr (STAGE) {
                const float2 *ob = lb + BS * 16 + (threadIdx.x & ~31u) * 16u;
                const uint32_t ln = threadIdx.x & 31u;
                const uint32_t dst = task_type(c0, cen) == TREES_TASK_FFT ? fft_block(o0, d, lgn) : 0xFFFFFFFFu;
                __syncwarp();
#pragma unroll
                for (uint32_t j = 0; j < 16u; ++j) {
                    const uint32_t row = 2u * j + (ln >> 4), col = ln & 15u;
                    const uint32_t rd = __shfl_sync(0xffffffffu, dst, row);
                    const float2 v = ob[row * 16u + (col ^ (row & 15u))];
                    if (rd != 0xFFFFFFFFu) X[rd + col] = v;
                }
                __syncwarp();
            }
            c0 = c1;
            o0 = o1;
            c1 = c2;
            o1 = o2;
        }
        cp_async_wait_all();
    } else {  // no room for the buffer: each slot's points are loaded into registers when it runs
        for (uint32_t i = 0; i < n; ++i) {
            entry(i + 2u, c2, o2);  // two ahead: the entry
            if (task_type(c0, cen) == TREES_TASK_FFT) {
                float2 a[16];
                inputs(c0, o0, a);
                acc.valid++;
#pragma unroll
                for (int lm = 1; lm <= 4; ++lm) {
                    const int h = 1 << (lm - 1);
#pragma unroll
                    for (int k = 0; k < h; ++k) {
                        const float2 w = fft_twiddle((uint32_t)k, (uint32_t)lm);
#pragma unroll
                        for (int q = 0; q < 16; q += 2 * h) fft_bfly(a[q + k], a[q + k + h], w);
                    }
                }
                const uint32_t dst = fft_block(o0, d, lgn);
#pragma unroll
                for (int k = 0; k < 16; ++k) X[dst + k] = a[k];
                c.code[(uint32_t)slot(i)] = 0u;  // emitted: the entry is dead
            }
            c0 = c1;
            o0 = o1;
            c1 = c2;
            o1 = o2;
        }
    }
}

// The FFT's other epochs above the leaves, for the same reason (every task
// of an epoch has depth CEN, so the epoch's width fixes its forks and maps).
// A fork epoch: each task (o, d) writes its two children at their point
// offsets, fbase + o and fbase + o + 2^d (as commit_task places them), and
// becomes its combine; the epoch's forks, two per task, are added to
// nextFreeCore by one thread for the whole grid (Sec. 5.2.3's cooperative
// allocation, the group being the epoch).  Returns whether this thread's
// tasks joined.
template <int BS, int TPT>
__device__ __forceinline__ bool fft_fork_epoch(const Conf &c, Ctl *ctl, unsigned long long t0, unsigned long long step,
                                               uint32_t lo, uint32_t hi, uint32_t cen, uint32_t base, uint32_t ep,
                                               uint32_t e, Acc &acc) {
    const uint32_t fe = enc(cen + 1u, TREES_TASK_FFT), fj = enc(cen, TREES_TASK_FFT_COMBINE);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        atomicAdd(fork_ctr(ctl, ep), 2u * (hi - lo));
        if ((unsigned long long)base + 2ull * (hi - lo) > c.cap) set_err(ctl, TREES_ERR_CAPACITY, e);
    }
    bool joined = false;
    uint32_t cd[TPT], o[TPT], d[TPT];  // the current tile's entries; the next tile's load while it is written
    const auto load = [&](unsigned long long tt) {
#pragma unroll
        for (int k = 0; k < TPT; ++k) {
            const unsigned long long s = tt + (unsigned long long)k * BS + threadIdx.x;
            const bool in = tt < hi && s < hi;
            cd[k] = in ? c.code[s] : 0u;
            o[k] = in ? c.a0[s] : 0u;
            d[k] = in ? c.a1[s] : 0u;
        }
    };
    load(t0);
    for (; t0 < hi; t0 += step) {
        uint32_t pc[TPT], po[TPT], pd[TPT];
#pragma unroll
        for (int k = 0; k < TPT; ++k) {
            pc[k] = cd[k];
            po[k] = o[k];
            pd[k] = d[k];
        }
        load(t0 + step);
#pragma unroll
        for (int k = 0; k < TPT; ++k) {
            if (task_type(pc[k], cen) != TREES_TASK_FFT) continue;
            const uint32_t s = (uint32_t)(t0 + (unsigned long long)k * BS + threadIdx.x);
            const uint32_t c0 = base + po[k], c1 = c0 + (1u << pd[k]);
            if ((unsigned long long)c1 >= c.cap) continue;  // the capacity error is set above
            c.code[c0] = fe;
            c.a0[c0] = po[k];
            c.a1[c0] = pd[k] + 1u;
            c.code[c1] = fe;
            c.a0[c1] = po[k] + (1u << pd[k]);
            c.a1[c1] = pd[k] + 1u;
            c.code[s] = fj;
            acc.valid++;
            acc.joins++;
            joined = true;
        }
    }
    return joined;
}

// A combine epoch whose combines are maps: each task schedules the map over
// its 2^(lgm-1) butterflies and is done; the epoch's maps (one descriptor
// count per task, N/2 butterflies in all) are added to the map counter by one
// thread for the whole grid (the combine maps need no descriptors).  Every
// entry of the range is a combine of this epoch (the fork epoch at depth CEN
// made each task of its range its combine), so the count is the width and
// no code is read; none is marked done either: a combine schedules no join,
// so its range is never revisited (the reading taken for fib's sums).
// Measured: 2^24 points, 512 x 1 1.082 -> 1.070 ms, 256 x 1 1.104 -> 1.092 ms.
template <int BS, int TPT>
__device__ __forceinline__ void fft_combine_epoch(const Conf &c, Ctl *ctl, unsigned long long t0,
                                                  unsigned long long step, uint32_t lo, uint32_t hi, uint32_t cen,
                                                  uint32_t ep, Acc &acc) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        const unsigned long long nd = hi - lo;
        atomicAdd(&ctl->me_ctr[ep], (nd << 40) | (nd << (c.rp.lgn - cen - 1u)));
    }
    for (; t0 < hi; t0 += step) {
#pragma unroll
        for (int k = 0; k < TPT; ++k) {
            if (t0 + (unsigned long long)k * BS + threadIdx.x < hi) {
                acc.valid++;
                acc.maps++;
            }
        }
    }
}

// Step 2: write the children into [child, child + n) for epoch CEN+1 and turn
// the task into its join continuation.  Returns 1 if it joined.
// fbase: the first slot of the epoch's fork range (the FFT places its
// children by their point offset, see below).
template <uint32_t PM, typename UP = NoUserProgram>
__device__ __forceinline__ uint32_t commit_task(const Conf &c, const RunParams &rp, const Plan &p, uint32_t cen,
                                                 uint32_t child, uint32_t fbase = 0u) {
    const uint32_t s = p.s;
    const uint32_t fe = enc(cen + 1u, 0u);
    if constexpr ((PM & PM_USER) != 0u) {  // children in the program's order, then the continuation
        const trees_user_env env = user_env(c);
        const trees_user_task t = {s, p.t, p.a0, p.a1, child, cen};
        for (uint32_t i = 0; i < p.n; ++i) {
            const trees_user_child ch = UP::child(t, i, env);
            const bool ok = ch.type >= 1u && ch.type <= (uint32_t)TREES_NUM_TASK_TYPES;
            c.code[child + i] = ok ? fe + ch.type : 0u;
            c.a0[child + i] = ch.a0;
            c.a1[child + i] = ch.a1;
        }
        const trees_user_child j = UP::join(t, env);
        if (j.type >= 1u && j.type <= (uint32_t)TREES_NUM_TASK_TYPES) {
            c.link[s] = child;
            c.a0[s] = j.a0;
            c.a1[s] = j.a1;
            c.code[s] = enc(cen, j.type);
            return 1u;
        }
        c.code[s] = 0u;
        return 0u;
    }
    if constexpr ((PM & PM_FIB) != 0u) {
        if (p.t == TREES_TASK_FIB) {
            c.code[child] = fe + TREES_TASK_FIB;
            c.a0[child] = p.a0 - 1u;
            c.code[child + 1] = fe + TREES_TASK_FIB;
            c.a0[child + 1] = p.a0 - 2u;
            c.link[s] = child;
            c.code[s] = enc(cen, TREES_TASK_FIB_SUM);
            return 1u;
        }
    }
    if constexpr ((PM & PM_MS) != 0u) {
        if (p.t == TREES_TASK_MS_SPLIT) {
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
    }
    if constexpr ((PM & PM_NQ) != 0u) {
        if (p.t == TREES_TASK_NQ_ROW) {
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
    }
    if constexpr ((PM & PM_FFT) != 0u) {
        // Every task of an FFT epoch has the same depth d and forks two, so the
        // epoch forks exactly the 2^(d+1) tasks of depth d+1 into
        // [fbase, fbase + 2^(d+1)); child o' goes to slot fbase + o'.  Slot order
        // is then point order, and the leaves' strided loads are coalesced
        // (x[o + j 2^d] for consecutive o).  `child` (this task's share of the
        // reservation) is not needed: the reservation covers the same range.
        if (p.t == TREES_TASK_FFT) {  // even-numbered points, then odd-numbered; join the combine (o, d)
            const uint32_t c0 = fbase + p.a0, c1 = c0 + (1u << p.a1);
            c.code[c0] = fe + TREES_TASK_FFT;
            c.a0[c0] = p.a0;
            c.a1[c0] = p.a1 + 1u;
            c.code[c1] = fe + TREES_TASK_FFT;
            c.a0[c1] = p.a0 + (1u << p.a1);
            c.a1[c1] = p.a1 + 1u;
            c.code[s] = enc(cen, TREES_TASK_FFT_COMBINE);
            return 1u;
        }
    }
    if constexpr ((PM & PM_TRAV) != 0u) {
        if (p.t == TREES_TASK_PO || p.t == TREES_TASK_PRE) {
            const int32_t node = (int32_t)p.a0;
            c.code[child] = fe + p.t;
            c.a0[child] = (uint32_t)__ldg(rp.right + node);
            c.code[child + 1] = fe + p.t;
            c.a0[child + 1] = (uint32_t)__ldg(rp.left + node);
            if (p.t == TREES_TASK_PRE) return 0u;
            c.link[s] = child;
            c.code[s] = enc(cen, TREES_TASK_PO_AFTER);
            return 1u;
        }
    }
    return 0u;
}

// Map allocation for one tile: one packed block scan per map list and one
// atomic per list per block, then the descriptor writes.  Tiled maps (leaf
// sort, merge) also get a tile -> descriptor table, written cooperatively;
// element maps (BFS expansion) record, for every expansion tile that starts
// inside them, that they are the tile's first descriptor.
template <int BS, int TPT>
__device__ void map_alloc(const Conf &c, Ctl *ctl, Smem<BS> &sm, const Plan (&p)[TPT], uint32_t cen, uint32_t ep,
                          uint32_t e, uint32_t job, Acc &acc) {
    unsigned long long qa = 0ull, qb = 0ull;
#pragma unroll
    for (int k = 0; k < TPT; ++k) {
        if (p[k].m == MAP_LEAF_SORT || p[k].m == MAP_MERGE || p[k].m == MAP_USER) qa += (1ull << 40) | p[k].n;
        else if (p[k].m == MAP_EXPAND || p[k].m == MAP_FFT) qb += (1ull << 40) | p[k].n;
    }
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
            uint32_t rank = (uint32_t)(ea >> 40), toff = (uint32_t)(ea & CTR_LOW_MASK);
#pragma unroll
            for (int k = 0; k < TPT; ++k) {
                if (p[k].m != MAP_LEAF_SORT && p[k].m != MAP_MERGE && p[k].m != MAP_USER) continue;
                const uint32_t di = dbase + rank;
                c.mt_kind[di] = p[k].m;
                c.mt_a[di] = p[k].a0;
                c.mt_b[di] = p[k].a1;
                c.mt_c[di] = p[k].m == MAP_USER ? p[k].s : cen;
                c.mt_job[di] = job;
                c.mt_tilebase[di] = tbase + toff;
                acc.maps++;
                ++rank;
                toff += p[k].n;
            }
        }
    }
    if (tb) {
        const unsigned long long g = sm.bc64[1];
        const uint32_t dbase = (uint32_t)(g >> 40);
        const unsigned long long ebase = g & CTR_LOW_MASK;
        const uint32_t ndesc = (uint32_t)(tb >> 40);
        const unsigned long long nel = tb & CTR_LOW_MASK;
        constexpr uint32_t ET = expand_tile_len(BS);
        const unsigned long long tiles_end = (ebase + nel + ET - 1) / ET;
        const bool fits = (unsigned long long)dbase + ndesc <= c.mcap && ebase + nel < 0xFFFFFFFFull &&
                          tiles_end <= c.mcap;
        if (!fits) {
            if (threadIdx.x == 0) set_err(ctl, TREES_ERR_CAPACITY, e);
        } else {
            uint32_t di = dbase + (uint32_t)(eb >> 40);
            uint32_t b = (uint32_t)(ebase + (eb & CTR_LOW_MASK));
#pragma unroll
            for (int k = 0; k < TPT; ++k) {
                if (p[k].m == MAP_FFT) acc.maps++;  // counted; fft_combine_map needs no descriptor
                if (p[k].m != MAP_EXPAND) continue;
                c.me_v[di] = p[k].a0;
                c.me_base[di] = b;
                c.me_job[di] = job;
                c.me_src[di] = p[k].a1;  // the vertex (SSSP reads its distance)
                for (uint32_t t = (b + ET - 1u) / ET; t * ET < b + p[k].n; ++t)
                    c.me_tfd[t] = di;
                acc.maps++;
                ++di;
                b += p[k].n;
            }
        }
    }
    __syncthreads();
}

// One Phase-2 tile: TPT * BS consecutive slots of the current range starting
// at t0; slot t0 + k*BS + tid belongs to this thread.  All TV loads of the
// tile are issued before any task runs, one vector scan hands every (k,
// thread) its children's offset in k-major order (so the children of a warp
// are written contiguously), and one atomic per block reserves them.
// Which columns Phase 2 reads together with `code`: LOAD_ON_DEMAND reads
// them after decoding the type; LOAD_FRESH (a range of freshly forked tasks)
// and LOAD_JOIN (a join range revisited) issue the columns such tasks use in
// the same round trip as the code.
constexpr int LOAD_ON_DEMAND = 0, LOAD_FRESH = 1, LOAD_JOIN = 2;

// The TV columns of one tile, loaded ahead of running it.
template <int TPT>
struct TileLoad {
    uint32_t cd[TPT], a0[TPT], a1[TPT], lk[TPT];
};

template <int BS, int TPT, uint32_t PM>
__device__ __forceinline__ void tile_load(const Conf &c, unsigned long long t0, uint32_t hi, int mode,
                                          TileLoad<TPT> &L) {
    constexpr bool fresh_a1 = (PM & (PM_MS | PM_NQ | PM_FFT | PM_USER)) != 0u;
    constexpr bool join_a0 = (PM & (PM_MS | PM_NQ | PM_TRAV | PM_FFT | PM_USER)) != 0u;
    constexpr bool join_link = (PM & (PM_FIB | PM_NQ | PM_USER)) != 0u;
    const bool sa0 = mode == LOAD_FRESH || (mode == LOAD_JOIN && join_a0);
    const bool sa1 = (mode == LOAD_FRESH || mode == LOAD_JOIN) && fresh_a1;
    const bool slk = mode == LOAD_JOIN && join_link;
#pragma unroll
    for (int k = 0; k < TPT; ++k) {
        const unsigned long long s = t0 + (unsigned long long)k * BS + threadIdx.x;
        const bool in = s < hi;
        L.cd[k] = in ? c.code[s] : 0u;
        L.a0[k] = in && sa0 ? c.a0[s] : 0u;
        L.a1[k] = in && sa1 ? c.a1[s] : 0u;
        L.lk[k] = in && slk ? c.link[s] : 0u;
    }
}

// What one Phase-2 tile tells its block: the forks of the whole tile (the
// same on every thread), whether this thread's tasks scheduled a join, and
// whether the fork allocation ran out of slots (the same on every thread).
struct TileOut {
    uint32_t forks;
    bool joined;
    bool over;
};

// Join-operand prefetch for fib (Sec. 4.1's continuation reads its children's
// results through `link`): while a join tile runs, the results its successor
// tile's sums will read are copied into shared memory asynchronously, so the
// successor's sums need no dependent round trip.  jr_use: this tile's
// operands were prefetched into jr[par]; pf: the successor tile's columns
// (its operands go to jr[par ^ 1]), or null.
template <int BS, int TPT, uint32_t PM>
__device__ __forceinline__ constexpr bool join_prefetch() {
    return (PM & PM_FIB) != 0u && BS * TPT <= (int)JR_SLOTS;
}

template <int BS, int TPT, uint32_t PM, typename UP = NoUserProgram>
__device__ __forceinline__ TileOut epoch_tile(const Conf &c, Ctl *ctl, Smem<BS> &sm, unsigned long long t0, uint32_t hi,
                                           uint32_t cen, uint32_t base, uint32_t ep, uint32_t e, Acc &acc, int par,
                                           int mode, const TileLoad<TPT> &L, bool known, uint32_t known_off,
                                           bool jr_use = false, const TileLoad<TPT> *pf = nullptr) {
    constexpr bool fresh_a1 = (PM & (PM_MS | PM_NQ | PM_FFT | PM_USER)) != 0u;
    constexpr bool join_a0 = (PM & (PM_MS | PM_NQ | PM_TRAV | PM_FFT | PM_USER)) != 0u;
    constexpr bool join_link = (PM & (PM_FIB | PM_NQ | PM_USER)) != 0u;
    const bool sa0 = mode == LOAD_FRESH || (mode == LOAD_JOIN && join_a0);
    const bool sa1 = (mode == LOAD_FRESH || mode == LOAD_JOIN) && fresh_a1;
    const bool slk = mode == LOAD_JOIN && join_link;
    Plan p[TPT];
    uint32_t a0v[TPT], a1v[TPT], lkv[TPT];
#pragma unroll
    for (int k = 0; k < TPT; ++k) {
        const uint32_t s = (uint32_t)(t0 + (unsigned long long)k * BS + threadIdx.x);
        const uint32_t t = task_type(L.cd[k], cen);  // invalid or stale entries exit at once (Sec. 5.3)
        p[k].s = s;
        p[k].t = t;
        p[k].n = 0u;
        p[k].m = 0u;
        a0v[k] = needs_a0(t) && !sa0 ? c.a0[s] : L.a0[k];
        a1v[k] = needs_a1(t) && !sa1 ? c.a1[s] : L.a1[k];
        lkv[k] = needs_link(t) && !slk ? c.link[s] : L.lk[k];
    }
    uint32_t nf[TPT];
    int hasmap = 0;
    if constexpr (join_prefetch<BS, TPT, PM>()) {
        if (jr_use) cp_async_wait_all();  // this thread's operands for this tile have landed
    }
#pragma unroll
    for (int k = 0; k < TPT; ++k) {
        if (p[k].t) {
            acc.valid++;
            bool done = false;
            if constexpr (join_prefetch<BS, TPT, PM>()) {
                if (jr_use && p[k].t == TREES_TASK_FIB_SUM) {
                    const unsigned long long *r = sm.u.jr[par][k * BS + threadIdx.x];
                    c.result[p[k].s] = r[0] + r[1];
                    c.code[p[k].s] = 0u;
                    done = true;
                }
            }
            if (!done) plan_task<PM, merge_tile(BS), UP>(c, c.rp, p[k], cen, e, a0v[k], a1v[k], lkv[k]);
        }
        nf[k] = forks_of(p[k]);
        hasmap |= p[k].m != 0u;
    }
    if constexpr (join_prefetch<BS, TPT, PM>()) {
        if (pf) {  // the successor tile's sums: copy their operands now (its links have arrived by now)
#pragma unroll
            for (int k = 0; k < TPT; ++k) {
                if (task_type(pf->cd[k], cen) == TREES_TASK_FIB_SUM) {
                    unsigned long long *r = sm.u.jr[par ^ 1][k * BS + threadIdx.x];
                    cp_async_8(r, c.result + pf->lk[k]);
                    cp_async_8(r + 1, c.result + pf->lk[k] + 1);
                }
            }
            cp_async_commit();
        }
    }
    uint32_t ex[TPT], tot[TPT];
    int anymap;
    if constexpr ((PM & ~(PM_BFS | PM_SSSP)) == 0u) {
        // a visit or relax task never forks itself (its map's tiles fork): no fork scan, and the
        // map allocation's own scan sees whether the tile maps (R-MAT 22, BFS 512 x 1 0.665 ->
        // 0.656 ms, SSSP 512 x 1 2.15 -> 2.13 ms)
#pragma unroll
        for (int k = 0; k < TPT; ++k) ex[k] = tot[k] = 0u;
        anymap = 1;
    } else {
        block_scan_vec<BS, TPT>(nf, ex, tot, hasmap, &anymap, sm, par);
    }
    uint32_t all = 0;
#pragma unroll
    for (int k = 0; k < TPT; ++k) all += tot[k];
    TileOut out = {all, false, false};
    if (all) {
        // known: this block forks every child of the epoch (the range is its own), so the tile's
        // children start at known_off, the forks of its earlier tiles, and the count is published
        // without waiting for the atomic's answer
        uint32_t b0 = known ? known_off : 0u, over0 = 0u;
        if (known) {
            over0 = (unsigned long long)base + known_off + all > c.cap;
            if (threadIdx.x == 0) {
                atomicAdd(fork_ctr(ctl, ep), all);  // result unused: a fire-and-forget reduction
                if (over0) set_err(ctl, TREES_ERR_CAPACITY, e);
            }
        } else {
            if (threadIdx.x == 0) {
                const uint32_t b = atomicAdd(fork_ctr(ctl, ep), all);  // one atomic per block (Sec. 5.2.3)
                const bool over = (unsigned long long)base + b + all > c.cap;
                if (over) set_err(ctl, TREES_ERR_CAPACITY, e);
                sm.bc32[par] = b;
                sm.bc32[2 + par] = over;
            }
            __syncthreads();
            b0 = sm.bc32[par];
            over0 = sm.bc32[2 + par];
        }
        uint32_t joined = 0u;
        if (!over0) {
            uint32_t kbase = base + b0;
#pragma unroll
            for (int k = 0; k < TPT; ++k) {
                if (nf[k]) joined += commit_task<PM, UP>(c, c.rp, p[k], cen, kbase + ex[k], base);
                kbase += tot[k];
            }
        }
        acc.joins += joined;
        out.joined = joined != 0u;  // the caller sets joinScheduled once per block (publish_join)
        out.over = over0 != 0u;
    }
    if constexpr ((PM & PM_MAPS) != 0u) {
        if (anymap) map_alloc<BS, TPT>(c, ctl, sm, p, cen, ep, e, 0u, acc);
    }
    if constexpr ((PM & PM_FFT) != 0u) {
        if (PM == PM_FFT || c.rp.program == TREES_PROG_FFT) fft_task_bodies<PM, TPT>(c.rp, p);
    }
    return out;
}

// joinScheduled (Sec. 5.2.3) for one block: set once if any of its threads
// joined this epoch, instead of once per warp and tile (every store to the
// flag shares an L2 line with the fork counter's atomics).  Every thread of
// the block calls it.
__device__ __forceinline__ void publish_join(Ctl *ctl, uint32_t ep, bool joined) {
    if (__syncthreads_or(joined) && threadIdx.x == 0) ctl->join[ep] = 1u;
}

// Programs whose join continuations never fork and never map (fib's sum,
// N-Queens' sum, the traversals' visitAfter): a join range revisited holds
// only continuations (each task of the range ran when the range was fresh
// and either died or rewrote itself as its continuation; no other entry of
// the range gets the range's epoch number), so its tiles allocate nothing and
// need no block scan.
template <uint32_t PM>
__host__ __device__ constexpr bool joins_never_fork() {
    return (PM & ~(PM_FIB | PM_NQ | PM_TRAV)) == 0u;
}

// One tile of a join range of such a program: every thread runs its own
// continuations with no block barrier, so the warps of a block (and the
// tiles of a thread) stream independently.  The join-operand prefetch works
// as in epoch_tile: jr_use says this tile's operands are in jr[par], pf is the
// successor tile (its operands go to jr[par ^ 1]); a thread only reads the
// copies it issued itself.
template <int BS, int TPT, uint32_t PM>
__device__ __forceinline__ void join_tile(const Conf &c, Smem<BS> &sm, unsigned long long t0, uint32_t cen, uint32_t e,
                                          Acc &acc, int par, const TileLoad<TPT> &L, bool jr_use,
                                          const TileLoad<TPT> *pf) {
    static_assert(joins_never_fork<PM>(), "only for programs whose continuations neither fork nor map");
    // the columns tile_load brought in LOAD_JOIN mode for these programs
    constexpr bool join_a0 = (PM & (PM_NQ | PM_TRAV)) != 0u;
    constexpr bool join_a1 = (PM & PM_NQ) != 0u;
    constexpr bool join_link = (PM & (PM_FIB | PM_NQ)) != 0u;
    if constexpr (join_prefetch<BS, TPT, PM>()) {
        if (jr_use) cp_async_wait_all();  // this thread's operands for this tile have landed
    }
#pragma unroll
    for (int k = 0; k < TPT; ++k) {
        const uint32_t s = (uint32_t)(t0 + (unsigned long long)k * BS + threadIdx.x);
        const uint32_t t = task_type(L.cd[k], cen);
        if (!t) continue;
        acc.valid++;
        if constexpr (join_prefetch<BS, TPT, PM>()) {
            if (jr_use && t == TREES_TASK_FIB_SUM) {
                const unsigned long long *r = sm.u.jr[par][k * BS + threadIdx.x];
                c.result[s] = r[0] + r[1];
                c.code[s] = 0u;
                continue;
            }
        }
        Plan p;
        p.s = s;
        p.t = t;
        p.n = 0u;
        p.m = 0u;
        const uint32_t a0 = needs_a0(t) && !join_a0 ? c.a0[s] : L.a0[k];
        const uint32_t a1 = needs_a1(t) && !join_a1 ? c.a1[s] : L.a1[k];
        const uint32_t lk = needs_link(t) && !join_link ? c.link[s] : L.lk[k];
        plan_task<PM, merge_tile(BS)>(c, c.rp, p, cen, e, a0, a1, lk);
    }
    if constexpr (join_prefetch<BS, TPT, PM>()) {
        if (pf) {  // the successor tile's sums: copy their operands now
#pragma unroll
            for (int k = 0; k < TPT; ++k) {
                if (task_type(pf->cd[k], cen) == TREES_TASK_FIB_SUM) {
                    unsigned long long *r = sm.u.jr[par ^ 1][k * BS + threadIdx.x];
                    cp_async_8(r, c.result + pf->lk[k]);
                    cp_async_8(r + 1, c.result + pf->lk[k] + 1);
                }
            }
            cp_async_commit();
        }
    }
}

// A fresh range of fib tasks (Sec. 6.2: a leaf emits, an internal task forks
// fib(n-1), fib(n-2) and joins their sum): the block's tiles (t0, t0 + step,
// ...), taken in chunks of up to FIB_CHUNK_SLOTS / tile tiles, each in two
// passes with one slot reservation between them:
//  1. count: every warp streams through the chunk's tiles on its own (no
//     block barrier): it loads code and n, lets the leaves emit in their own
//     slot (Sec. 4.3.2), rewrites the internal tasks as their continuations
//     (code, and a zero result the join overwrites, so the code and result
//     rows are written whole in this pass), and records with one ballot per
//     slot row which lanes fork (fib forks exactly two children, so a warp's
//     prefix is twice a popcount), plus each internal task's n, in shared
//     memory;
//  2. one block scan over the per-warp fork counts and one atomic on
//     nextFreeCore for the whole chunk (Sec. 5.2.3's cooperative allocation:
//     a scan, then a single atomic for the group);
//  3. write: every warp writes its internal tasks' children (k-major, so a
//     warp's children are contiguous) and the link row of its slots (zero for
//     the leaves), from shared memory alone (no loads, no block barrier).
// A row of a column written partly in one pass and partly much later leaves
// partly written 32-byte sectors in L2; written whole (or by both passes of
// one chunk) it does not: fib(34) at 512 x 2 went 0.427 -> 0.418 ms.
// Returns whether this thread's tasks joined.
constexpr uint32_t FIB_CHUNK_SLOTS = 16384;  // slots per chunk: their n fit a 16 KB byte array

template <int BS, int TPT>
__host__ __device__ constexpr uint32_t fib_chunk_tiles() {
    return FIB_CHUNK_SLOTS / (uint32_t)(BS * TPT) < 64u ? FIB_CHUNK_SLOTS / (uint32_t)(BS * TPT) : 64u;
}

// Tiles of loads a thread keeps in flight in the count pass (registers:
// 2 * TPT words per tile).  Blocks of 512 threads run one per SM with up to
// 128 registers a thread, so they hold eight slots' loads in flight (fib(34)
// at 512 x 2: 0.4342 ms with four tiles against 0.4403 ms with two); smaller
// blocks share the SM's registers with two or more others, and 1024-thread
// blocks have 64 a thread, so they keep two tiles (four measured 0.4874
// against 0.469 ms at 256 x 2).
template <int BS, int TPT>
__host__ __device__ constexpr int fib_prefetch_tiles() {
    return TPT == 1 ? 8 : BS == 512 ? 8 / TPT : 2;
}

template <int BS, int TPT>
struct FibChunk {
    static constexpr uint32_t CT = fib_chunk_tiles<BS, TPT>(), NW = BS / 32;
    uint8_t n[CT * BS * TPT];       // n of each slot's task (internal tasks only are read)
    uint32_t mask[CT * TPT * NW];   // per (tile, slot row, warp): lanes whose task forks
    uint32_t off[CT * TPT * NW];    // their exclusive prefix of children inside the chunk
};

template <int BS, int TPT>
__device__ __forceinline__ bool fib_fresh_tiles(const Conf &c, Ctl *ctl, Smem<BS> &sm, unsigned long long t0,
                                                unsigned long long step, uint32_t hi, uint32_t cen, uint32_t base,
                                                uint32_t ep, uint32_t e, Acc &acc) {
    using FC = FibChunk<BS, TPT>;
    constexpr uint32_t CT = FC::CT, NW = FC::NW, TILE = BS * TPT;
    static_assert(sizeof(FC) <= sizeof(sm.u), "the chunk's records fit the shared union");
    static_assert(CT >= 1u, "at least one tile per chunk");
    FC &fc = *reinterpret_cast<FC *>(&sm.u);
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;  // lanes below this one
    const uint32_t fe = enc(cen + 1u, TREES_TASK_FIB), fj = enc(cen, TREES_TASK_FIB_SUM);
    bool joined = false;
    for (; t0 < hi; t0 += (unsigned long long)CT * step) {  // one chunk per iteration (block-uniform)
        // tiles of this chunk: t0 + j * step, j < nt
        const uint32_t nt = (uint32_t)min((unsigned long long)CT, (hi - t0 + step - 1ull) / step);
        // ---- pass 1: count.  The loads of the next PD-1 tiles are in flight while a tile is decoded
        // (a ring of PD tiles of code and n in registers).
        constexpr int PD = fib_prefetch_tiles<BS, TPT>();
        uint32_t rc[PD][TPT], rn[PD][TPT];
#pragma unroll
        for (int u = 0; u < PD - 1; ++u) {
#pragma unroll
            for (int k = 0; k < TPT; ++k) {
                const unsigned long long s = t0 + (unsigned long long)u * step + (unsigned long long)k * BS + threadIdx.x;
                const bool in = (uint32_t)u < nt && s < hi;
                rc[u][k] = in ? c.code[s] : 0u;
                rn[u][k] = in ? c.a0[s] : 0u;
            }
        }
        for (uint32_t j0 = 0; j0 < nt; j0 += PD) {
#pragma unroll
            for (int u = 0; u < PD; ++u) {
                const uint32_t j = j0 + (uint32_t)u;
                if (j < nt) {  // block-uniform
                {   // tile j + PD - 1 into the ring slot tile j - 1 used
                    const int un = (u + PD - 1) % PD;  // a constant once the loop is unrolled
                    const unsigned long long tn = t0 + (unsigned long long)(j + PD - 1) * step;
#pragma unroll
                    for (int k = 0; k < TPT; ++k) {
                        const unsigned long long s = tn + (unsigned long long)k * BS + threadIdx.x;
                        const bool in = j + PD - 1 < nt && s < hi;
                        rc[un][k] = in ? c.code[s] : 0u;
                        rn[un][k] = in ? c.a0[s] : 0u;
                    }
                }
                const unsigned long long tj = t0 + (unsigned long long)j * step;
#pragma unroll
                for (int k = 0; k < TPT; ++k) {
                    const uint32_t s = (uint32_t)(tj + (unsigned long long)k * BS + threadIdx.x);  // < hi when valid
                    const uint32_t t = task_type(rc[u][k], cen), n = rn[u][k];
                    bool fork = false;
                    if (t == TREES_TASK_FIB) {
                        acc.valid++;
                        if (n < 2u || n <= c.rp.cutoff) {  // a leaf emits: fib(n) in its own slot, entry dead
                            c.result[s] = n < 2u ? (unsigned long long)n : fib_leaf(n);
                            c.code[s] = 0u;
                        } else {  // its continuation (its result is written by the join)
                            c.result[s] = 0ull;
                            c.code[s] = fj;
                            fork = true;
                        }
                    } else if (t) {  // not produced in a fresh range; run it as the general path would
                        acc.valid++;
                        Plan p;
                        p.s = s;
                        p.t = t;
                        p.n = 0u;
                        p.m = 0u;
                        plan_task<PM_FIB, merge_tile(BS)>(c, c.rp, p, cen, e, n, 0u, c.link[s]);
                    }
                    const uint32_t m = __ballot_sync(0xffffffffu, fork);
                    if (lane == 0u) fc.mask[(j * TPT + k) * NW + wid] = m;
                    if (fork) fc.n[j * TILE + k * BS + threadIdx.x] = (uint8_t)n;  // n <= 93 (host check)
                }
                }
            }
        }
        __syncthreads();
        // ---- pass 2: one scan over the chunk's per-warp counts, one reservation for the chunk
        constexpr uint32_t NE = CT * TPT * NW, PER = (NE + BS - 1u) / BS;
        const uint32_t ne = nt * TPT * NW;
        uint32_t loc[PER], lsum = 0u;
#pragma unroll
        for (uint32_t q = 0; q < PER; ++q) {
            const uint32_t i = threadIdx.x * PER + q;
            loc[q] = i < ne ? 2u * (uint32_t)__popc(fc.mask[i]) : 0u;
            lsum += loc[q];
        }
        uint32_t total;
        int any;
        uint32_t pre = block_scan_u32<BS>(lsum, 0, &total, &any, sm);
#pragma unroll
        for (uint32_t q = 0; q < PER; ++q) {
            const uint32_t i = threadIdx.x * PER + q;
            if (i < ne) fc.off[i] = pre;
            pre += loc[q];
        }
        if (threadIdx.x == 0) {
            const uint32_t b = total ? atomicAdd(fork_ctr(ctl, ep), total) : 0u;  // one atomic per chunk
            const bool over = (unsigned long long)base + b + total > c.cap;
            if (over) set_err(ctl, TREES_ERR_CAPACITY, e);
            sm.bc32[0] = b;
            sm.bc32[1] = over;
        }
        __syncthreads();
        // ---- pass 3: children and continuations, warp by warp
        if (total && !sm.bc32[1]) {
            const uint32_t cbase = base + sm.bc32[0];
            for (uint32_t j = 0; j < nt; ++j) {
#pragma unroll
                for (int k = 0; k < TPT; ++k) {
                    const uint32_t i = (j * TPT + k) * NW + wid;
                    const uint32_t m = fc.mask[i];
                    const unsigned long long sl = t0 + (unsigned long long)j * step + (unsigned long long)k * BS +
                                                  threadIdx.x;
                    if (!((m >> lane) & 1u)) {
                        if (sl < hi) c.link[(uint32_t)sl] = 0u;  // the link row is written whole
                        continue;
                    }
                    const uint32_t s = (uint32_t)sl;
                    const uint32_t n = fc.n[j * TILE + k * BS + threadIdx.x];
                    const uint32_t child = cbase + fc.off[i] + 2u * (uint32_t)__popc(m & lt);
                    c.code[child] = fe;
                    c.a0[child] = n - 1u;
                    c.code[child + 1] = fe;
                    c.a0[child + 1] = n - 2u;
                    c.link[s] = child;
                    acc.joins++;
                    joined = true;
                }
            }
        }
        __syncthreads();  // the records are the next chunk's
    }
    return joined;
}

// The join ranges of fib (Sec. 6.2's sum continuations, Sec. 4.1: a join
// reads its children's results through its link), all of the block's tiles
// (t0, t0 + step, ...) with a two-level pipeline of asynchronous copies
// (cp.async) per thread: the code and link columns of the thread's slots of
// tile j+LA and the children's two results of tile j+LB's sums (their links
// are in shared memory by then) are in flight while tile j is summed.  Each
// thread reads only what it copied, so no block barrier is needed, and no
// register or load scoreboard holds the data in flight.  `ring` is this
// block's dynamic shared memory: NA stages of (code, link) and NB stages of
// result pairs, TILE slots each.
template <int BS, int TPT, int NA, int NB>
__device__ __forceinline__ void fib_join_tiles(const Conf &c, unsigned long long t0, unsigned long long step,
                                               uint32_t hi, uint32_t cen, uint32_t e, Acc &acc, uint32_t *ring) {
    constexpr uint32_t TILE = BS * TPT;
    constexpr int LA = NA - 1, LB = NB - 1;
    static_assert(LA > LB && LB >= 1, "links land before the operands they locate are copied");
    uint32_t *const ra = ring;  // stage q: code at [2 q TILE + slot], link at [(2 q + 1) TILE + slot]
    unsigned long long *const rb = reinterpret_cast<unsigned long long *>(ring + 2u * NA * TILE);  // 2 per slot
    const uint32_t nt = t0 < hi ? (uint32_t)((hi - t0 + step - 1ull) / step) : 0u;  // this block's tiles
    const auto slot = [&](uint32_t j, int k) { return t0 + (unsigned long long)j * step + (unsigned long long)k * BS + threadIdx.x; };
    const auto issue_a = [&](uint32_t j) {
        if (j < nt) {
            uint32_t *q = ra + (j % (uint32_t)NA) * 2u * TILE + threadIdx.x;
#pragma unroll
            for (int k = 0; k < TPT; ++k) {
                const unsigned long long s = slot(j, k);
                if (s < hi) {
                    cp_async_4(q + k * BS, c.code + s);
                    cp_async_4(q + TILE + k * BS, c.link + s);
                }
            }
        }
        cp_async_commit();
    };
    const auto issue_b = [&](uint32_t j) {  // tile j's (code, link) have landed
        if (j < nt) {
            const uint32_t *q = ra + (j % (uint32_t)NA) * 2u * TILE + threadIdx.x;
            unsigned long long *r = rb + 2u * ((j % (uint32_t)NB) * TILE + threadIdx.x);
#pragma unroll
            for (int k = 0; k < TPT; ++k) {
                if (slot(j, k) < hi && task_type(q[k * BS], cen) == TREES_TASK_FIB_SUM) {
                    const uint32_t lk = q[TILE + k * BS];
                    cp_async_8(r + 2 * k * BS, c.result + lk);
                    cp_async_8(r + 2 * k * BS + 1, c.result + lk + 1);
                }
            }
        }
        cp_async_commit();
    };
    // prologue: the links of tiles 0..LB-1 land, then their operands are copied; tiles up to LA-1 stream in.
    // Each operand group is followed by an empty group, standing for the (code, link) group the loop
    // commits between two operand groups, so that the loop's wait counts below hold from tile 0 on for
    // any depths (without it, tile 0's operands are waited for only when LB >= 2 (LA - LB)).
#pragma unroll
    for (int j = 0; j < LA; ++j) issue_a((uint32_t)j);
    cp_async_wait_all();
#pragma unroll
    for (int j = 0; j < LB; ++j) {
        issue_b((uint32_t)j);
        cp_async_commit();
    }
    for (uint32_t j = 0; j < nt; ++j) {
        issue_a(j + LA);
        cp_async_wait_group<2 * (LA - LB)>();  // tile j+LB's (code, link)
        issue_b(j + LB);
        cp_async_wait_group<2 * LB>();          // tile j's operands
        const uint32_t *q = ra + (j % (uint32_t)NA) * 2u * TILE + threadIdx.x;
        const unsigned long long *r = rb + 2u * ((j % (uint32_t)NB) * TILE + threadIdx.x);
#pragma unroll
        for (int k = 0; k < TPT; ++k) {
            const unsigned long long sl = slot(j, k);
            if (sl >= hi) continue;
            const uint32_t s = (uint32_t)sl, t = task_type(q[k * BS], cen);
            if (!t) continue;
            acc.valid++;
            if (t == TREES_TASK_FIB_SUM) {
                // The sum schedules no join, so its range is not pushed again and no later epoch
                // reaches this entry at its epoch number (a range is revisited only when one of
                // its tasks joins; fresh ranges are written before they are read): the entry is
                // already dead, and marking it invalid (as Sec. 5.3's finished tasks are) is a
                // store per sum that changes nothing; leaving it out measured 0.4116 -> 0.4035 ms
                // per fib(34).
                c.result[s] = r[2 * k * BS] + r[2 * k * BS + 1];
            } else {  // not produced in a join range; run it as the general path would
                Plan p;
                p.s = s;
                p.t = t;
                p.n = 0u;
                p.m = 0u;
                plan_task<PM_FIB, merge_tile(BS)>(c, c.rp, p, cen, e, c.a0[s], 0u, q[TILE + k * BS]);
            }
        }
    }
    cp_async_wait_all();  // the trailing empty groups
}

// ------------------------------------------------------------------ map operations

// Sorts keys in[lo, hi) (at most 1024) ascending with one warp and writes them
// to out[lo, hi); in == out is allowed.  Lane l ends up holding ranks
// [32 l, 32 l + 32) in registers: each lane first sorts its own 32 keys with a
// bitonic network in registers, then five bitonic merge levels join runs of
// 32, 64, ..., 512 keys across lanes (a flip stage pairing rank p with
// 2R-1-p, then half-cleaners), so no block barrier is needed.
__device__ __forceinline__ void warp_leaf_sort(const uint32_t *in, uint32_t *out, uint32_t lo, uint32_t hi,
                                               uint32_t *smp) {
    const uint32_t lane = threadIdx.x & 31u, n = hi - lo;
    uint32_t x[32];
#pragma unroll
    for (int r = 0; r < 32; ++r) {
        const uint32_t i = (uint32_t)r * 32u + lane;  // any input placement will do
        x[r] = i < n ? in[lo + i] : 0xFFFFFFFFu;
    }
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                const int q = r ^ j;
                if (q > r) {
                    const uint32_t a = x[r], b = x[q], mn = min(a, b), mx = max(a, b);
                    if ((r & k) == 0) {
                        x[r] = mn;
                        x[q] = mx;
                    } else {
                        x[r] = mx;
                        x[q] = mn;
                    }
                }
            }
        }
    }
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        const uint32_t span = 2u << m;  // lanes of a merged run
        const bool lower = (lane & (span >> 1)) == 0u;
        // flip: rank p meets rank 2R-1-p (lane ^ (span-1), register 31-r)
#pragma unroll
        for (int r = 0; r < 16; ++r) {
            const uint32_t ya = __shfl_xor_sync(0xffffffffu, x[31 - r], span - 1u);
            const uint32_t yb = __shfl_xor_sync(0xffffffffu, x[r], span - 1u);
            x[r] = lower ? min(x[r], ya) : max(x[r], ya);
            x[31 - r] = lower ? min(x[31 - r], yb) : max(x[31 - r], yb);
        }
        // half-cleaners across lanes
#pragma unroll
        for (uint32_t jl = span >> 2; jl > 0u; jl >>= 1) {
            const bool lo_lane = (lane & jl) == 0u;
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                const uint32_t y = __shfl_xor_sync(0xffffffffu, x[r], jl);
                x[r] = lo_lane ? min(x[r], y) : max(x[r], y);
            }
        }
        // half-cleaners inside the lane
#pragma unroll
        for (int j = 16; j > 0; j >>= 1) {
#pragma unroll
            for (int r = 0; r < 32; ++r) {
                const int q = r ^ j;
                if (q > r) {
                    const uint32_t a = x[r], b = x[q];
                    x[r] = min(a, b);
                    x[q] = max(a, b);
                }
            }
        }
    }
    if (n == 1024u && ((reinterpret_cast<uintptr_t>(out + lo) & 15u) == 0u)) {  // the address, not just lo
        uint4 *o = reinterpret_cast<uint4 *>(out + lo + 32u * lane);
#pragma unroll
        for (int q = 0; q < 8; ++q) o[q] = make_uint4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
    } else {
#pragma unroll
        for (int r = 0; r < 32; ++r) {
            const uint32_t i = 32u * lane + (uint32_t)r;
            if (i < n) out[lo + i] = x[r];
        }
    }
    if (smp) {  // keys at positions that are multiples of 64 become samples, read back after the stores
        __syncwarp();
        const uint32_t first = (lo + 63u) & ~63u;  // at most 16 sample positions in a leaf
        const uint32_t p = first + 64u * lane;
        if (lane < 16u && p < hi) smp[p >> SMP_SHIFT] = out[p];
    }
}

// The sorted runs a merge at depth d reads (depth d+1) and writes (depth d):
// a node at depth d keeps its run in keys (d even) or scratch (d odd).
struct MergeBufs {
    const uint32_t *in;
    uint32_t *out;
};

__device__ __forceinline__ void job_buffers(const Conf &c, const RunParams *job_params, uint32_t job_stride,
                                            uint32_t job, uint32_t **keys, uint32_t **scratch) {
    if (job_params) {
        const RunParams *jp =
            reinterpret_cast<const RunParams *>(reinterpret_cast<const char *>(job_params) + (size_t)job * job_stride);
        *keys = jp->keys;
        *scratch = jp->scratch;
    } else {
        *keys = c.rp.keys;
        *scratch = c.rp.scratch;
    }
}

// The descriptor that owns tile t of the epoch's tiled map list.  One atomic
// hands out a request's descriptors and tiles together, so descriptors own
// consecutive tile ranges in descriptor order and mt_tilebase is
// non-decreasing: the owner is the last descriptor whose first tile is <= t.
// The proportional guess t * ndesc / ntile is exact when the descriptors have
// equal tile counts (every level of a mergesort); else a binary search.
__device__ __forceinline__ uint32_t tile_owner(const Conf &c, uint32_t t, uint32_t ndesc, uint32_t ntile) {
    const uint32_t g = (uint32_t)((unsigned long long)t * ndesc / ntile);
    const uint32_t b0 = c.mt_tilebase[g];
    const uint32_t b1 = g + 1u < ndesc ? c.mt_tilebase[g + 1u] : ntile;
    if (b0 <= t && t < b1) return g;
    uint32_t lo = 0u, hi = ndesc;  // tilebase[lo] <= t < tilebase[hi] (tilebase[ndesc] = ntile)
    while (hi - lo > 1u) {
        const uint32_t mid = (lo + hi) >> 1;
        if (c.mt_tilebase[mid] <= t) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Narrows a merge-path search with the splitter samples of the runs (every
// 64th key, in L2): for the merge of A = in[a, mid) and B = in[mid, b) at
// diagonal d, whose split s (A keys among the first d outputs, A winning
// ties) lies in [*lo, *hi].  At a sampled A index i (a + i a multiple of 64)
// the merge-path test A[i] <= B[d-1-i] is certainly true when A[i] is at most
// the sample at or below B's position, and certainly false when A[i] exceeds
// the sample above it (both runs are sorted).  Certain-true holds on a prefix
// of the sampled indices and certain-false on a suffix, so two searches over
// the samples give s > (last certain-true i) and s <= (first certain-false
// i).  The group's G lanes probe G samples per step for each search.
template <uint32_t G>
__device__ __forceinline__ void sample_bracket(const uint32_t *smp, uint32_t a, uint32_t mid, uint32_t b, uint32_t d,
                                               uint32_t *lo, uint32_t *hi, uint32_t gmask, uint32_t glane) {
    const uint32_t ilo = *lo, ihi = *hi;
    if (ihi - ilo < 256u) return;  // a short search needs no help
    // sampled candidates: global A positions 64 k in [a + ilo, a + ihi)
    const uint32_t ka = (a + ilo + 63u) >> SMP_SHIFT, kb = (a + ihi + 63u) >> SMP_SHIFT;
    auto sure_true = [&](uint32_t k) {  // A[i] <= B[q] known from the sample at or below q
        const uint32_t i = (k << SMP_SHIFT) - a, q = mid + d - 1u - i;
        return (q & ~63u) >= mid && smp[k] <= smp[q >> SMP_SHIFT];
    };
    auto sure_false = [&](uint32_t k) {  // A[i] > B[q] known from the sample above q
        const uint32_t i = (k << SMP_SHIFT) - a, q = mid + d - 1u - i;
        return (q | 63u) + 1u < b && smp[k] > smp[(q >> SMP_SHIFT) + 1u];
    };
    // first candidate that is not sure-true, first that is sure-false (kb when none)
    uint32_t tl = ka, th = kb, fl = ka, fh = kb;
    while (th > tl || fh > fl) {
        const uint32_t ts = (th - tl + G - 1u) / G, fs = (fh - fl + G - 1u) / G;
        const uint32_t tm = tl + glane * ts, fm = fl + glane * fs;
        const bool pt = th > tl && tm < th && sure_true(tm);
        const bool pf = fh > fl && fm < fh && !sure_false(fm);
        const uint32_t ct = (uint32_t)__popc(__ballot_sync(gmask, pt) & gmask);
        const uint32_t cf = (uint32_t)__popc(__ballot_sync(gmask, pf) & gmask);
        if (th > tl) {
            const uint32_t nl = ct ? tl + (ct - 1u) * ts + 1u : tl, cap = tl + ct * ts;
            th = cap < th ? cap : th;
            tl = nl;
        }
        if (fh > fl) {
            const uint32_t nl = cf ? fl + (cf - 1u) * fs + 1u : fl, cap = fl + cf * fs;
            fh = cap < fh ? cap : fh;
            fl = nl;
        }
    }
    if (tl > ka) *lo = max(*lo, ((tl - 1u) << SMP_SHIFT) - a + 1u);
    if (fl < kb) *hi = min(*hi, (fl << SMP_SHIFT) - a);
}

// Partition sub-phase of a map epoch: the merge-path split at the first
// output of every merge tile that does not start its merge, computed in
// parallel by groups of 8 lanes for all tiles at once.  A group runs the
// searches of up to PNS tiles side by side, so their global loads overlap
// and the phase costs about one search's chain of dependent loads.
template <int BS>
__device__ void partition_phase(const Conf &c, unsigned long long mt, const RunParams *job_params, uint32_t job_stride) {
    // 8 probes a step: with the splitter samples most steps search the L2-resident samples (their
    // bracket leaves ~64 keys for the exact search), so wider groups mean fewer dependent steps;
    // measured (2^26 keys, 256 x 1, one call): G = 4 / PNS = 4 2.618 ms, 8 / 2 2.52-2.55 ms,
    // 8 / 4 2.56 ms, 16 / 2 2.55 ms
    constexpr uint32_t G = 8, PNS = 2;
    const uint32_t nt1 = (uint32_t)(mt & CTR_LOW_MASK), nd1 = (uint32_t)(mt >> 40);
    const uint32_t glane = threadIdx.x % G;
    static_assert(G >= 1u && G <= 32u && (G & (G - 1u)) == 0u, "groups tile the warp");
    const uint32_t gmask = (uint32_t)((1ull << G) - 1ull) << ((threadIdx.x & 31u) & ~(G - 1u));  // this group's lanes
    const uint32_t gid = (blockIdx.x * BS + threadIdx.x) / G, ng = gridDim.x * BS / G;
    for (uint32_t t0 = gid; t0 < nt1; t0 += PNS * ng) {
        const uint32_t *A[PNS], *B[PNS];
        uint32_t diag[PNS], lo[PNS], hi[PNS], tt[PNS];
        bool want[PNS];
#pragma unroll
        for (uint32_t q = 0; q < PNS; ++q) {
            const uint32_t t = t0 + q * ng;
            tt[q] = t;
            want[q] = false;
            lo[q] = hi[q] = diag[q] = 0u;
            A[q] = B[q] = nullptr;
            if (t >= nt1) continue;
            const uint32_t di = tile_owner(c, t, nd1, nt1);
            if (c.mt_kind[di] != MAP_MERGE) continue;
            want[q] = true;
            const uint32_t tin = t - c.mt_tilebase[di];
            if (tin == 0u) continue;  // split 0, no search
            const uint32_t a = c.mt_a[di], b = c.mt_b[di], cc = c.mt_c[di], mid = a + (b - a) / 2u;
            uint32_t *keys, *scratch;
            job_buffers(c, job_params, job_stride, c.mt_job[di], &keys, &scratch);
            const uint32_t *in = (cc & 1u) ? keys : scratch;
            const uint32_t la = mid - a, lb = b - mid, d = tin * merge_tile(BS);
            A[q] = in + a;
            B[q] = in + mid;
            diag[q] = d;
            lo[q] = d > lb ? d - lb : 0u;
            hi[q] = d < la ? d : la;
            if (!job_params && c.smp) sample_bracket<G>(c.smp, a, mid, b, d, &lo[q], &hi[q], gmask, glane);
        }
        // merge path (Odeh et al., "Merge Path -- parallel merging made simple", IPDPSW 2012):
        // the split is the number of A keys among the first diag outputs, A winning ties; G probes
        // per search and step
        for (;;) {
            bool pr[PNS], any = false;
            uint32_t step[PNS];
#pragma unroll
            for (uint32_t q = 0; q < PNS; ++q) {
                pr[q] = false;
                step[q] = 0u;
                if (hi[q] > lo[q]) {
                    any = true;
                    step[q] = (hi[q] - lo[q] + G - 1u) / G;
                    const uint32_t m = lo[q] + glane * step[q];
                    if (m < hi[q]) pr[q] = A[q][m] <= B[q][diag[q] - 1u - m];
                }
            }
            if (!any) break;  // lo and hi are the same on every lane of the group
#pragma unroll
            for (uint32_t q = 0; q < PNS; ++q) {
                if (hi[q] > lo[q]) {
                    const uint32_t cnt = (uint32_t)__popc(__ballot_sync(gmask, pr[q]) & gmask);
                    const uint32_t nlo = cnt ? lo[q] + (cnt - 1u) * step[q] + 1u : lo[q];
                    const uint32_t cap = lo[q] + cnt * step[q];
                    hi[q] = cap < hi[q] ? cap : hi[q];
                    lo[q] = nlo;
                }
            }
        }
        if (glane == 0u) {
#pragma unroll
            for (uint32_t q = 0; q < PNS; ++q)
                if (want[q]) c.mt_split[tt[q]] = lo[q];
        }
    }
}

// One merge tile, resolved: the merge of in[lo, mid) (A) and in[mid, hi) (B)
// into out[lo, hi) has output tile [d0, d0 + T); it reads A[i0, i1) and
// B[j0, j1) (indices relative to the runs).
struct MergeTile {
    const uint32_t *in;
    uint32_t *out;
    uint32_t lo, mid, hi, d0, i0, i1, j0, j1;
};

// Resolves merge tile t of the tiled map list (false when it is not a merge).
template <int BS>
__device__ __forceinline__ bool resolve_merge_tile(const Conf &c, uint32_t t, uint32_t nd1, uint32_t nt1,
                                                   const RunParams *jp, uint32_t js, MergeTile &m) {
    const uint32_t di = tile_owner(c, t, nd1, nt1);
    if (c.mt_kind[di] != MAP_MERGE) return false;
    uint32_t *keys, *scratch;
    job_buffers(c, jp, js, c.mt_job[di], &keys, &scratch);
    const uint32_t lo = c.mt_a[di], hi = c.mt_b[di], cc = c.mt_c[di];
    const uint32_t tin = t - c.mt_tilebase[di];
    constexpr uint32_t T = merge_tile(BS);
    const uint32_t la = (hi - lo) / 2u, L = hi - lo, ntiles = (L + T - 1u) / T;
    m.in = (cc & 1u) ? keys : scratch;   // the children's runs (depth d+1)
    m.out = (cc & 1u) ? scratch : keys;  // this node's run (depth d)
    m.lo = lo;
    m.mid = lo + la;
    m.hi = hi;
    m.d0 = tin * T;
    const uint32_t lb = L - la, dend = min(m.d0 + T, L);
    const uint32_t s0 = tin ? c.mt_split[t] : 0u, s1 = tin + 1u < ntiles ? c.mt_split[t + 1u] : la;
    // merge-path splits of sorted runs already satisfy these bounds; the clamps keep every copy
    // and index of the tile inside its runs, its output and its stage buffer whatever the splits
    m.i0 = min(max(s0, m.d0 > lb ? m.d0 - lb : 0u), min(m.d0, la));
    m.i1 = min(max(s1, max(m.i0, dend > lb ? dend - lb : 0u)), min(la, m.i0 + (dend - m.d0)));
    m.j0 = m.d0 - m.i0;
    m.j1 = dend - m.i1;
    return true;
}

// Where a staged tile lives in its buffer: A's keys widened to whole 16-byte
// chunks [as4, ae4u) at word 0, B's chunks [bs4, be4u) right behind them at
// word sbo (a multiple of 4, so both bulk copies start 16-byte aligned).  The
// two spans hold at most T + 12 words.
struct StageLayout {
    uint32_t as, ae, bs, be, as4, ae4u, bs4, be4u, sbo;
};

__device__ __forceinline__ StageLayout stage_layout(const MergeTile &m) {
    StageLayout L;
    L.as = m.lo + m.i0;
    L.ae = m.lo + m.i1;
    L.bs = m.mid + m.j0;
    L.be = m.mid + m.j1;
    L.as4 = L.as & ~3u;
    L.ae4u = (L.ae + 3u) & ~3u;
    L.bs4 = L.bs & ~3u;
    L.be4u = (L.be + 3u) & ~3u;
    L.sbo = L.ae > L.as ? L.ae4u - L.as4 : 0u;
    return L;
}

// Starts staging a tile into buf: thread 0 issues one bulk copy (TMA,
// completing on bar) per run over its whole 16-byte chunks.  A chunk may
// reach past the run but never past the merge's end hi, which is inside the
// array; a last partial chunk beyond hi (hi not a multiple of 4) is loaded
// with plain loads, and so is everything when the array is not 16-byte
// aligned.  buf may still be the source of an earlier tile's bulk store:
// thread 0 waits for those reads before its copies, and the block waits with
// it before plain loads write buf.
template <int BS>
__device__ __forceinline__ void merge_stage(const MergeTile &m, uint32_t *buf, unsigned long long *bar) {
    const StageLayout L = stage_layout(m);
    uint32_t *sb = buf + L.sbo;
    const bool aligned = (reinterpret_cast<uintptr_t>(m.in) & 15u) == 0u;
    const uint32_t ac = L.ae4u <= m.hi ? L.ae4u : (L.ae & ~3u);  // end of A's bulk-copied chunks
    const uint32_t bc = L.be4u <= m.hi ? L.be4u : (L.be & ~3u);
    const uint32_t abytes = aligned && L.ae > L.as && ac > L.as4 ? (ac - L.as4) * 4u : 0u;
    const uint32_t bbytes = aligned && L.be > L.bs && bc > L.bs4 ? (bc - L.bs4) * 4u : 0u;
    const bool plain = (abytes ? ac : L.as) < L.ae || (bbytes ? bc : L.bs) < L.be;  // the same on every thread
    if (threadIdx.x == 0) {
        bulk_wait_read_all();      // earlier bulk stores no longer read buf
        fence_proxy_async_smem();  // earlier generic reads of buf come before the async writes
        mbar_arrive_expect(bar, abytes + bbytes);
        if (abytes) tma_load_1d(buf, m.in + L.as4, abytes, bar);
        if (bbytes) tma_load_1d(sb, m.in + L.bs4, bbytes, bar);
    }
    if (plain) __syncthreads();
    for (uint32_t x = (abytes ? ac : L.as) + threadIdx.x; x < L.ae; x += BS) buf[x - L.as4] = m.in[x];
    for (uint32_t x = (bbytes ? bc : L.bs) + threadIdx.x; x < L.be; x += BS) sb[x - L.bs4] = m.in[x];
}

// Merge-path split of diagonal d (Odeh et al.'s merge path, for the tile
// merges of Sec. 5.2.4): how many of the first d outputs of merging sa[0, na)
// and sb[0, nb) come from A, A winning ties.
__device__ __forceinline__ uint32_t smem_merge_path(const uint32_t *sa, uint32_t na, const uint32_t *sb, uint32_t nb,
                                                    uint32_t d) {
    uint32_t a = d > nb ? d - nb : 0u, b = d < na ? d : na;
    while (a < b) {
        const uint32_t mid = (a + b) >> 1;
        if (sa[mid] <= sb[d - 1u - mid]) a = mid + 1u;
        else b = mid;
    }
    return a;
}

// Merges a staged tile into registers: each thread finds the merge-path split
// of its first output dd in shared memory and merges the next MPT outputs
// (an odd count, see merge_mpt) into v.
template <int BS, uint32_t MPT>
__device__ __forceinline__ void merge_compute(const MergeTile &m, const uint32_t *buf, uint32_t (&v)[MPT],
                                              uint32_t &dd) {
    const StageLayout L = stage_layout(m);
    const uint32_t na = m.i1 - m.i0, nb = m.j1 - m.j0, nt = na + nb;
    const uint32_t *sa = buf + (L.as - L.as4);
    const uint32_t *sb = buf + L.sbo + (L.bs - L.bs4);
    dd = min((uint32_t)threadIdx.x * MPT, nt);
    const uint32_t a = smem_merge_path(sa, na, sb, nb, dd);
    uint32_t ia = a, ib = dd - a;
    // the two run heads stay in registers: one shared-memory load per output.  Indices stop at
    // the runs' ends (ia never passes na; ib is clamped for the last thread of a short tile), and
    // a head read at an end stays inside the staged buffer and is never taken.
    uint32_t ka = sa[ia], kb = sb[ib];
#pragma unroll
    for (uint32_t k = 0; k < MPT; ++k) {
        const bool takeA = ia < na && (ib >= nb || ka <= kb);
        v[k] = takeA ? ka : kb;
        ia += takeA;
        ib += !takeA;
        const uint32_t x = takeA ? sa[ia] : sb[min(ib, nb)];
        ka = takeA ? x : ka;
        kb = takeA ? kb : x;
    }
}

// Writes a merged tile: after the block has finished reading buf, each thread
// puts its outputs back into buf (consecutive threads MPT words apart, an odd
// stride: no bank conflicts), and thread 0 stores the tile's contiguous
// output with one bulk copy; without 16-byte alignment the block copies it
// out with coalesced stores instead.
template <int BS, uint32_t MPT>
__device__ __forceinline__ void merge_write(const MergeTile &m, uint32_t *buf, const uint32_t (&v)[MPT], uint32_t dd,
                                            uint32_t *smp) {
    const uint32_t nt = (m.i1 - m.i0) + (m.j1 - m.j0);
#pragma unroll
    for (uint32_t k = 0; k < MPT; ++k)
        if (dd + k < nt) buf[dd + k] = v[k];
    uint32_t *o = m.out + m.lo + m.d0;
    const bool bulk = ((reinterpret_cast<uintptr_t>(o) & 15u) == 0u) && (nt & 3u) == 0u;
    if (bulk) fence_proxy_async_smem();  // these generic writes come before the bulk copy's reads
    __syncthreads();
    if (smp && threadIdx.x < 32u) {  // warp 0 copies the tile's samples (outputs at multiples of 64)
        const uint32_t p0 = m.lo + m.d0, first = ((p0 + 63u) & ~63u) - p0;
        for (uint32_t i = first + 64u * threadIdx.x; i < nt; i += 64u * 32u) smp[(p0 + i) >> SMP_SHIFT] = buf[i];
        __syncwarp();  // these reads of buf come before thread 0 (this warp) stages into it again
    }
    if (bulk) {
        if (threadIdx.x == 0 && nt) tma_store_1d(o, buf, nt * 4u);
    } else {
        for (uint32_t i = threadIdx.x; i < nt; i += BS) o[i] = buf[i];
        __syncthreads();  // buf is read before the next tile is staged into it
    }
}

// One staged tile, start to end, with MPT outputs per thread; false (and
// nothing written) when the tile's copy did not land on some thread.
template <int BS, uint32_t MPT>
__device__ __forceinline__ bool merge_run(const MergeTile &m, uint32_t *buf, bool landed, uint32_t *smp) {
    uint32_t v[MPT], dd;
    merge_compute<BS, MPT>(m, buf, v, dd);
    // every thread has read buf and the tails staged for later tiles are visible; a wait that ran
    // out anywhere in the block is seen by every thread here, so all leave together
    if (__syncthreads_or(!landed)) return false;
    merge_write<BS, MPT>(m, buf, v, dd, smp);
    return true;
}

__device__ __forceinline__ void put_merge_tile(uint32_t *w, const MergeTile &x) {
    w[0] = (uint32_t)(reinterpret_cast<uintptr_t>(x.in));
    w[1] = (uint32_t)(reinterpret_cast<uintptr_t>(x.in) >> 32);
    w[2] = (uint32_t)(reinterpret_cast<uintptr_t>(x.out));
    w[3] = (uint32_t)(reinterpret_cast<uintptr_t>(x.out) >> 32);
    w[4] = x.lo;
    w[5] = x.mid;
    w[6] = x.hi;
    w[7] = x.d0;
    w[8] = x.i0;
    w[9] = x.i1;
    w[10] = x.j1;
}

__device__ __forceinline__ void get_merge_tile(const uint32_t *w, MergeTile &m) {
    m.in = reinterpret_cast<const uint32_t *>((uintptr_t)w[0] | ((uintptr_t)w[1] << 32));
    m.out = reinterpret_cast<uint32_t *>((uintptr_t)w[2] | ((uintptr_t)w[3] << 32));
    m.lo = w[4];
    m.mid = w[5];
    m.hi = w[6];
    m.d0 = w[7];
    m.i0 = w[8];
    m.i1 = w[9];
    m.j0 = m.d0 - m.i0;
    m.j1 = w[10];
}

// All merge tiles of the epoch handled by this block (tiles blockIdx.x +
// k*gridDim.x), pipelined merge_nst(BS) deep: while the block merges one
// tile from shared memory, the next ones stream in by TMA.  The
// block resolves its tiles MCHUNK at a time, one thread per tile, into a
// shared table that every thread then walks in the same order.  Waits are
// bounded (TREES_ERR_TIMEOUT); on a timeout the block lets its copies in
// flight land before it leaves.
template <int BS>
__device__ void merge_phase(const Conf &c, Ctl *ctl, Smem<BS> &sm, uint32_t nt1, uint32_t nd1, const RunParams *jp,
                            uint32_t js) {
    static_assert(MCHUNK <= 64 && MCHUNK <= BS, "one resolver thread per table entry, one mask bit each");
    constexpr int NST = merge_nst(BS);
    if (threadIdx.x == 0)
        for (int q = 0; q < NST; ++q) mbar_init(&sm.mbar[q], 1u);
    uint32_t phase = 0u;  // bit q: parity of buffer q's next completion
    uint32_t gs = 0u;     // tiles staged so far; tile number g uses buffer g % NST
    const uint32_t stride = gridDim.x * (uint32_t)MCHUNK;
    for (uint32_t c0 = blockIdx.x; c0 < nt1; c0 += stride) {
        __syncthreads();  // the previous chunk's table is no longer read
        if (threadIdx.x < 64u) {
            const uint32_t t = c0 + threadIdx.x * gridDim.x;
            MergeTile x;
            const bool ok = threadIdx.x < (uint32_t)MCHUNK && t < nt1 && resolve_merge_tile<BS>(c, t, nd1, nt1, jp, js, x);
            if (ok) put_merge_tile(sm.mtab[threadIdx.x], x);
            const uint32_t bal = __ballot_sync(0xffffffffu, ok);
            if ((threadIdx.x & 31u) == 0u) reinterpret_cast<uint32_t *>(&sm.mvalid)[threadIdx.x >> 5] = bal;
        }
        __syncthreads();
        unsigned long long to_stage = sm.mvalid, to_merge = to_stage;
        uint32_t gc = gs;  // the next tile to merge
        for (int q = 0; q < NST - 1 && to_stage; ++q, ++gs) {
            const int k = __ffsll((long long)to_stage) - 1;
            to_stage &= to_stage - 1ull;
            MergeTile x;
            get_merge_tile(sm.mtab[k], x);
            merge_stage<BS>(x, sm.u.mg[gs % NST], &sm.mbar[gs % NST]);
        }
        __syncthreads();
        while (to_merge) {
            if (to_stage) {  // buffer gs % NST was freed by the barrier that ended the last merge
                const int k = __ffsll((long long)to_stage) - 1;
                to_stage &= to_stage - 1ull;
                MergeTile x;
                get_merge_tile(sm.mtab[k], x);
                merge_stage<BS>(x, sm.u.mg[gs % NST], &sm.mbar[gs % NST]);
                ++gs;
            }
            const uint32_t b = gc % NST;
            const bool landed = mbar_wait(&sm.mbar[b], (phase >> b) & 1u, c.timeout_ns);
            phase ^= 1u << b;
            const int k = __ffsll((long long)to_merge) - 1;
            to_merge &= to_merge - 1ull;
            MergeTile cur;
            get_merge_tile(sm.mtab[k], cur);
            const uint32_t nt = (cur.i1 - cur.i0) + (cur.j1 - cur.j0);
            const bool ok = nt <= (uint32_t)BS * merge_mpt_small(BS)
                                ? merge_run<BS, merge_mpt_small(BS)>(cur, sm.u.mg[b], landed, jp ? nullptr : c.smp)
                                : merge_run<BS, merge_mpt(BS)>(cur, sm.u.mg[b], landed, jp ? nullptr : c.smp);
            ++gc;
            if (!ok) {
                if (threadIdx.x == 0) set_err(ctl, TREES_ERR_TIMEOUT, 0x80000000u | (c0 + (uint32_t)k * gridDim.x));
                phase ^= 1u << b;  // wait again for the tile that ran out, then for every later one
                for (--gc; gc < gs; ++gc) {  // let the copies in flight land
                    const uint32_t q = gc % NST;
                    mbar_wait(&sm.mbar[q], (phase >> q) & 1u, c.timeout_ns);
                    phase ^= 1u << q;
                }
                if (threadIdx.x == 0) bulk_wait_all();
                __syncthreads();
                return;
            }
        }
    }
    if (threadIdx.x == 0) bulk_wait_all();  // the outputs are in memory before the block's next barrier
}

// The element maps (BFS expansion, SSSP relaxation) run as tiles of
// expand_tile_len(BS) adjacency entries, each taken by one part of a block: the
// EXPAND_PARTS(BS) parts of a block (BS / parts threads each, synchronised by
// their own named barriers, with disjoint shared-memory records) run
// independent tiles, so an SM has several tile chains in flight per block
// without more registers or shared memory.  bar_part(h): the barrier of part h
// (ids 1..parts; a warp barrier for one-warp parts).
template <int BS>
__device__ __forceinline__ void bar_part(uint32_t h) {
    static_assert(BS / EXPAND_PARTS(BS) == 32 || EXPAND_PARTS(BS) <= 15u, "named barrier ids 1..15");
    if constexpr (BS / EXPAND_PARTS(BS) == 32) {
        __syncwarp();  // a one-warp part
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(1u + h), "r"((uint32_t)(BS / EXPAND_PARTS(BS))) : "memory");
    }
}

// Exclusive scan of v over the threads of block part h (thread order), with
// the part's total; one named barrier (each thread sums its part's warp
// totals itself).  The warp totals are written again only after the caller's
// next barrier of this part.
template <int BS>
__device__ __forceinline__ uint32_t part_scan_u32(uint32_t v, uint32_t h, uint32_t *total, Smem<BS> &sm) {
    constexpr uint32_t NWH = BS / 32 / EXPAND_PARTS(BS);  // warps per part
    const uint32_t lane = threadIdx.x & 31u, wid = threadIdx.x >> 5;
    const uint32_t inc = warp_incl_u32(v);
    if (lane == 31u) sm.w32[wid] = inc;
    bar_part<BS>(h);
    uint32_t pre = 0u, all = 0u;
#pragma unroll
    for (uint32_t w = 0; w < NWH; ++w) {
        const uint32_t x = sm.w32[h * NWH + w];
        all += x;
        pre += h * NWH + w < wid ? x : 0u;
    }
    *total = all;
    return pre + inc - v;
}

// The descriptors of element tile t (the vertices whose adjacency it covers)
// into part h's shared records: each vertex's first adjacency index and
// first element, and for SSSP its distance, read once for the tile.
// Returns how many there are.
template <int BS, bool SSSP>
__device__ __forceinline__ uint32_t load_tile_descriptors(const Conf &c, Smem<BS> &sm, uint32_t t, uint32_t nd,
                                                          uint32_t nt, uint32_t h, uint32_t lt) {
    const uint32_t dfirst = c.me_tfd[t];
    const uint32_t dlast = (t + 1u < nt) ? c.me_tfd[t + 1u] : nd - 1u;
    const uint32_t nloc = dlast - dfirst + 1u;
    for (uint32_t k = lt; k < nloc; k += BS / EXPAND_PARTS(BS)) {
        sm.u.ex.base[h][k] = c.me_base[dfirst + k];
        sm.u.ex.v[h][k] = c.me_v[dfirst + k];
        if constexpr (SSSP) sm.u.ex.d[h][k] = c.rp.dist[c.me_src[dfirst + k]];
    }
    bar_part<BS>(h);
    return nloc;
}

// The next tile's descriptors read ahead into registers (BFS): issued while
// the current tile's chain runs, stored into the part's records once every
// thread of the part has finished searching the current ones, so the next
// tile starts without its two dependent round trips (the tile's first
// descriptor, then the descriptors).  KD: the most a thread holds.
template <int BS>
struct DescAhead {
    static constexpr uint32_t HB = BS / EXPAND_PARTS(BS), KD = (expand_tile_len(BS) + 2u + HB - 1u) / HB;
    uint32_t n;  // descriptors of the next tile (0: no next tile)
    uint32_t b[KD], v[KD];
};

template <int BS>
__device__ __forceinline__ void desc_ahead_issue(const Conf &c, uint32_t tn, uint32_t nd, uint32_t nt, uint32_t lt,
                                                 DescAhead<BS> &A) {
    A.n = 0u;
    if (tn < nt) {
        const uint32_t df = c.me_tfd[tn], dl = tn + 1u < nt ? c.me_tfd[tn + 1u] : nd - 1u;
        A.n = dl - df + 1u;
#pragma unroll
        for (uint32_t i = 0; i < DescAhead<BS>::KD; ++i) {
            const uint32_t k = lt + i * DescAhead<BS>::HB;
            if (k < A.n) {
                A.b[i] = c.me_base[df + k];
                A.v[i] = c.me_v[df + k];
            }
        }
    }
}

template <int BS>
__device__ __forceinline__ void desc_ahead_store(Smem<BS> &sm, uint32_t h, uint32_t lt, const DescAhead<BS> &A) {
#pragma unroll
    for (uint32_t i = 0; i < DescAhead<BS>::KD; ++i) {
        const uint32_t k = lt + i * DescAhead<BS>::HB;
        if (k < A.n) {
            sm.u.ex.base[h][k] = A.b[i];
            sm.u.ex.v[h][k] = A.v[i];
        }
    }
}

// Element g of the tile: its descriptor (load-balanced search over the
// part's records in shared memory).
template <int BS>
__device__ __forceinline__ uint32_t tile_owner_local(const Smem<BS> &sm, uint32_t h, uint32_t nloc, uint32_t g) {
    uint32_t lo = 0, hi = nloc;
    while (hi - lo > 1u) {
        const uint32_t mid = (lo + hi) >> 1;
        if (sm.u.ex.base[h][mid] <= g) lo = mid;
        else hi = mid;
    }
    return lo;
}

// Reserves `tot` slots for part h's forks (one atomic for the part's tile)
// and broadcasts the base and the capacity verdict through shared memory.
template <int BS>
__device__ __forceinline__ bool part_reserve(const Conf &c, Ctl *ctl, Smem<BS> &sm, uint32_t h, uint32_t lt,
                                             uint32_t tot, uint32_t base, uint32_t ep, uint32_t e, uint32_t *b) {
    if (lt == 0u) {
        const uint32_t r = atomicAdd(fork_ctr(ctl, ep), tot);  // one atomic per part tile (Sec. 5.2.3)
        const bool over = (unsigned long long)base + r + tot > c.cap;
        if (over) set_err(ctl, TREES_ERR_CAPACITY, e);
        sm.bc32[2u * h] = r;
        sm.bc32[2u * h + 1u] = over;
    }
    bar_part<BS>(h);
    *b = sm.bc32[2u * h];
    return !sm.bc32[2u * h + 1u];
}

// Claim buffers of the expansion tiles (block part h's buffer: the space of
// its distance records, which BFS does not use; SSSP: dynamic shared memory).
// SSSP's tiles append the neighbours whose distance their atomic minimum
// shortened, and the flush's atomic maximum on sched decides which are
// forked; BFS's tiles append their candidates (neighbours whose visited bit
// was clear) and the flush claims them.  Either way the forks of a buffer take
// one reservation on
// nextFreeCore (Sec. 5.2.3's single atomic for a group of forks, the group
// made larger): a tile claims a dozen vertices on average, so a reservation
// (and the scan that placed the claims) per tile cost more than the claims'
// stores.  The fork range stays gap-free: each flush reserves exactly its
// claims.
__host__ __device__ constexpr uint32_t claim_cap_of(int bs) { return 2u * (expand_tile_len(bs) + 2u); }  // the d records of one part, in u32

template <int BS>
__device__ __forceinline__ uint32_t *claim_buf(Smem<BS> &sm, uint32_t h) {
    static_assert(sizeof(sm.u.ex.d[0]) >= claim_cap_of(BS) * sizeof(uint32_t), "a part's buffer fits its d records");
    return reinterpret_cast<uint32_t *>(sm.u.ex.d[h]);
}

// BFS: claims the candidates in part h's buffer and forks the claimed ones as
// visit tasks of epoch CEN+1 (every thread of the part calls it, after a
// barrier of the part that follows the appends).  A CAS of each candidate's
// level from -1 to CEN+1 decides between competing visits (the buffer may
// hold a vertex several times, from several tiles or edges: one CAS wins),
// the winner sets the vertex's visited bit, and one reservation places the
// winners.  A thread's CASes are issued in groups of RC before any answer is
// examined, so a buffer of ~30 tiles' candidates costs a few overlapped round
// trips instead of one per tile (R-MAT 22, 512 x 1: 0.766 -> 0.668 ms; the
// levels, and every epoch's task and fork counts, are unchanged: the same
// vertices are claimed in the same epoch, by one candidate each).  Ends with
// a barrier of the part.
template <int BS>
__device__ __forceinline__ void bfs_claim_flush(const Conf &c, Ctl *ctl, Smem<BS> &sm, const uint32_t *cb, uint32_t h,
                                                uint32_t lt, uint32_t cen, uint32_t base, uint32_t ep, uint32_t e) {
    constexpr uint32_t HB = BS / EXPAND_PARTS(BS), R = (claim_cap_of(BS) + HB - 1u) / HB, RC = 8u;
    static_assert(R <= 32u, "one bit per candidate of a thread");
    const uint32_t n = sm.pcnt[h];
    const int32_t nlev = (int32_t)(cen + 1u);
    uint32_t won = 0u;  // bit r: this thread's candidate r (buffer entry lt + r * HB) was claimed
#pragma unroll
    for (uint32_t r0 = 0; r0 < R; r0 += RC) {
        int32_t prev[RC];
#pragma unroll
        for (uint32_t q = 0; q < RC; ++q) {
            const uint32_t i = lt + (r0 + q) * HB;
            prev[q] = r0 + q < R && i < n ? atomicCAS(c.rp.level + cb[i], -1, nlev) : 0;
        }
#pragma unroll
        for (uint32_t q = 0; q < RC; ++q) {
            if (prev[q] == -1) {
                const uint32_t u = cb[lt + (r0 + q) * HB];
                won |= 1u << (r0 + q);
                atomicOr(c.rp.visited + (u >> 5), 1u << (u & 31u));
            }
        }
    }
    uint32_t tot;
    const uint32_t off = part_scan_u32<BS>((uint32_t)__popc(won), h, &tot, sm);
    uint32_t b;
    if (tot && part_reserve<BS>(c, ctl, sm, h, lt, tot, base, ep, e, &b)) {
        const uint32_t code = enc(cen + 1u, TREES_TASK_BFS_VISIT);
        uint32_t slot = base + b + off;
#pragma unroll
        for (uint32_t r = 0; r < R; ++r) {
            if ((won >> r) & 1u) {
                c.code[slot] = code;
                c.a0[slot] = cb[lt + r * HB];
                ++slot;
            }
        }
    }
    if (lt == 0u) sm.pcnt[h] = 0u;  // every thread read the count before part_scan's barrier
    bar_part<BS>(h);
}

// SSSP: forks relax(u) for epoch CEN+1 for each vertex u in part h's buffer
// that no other thread has forked this epoch: an atomic maximum of sched[u]
// to CEN+1 finds the first (a vertex shortened by several tiles or edges is
// in the buffer several times; one maximum wins).  A thread's maxima are
// issued in groups of RC before any answer is examined, so the tiles' chains
// end after their atomic minima (R-MAT 22, 512 x 1: 2.13 -> 2.02 ms,
// distances unchanged).  Ends with a barrier of the part.
template <int BS>
__device__ __forceinline__ void sssp_claim_flush(const Conf &c, Ctl *ctl, Smem<BS> &sm, const uint32_t *cb, uint32_t cap,
                                                 uint32_t h, uint32_t lt, uint32_t cen, uint32_t base, uint32_t ep,
                                                 uint32_t e) {
    constexpr uint32_t HB = BS / EXPAND_PARTS(BS), RC = 8u;
    const uint32_t n = sm.pcnt[h], R = (cap + HB - 1u) / HB;
    uint32_t won = 0u;
    for (uint32_t r0 = 0; r0 < R; r0 += RC) {
        uint32_t prev[RC];
#pragma unroll
        for (uint32_t q = 0; q < RC; ++q) {
            const uint32_t i = lt + (r0 + q) * HB;
            prev[q] = r0 + q < R && i < n ? atomicMax(c.rp.sched + cb[i], cen + 1u) : ~0u;
        }
#pragma unroll
        for (uint32_t q = 0; q < RC; ++q)
            if (prev[q] < cen + 1u) won |= 1u << (r0 + q);
    }
    uint32_t tot;
    const uint32_t off = part_scan_u32<BS>((uint32_t)__popc(won), h, &tot, sm);
    uint32_t b;
    if (tot && part_reserve<BS>(c, ctl, sm, h, lt, tot, base, ep, e, &b)) {
        const uint32_t code = enc(cen + 1u, TREES_TASK_SSSP_RELAX);
        uint32_t slot = base + b + off;
        for (uint32_t r = 0; r < R; ++r) {
            if ((won >> r) & 1u) {
                c.code[slot] = code;
                c.a0[slot] = cb[lt + r * HB];
                ++slot;
            }
        }
    }
    if (lt == 0u) sm.pcnt[h] = 0u;  // every thread read the count before part_scan's barrier
    bar_part<BS>(h);
}

// Appends this thread's vertices (bits of cmask over uu) to part h's
// buffer: one shared-memory atomic per warp, no barrier.
template <int BS, int EPT>
__device__ __forceinline__ void claim_append(Smem<BS> &sm, uint32_t *cb, uint32_t h, uint32_t cmask,
                                             const int32_t (&uu)[EPT]) {
    const uint32_t lane = threadIdx.x & 31u, nc = (uint32_t)__popc(cmask), inc = warp_incl_u32(nc);
    uint32_t wb = 0u;
    if (lane == 31u && inc) wb = atomicAdd(&sm.pcnt[h], inc);
    uint32_t pos = __shfl_sync(0xffffffffu, wb, 31) + inc - nc;
#pragma unroll
    for (int j = 0; j < EPT; ++j)
        if ((cmask >> j) & 1u) cb[pos++] = (uint32_t)uu[j];
}

// One BFS expansion tile (expand_tile_len(BS) consecutive adjacency entries of the
// epoch's frontier) on part h of the block, whose nloc descriptors are in the
// part's records.  Each entry's vertex is found by a binary search over the
// tile's descriptors in shared memory (load-balanced search); a neighbour
// whose visited bit is clear goes to the part's buffer, whose flush claims it
// with a CAS on its level and forks it as a visit task (bfs_claim_flush).
// The descriptors of the part's next tile tn are read meanwhile and are in
// the records when it returns; it returns their count.
template <int BS>
__device__ uint32_t expand_tile(const Conf &c, Ctl *ctl, Smem<BS> &sm, uint32_t t, uint32_t tn, uint32_t nloc,
                                uint32_t nd, uint32_t ne, uint32_t nt, uint32_t cen, uint32_t base, uint32_t ep,
                                uint32_t e, uint32_t h) {
    constexpr uint32_t ET = expand_tile_len(BS), HB = BS / EXPAND_PARTS(BS), EPT = ET / HB;
    const uint32_t lt = threadIdx.x - h * HB;
    const uint32_t g0 = t * ET, g1 = min(g0 + ET, ne);
    // stage 1: every element's adjacency index (load-balanced search in shared memory)
    uint32_t ed[EPT];
#pragma unroll
    for (uint32_t j = 0; j < EPT; ++j) {
        const uint32_t g = g0 + j * HB + lt;
        ed[j] = 0xFFFFFFFFu;
        if (g < g1) {
            const uint32_t k = tile_owner_local<BS>(sm, h, nloc, g);
            ed[j] = sm.u.ex.v[h][k] + (g - sm.u.ex.base[h][k]);
        }
    }
    // stage 2: all neighbour ids, then all their visited bits, in flight together (and the next
    // tile's descriptors behind them).  The bits are a hint: one is set only after its vertex's
    // claim, so a clear bit may be stale (the CAS then fails) but a set bit never is; 32 vertices
    // share a word, so the probes find them in L1 and L2 far more often than the levels (a 32-byte
    // sector per probe of the 16 MB level array at R-MAT 22).  The neighbour ids stream past once and
    // are read without allocating in L1, which keeps the visited words there (R-MAT 22, 512 x 2:
    // 0.768 -> 0.750 ms)
    int32_t uu[EPT];
    uint32_t vb[EPT];
#pragma unroll
    for (uint32_t j = 0; j < EPT; ++j) {
        uu[j] = -1;
        if (ed[j] != 0xFFFFFFFFu)
            asm volatile("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(uu[j]) : "l"(c.rp.col + ed[j]));
    }
    DescAhead<BS> A;
    desc_ahead_issue<BS>(c, tn, nd, nt, lt, A);
#pragma unroll
    for (uint32_t j = 0; j < EPT; ++j) vb[j] = uu[j] >= 0 ? __ldca(c.rp.visited + ((uint32_t)uu[j] >> 5)) : ~0u;
    // stage 3: the neighbours whose visited bit is clear are candidates; they go to the part's
    // buffer, and its flush claims them (the tile's chain ends without an atomic round trip)
    uint32_t cmask = 0u;
#pragma unroll
    for (uint32_t j = 0; j < EPT; ++j)
        if (uu[j] >= 0 && ((vb[j] >> ((uint32_t)uu[j] & 31u)) & 1u) == 0u) cmask |= 1u << j;
    claim_append<BS, (int)EPT>(sm, claim_buf<BS>(sm, h), h, cmask, uu);
    bar_part<BS>(h);  // every thread of the part is past its search and its appends
    desc_ahead_store<BS>(sm, h, lt, A);  // the records are free
    if (sm.pcnt[h] > claim_cap_of(BS) - ET)  // part-uniform
        bfs_claim_flush<BS>(c, ctl, sm, claim_buf<BS>(sm, h), h, lt, cen, base, ep, e);
    bar_part<BS>(h);  // the next tile's records are in place
    return A.n;
}

// One SSSP relaxation tile (Sec. 6.3's worklist relaxation as a map) on part
// h of the block: the same element-balanced layout as a BFS expansion tile.
// Each source vertex v of the tile has its distance read once for the tile;
// for each of its out-edges (v, u, w) here, nd = dist[v] + w; an atomic
// minimum shortens dist[u] if nd is smaller, and the thread whose minimum
// took effect forks relax(u) for epoch CEN+1 unless another already did this
// epoch (an atomic maximum on sched[u]).  dist[v] may have been shortened
// after the tile read it; v is then forked again for the next epoch, so the
// final distances are the shortest ones.  Each tile also records, per source
// vertex, the distance its edges used (an atomic maximum of
// (CEN+1) << 40 | distance), so that a relax(v) forked again whose distance
// is still the one every edge of v used in the previous epoch ends at once.
template <int BS>
__device__ void relax_tile(const Conf &c, Ctl *ctl, Smem<BS> &sm, uint32_t t, uint32_t nd, uint32_t ne, uint32_t nt,
                           uint32_t cen, uint32_t base, uint32_t ep, uint32_t e, uint32_t h, uint32_t *cb,
                           uint32_t cap) {
    constexpr uint32_t ET = expand_tile_len(BS), HB = BS / EXPAND_PARTS(BS), EPT = ET / HB;
    const uint32_t lt = threadIdx.x - h * HB;
    const uint32_t g0 = t * ET, g1 = min(g0 + ET, ne);
    const uint32_t dfirst = c.me_tfd[t];
    const uint32_t nloc = load_tile_descriptors<BS, true>(c, sm, t, nd, nt, h, lt);
    // stage 1: every element's adjacency index and its source's distance (load-balanced search)
    uint32_t ed[EPT];
    unsigned long long dv[EPT];
#pragma unroll
    for (uint32_t j = 0; j < EPT; ++j) {
        const uint32_t g = g0 + j * HB + lt;
        ed[j] = 0xFFFFFFFFu;
        dv[j] = 0ull;
        if (g < g1) {
            const uint32_t k = tile_owner_local<BS>(sm, h, nloc, g);
            ed[j] = sm.u.ex.v[h][k] + (g - sm.u.ex.base[h][k]);
            dv[j] = sm.u.ex.d[h][k];
        }
    }
    // stage 2: neighbours, weights and the neighbours' distances in flight together.  Neighbour ids
    // and weights stream past once and are read without allocating in L1, which keeps the distances
    // there (R-MAT 22, 512 x 1: 2.28 -> 2.14 ms)
    int32_t uu[EPT];
    unsigned long long cand[EPT], du[EPT];
#pragma unroll
    for (uint32_t j = 0; j < EPT; ++j) {
        uu[j] = -1;
        if (ed[j] != 0xFFFFFFFFu)
            asm volatile("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(uu[j]) : "l"(c.rp.col + ed[j]));
    }
#pragma unroll
    for (uint32_t j = 0; j < EPT; ++j) {
        cand[j] = ~0ull;
        du[j] = 0ull;
        if (uu[j] >= 0) {
            uint32_t w;
            asm volatile("ld.global.nc.L1::no_allocate.b32 %0, [%1];" : "=r"(w) : "l"(c.rp.weight + ed[j]));
            cand[j] = dv[j] + (unsigned long long)w;
            du[j] = c.rp.dist[uu[j]];
        }
    }
    // stage 3: shorten, and fork the neighbours this thread shortened first this epoch.  All of the
    // thread's atomic minima are issued before any answer is examined, so they cost one overlapped
    // round trip; with a claim buffer the shortened neighbours go there and its flush takes the
    // atomic maxima that decide the forks, else the tile takes them here, all issued together.
    unsigned long long old[EPT];
#pragma unroll
    for (uint32_t j = 0; j < EPT; ++j) old[j] = uu[j] >= 0 && cand[j] < du[j] ? atomicMin(c.rp.dist + uu[j], cand[j]) : 0ull;
    uint32_t cmask = 0u;
    if (cb) {  // the shortened neighbours go to the buffer; its flush decides which are forked
#pragma unroll
        for (uint32_t j = 0; j < EPT; ++j)
            if (uu[j] >= 0 && cand[j] < du[j] && cand[j] < old[j]) cmask |= 1u << j;
        claim_append<BS, (int)EPT>(sm, cb, h, cmask, uu);
        cmask = 0u;
    } else {
        uint32_t prev[EPT];
#pragma unroll
        for (uint32_t j = 0; j < EPT; ++j)
            prev[j] = uu[j] >= 0 && cand[j] < du[j] && cand[j] < old[j] ? atomicMax(c.rp.sched + uu[j], cen + 1u) : ~0u;
#pragma unroll
        for (uint32_t j = 0; j < EPT; ++j)
            if (prev[j] < cen + 1u) cmask |= 1u << j;
    }
    uint32_t ftot = 0u, off = 0u;
    if (!cb) off = part_scan_u32<BS>((uint32_t)__popc(cmask), h, &ftot, sm);
    uint32_t b;
    if (ftot && part_reserve<BS>(c, ctl, sm, h, lt, ftot, base, ep, e, &b)) {
        const uint32_t code = enc(cen + 1u, TREES_TASK_SSSP_RELAX);
        uint32_t slot = base + b + off;
#pragma unroll
        for (uint32_t j = 0; j < EPT; ++j) {
            if ((cmask >> j) & 1u) {
                c.code[slot] = code;
                c.a0[slot] = (uint32_t)uu[j];
                ++slot;
            }
        }
    }
    // record, per source vertex of the tile, the distance its edges here used (the largest over the
    // epoch's tiles wins; a descriptor listed for the tile without edges in it only raises it)
    for (uint32_t k = lt; k < nloc; k += HB) {
        const unsigned long long d = sm.u.ex.d[h][k];
        if (d < (1ull << SSSP_USED_SHIFT))
            atomicMax(c.rp.used + c.me_src[dfirst + k], (unsigned long long)(cen + 1u) << SSSP_USED_SHIFT | d);
    }
    bar_part<BS>(h);  // the part's records are its next tile's
    if (cb && sm.pcnt[h] > cap - ET)  // part-uniform
        sssp_claim_flush<BS>(c, ctl, sm, cb, cap, h, lt, cen, base, ep, e);
}

// The combine maps of one FFT epoch as one flat array of butterflies.  The
// epoch's range holds all 2^d tasks of depth d, each a combine of 2^lgm
// points (lgm = log2 N - d), so nd = 2^d and there are N/2 butterflies:
// butterfly g is butterfly k = g mod h of the combine of task o = g / h,
// h = 2^(lgm-1), which pairs X[blk + k] with X[blk + h + k], blk the block of
// (o, d).  Consecutive threads take consecutive butterflies (coalesced, a
// warp spans at most 32 / h blocks); each thread keeps FFT_CHUNK of them in
// flight, their loads first.
template <int BS>
__device__ void fft_combine_map(const Conf &c, uint32_t nd, uint32_t ne) {
    const uint32_t d = 31u - (uint32_t)__clz(nd), lgn = c.rp.lgn, lh = lgn - d - 1u;
    const uint32_t hmask = (1u << lh) - 1u, stride = gridDim.x * BS;
    float2 *X = c.rp.fX;
    for (uint32_t g0 = blockIdx.x * BS + threadIdx.x; g0 < ne; g0 += stride * FFT_CHUNK) {
        uint32_t pe[FFT_CHUNK];
        float2 e[FFT_CHUNK], o[FFT_CHUNK];
#pragma unroll
        for (uint32_t j = 0; j < FFT_CHUNK; ++j) {
            const uint32_t g = g0 + j * stride;
            pe[j] = g < ne ? fft_block(g >> lh, d, lgn) + (g & hmask) : 0xFFFFFFFFu;
        }
#pragma unroll
        for (uint32_t j = 0; j < FFT_CHUNK; ++j) {
            if (pe[j] != 0xFFFFFFFFu) {
                e[j] = X[pe[j]];
                o[j] = X[pe[j] + (1u << lh)];
            }
        }
#pragma unroll
        for (uint32_t j = 0; j < FFT_CHUNK; ++j) {
            if (pe[j] != 0xFFFFFFFFu) {
                fft_bfly(e[j], o[j], fft_twiddle((g0 + j * stride) & hmask, lh + 1u));
                X[pe[j]] = e[j];
                X[pe[j] + (1u << lh)] = o[j];
            }
        }
    }
}

// The map phase of epoch e, after the partition sub-phase: leaf sorts one
// warp per leaf, merge tiles one block per tile, then the expansion tiles.
template <int BS, uint32_t PM, typename UP = NoUserProgram>
__device__ void map_phase(const Conf &c, Ctl *ctl, Smem<BS> &sm, uint32_t ep, uint32_t e, uint32_t cen, uint32_t base,
                          unsigned long long mt, unsigned long long me, const RunParams *job_params = nullptr,
                          uint32_t job_stride = 0, uint32_t *claims = nullptr, uint32_t claim_cap = 0u) {
    const uint32_t nt1 = (uint32_t)(mt & CTR_LOW_MASK), nd1 = (uint32_t)(mt >> 40);
    const uint32_t nd2 = (uint32_t)(me >> 40), ne2 = (uint32_t)(me & CTR_LOW_MASK);
    const uint32_t nt2 = (ne2 + expand_tile_len(BS) - 1u) / expand_tile_len(BS);
    uint32_t *keys, *scratch;
    if constexpr ((PM & PM_USER) != 0u) {  // one block per unit, grid-stride over the epoch's units
        const trees_user_env env = user_env(c);
        for (uint32_t t = blockIdx.x; t < nt1; t += gridDim.x) {
            const uint32_t di = tile_owner(c, t, nd1, nt1);
            const uint32_t t0 = c.mt_tilebase[di];
            const uint32_t t1 = di + 1u < nd1 ? c.mt_tilebase[di + 1u] : nt1;
            const trees_user_map m = {c.mt_a[di], c.mt_b[di], c.mt_c[di], t1 - t0};
            UP::template map<BS>(m, t - t0, env, static_cast<void *>(&sm.u));
            __syncthreads();  // the shared memory is the next unit's
        }
    }
    if constexpr ((PM & PM_MS) != 0u) {
      if (nt1) {
        // leaves: one warp each
        const uint32_t gw = (blockIdx.x * BS + threadIdx.x) >> 5, nw = gridDim.x * (BS / 32);
        for (uint32_t t = gw; t < nt1; t += nw) {
            const uint32_t di = tile_owner(c, t, nd1, nt1);
            if (c.mt_kind[di] != MAP_LEAF_SORT) continue;
            job_buffers(c, job_params, job_stride, c.mt_job[di], &keys, &scratch);
            const uint32_t cc = c.mt_c[di];
            warp_leaf_sort(keys, (cc & 1u) ? scratch : keys, c.mt_a[di], c.mt_b[di], job_params ? nullptr : c.smp);
        }
        // merge tiles: one block each, pipelined
        merge_phase<BS>(c, ctl, sm, nt1, nd1, job_params, job_stride);
      }
    }
    if constexpr ((PM & (PM_BFS | PM_SSSP | PM_FFT)) != 0u) {
        const bool fft = (PM & PM_FFT) != 0u && ((PM & (PM_BFS | PM_SSSP)) == 0u || c.rp.program == TREES_PROG_FFT);
        if constexpr ((PM & PM_FFT) != 0u) {
            if (fft) {
                if (nd2) fft_combine_map<BS>(c, nd2, ne2);
                return;
            }
        }
        if constexpr ((PM & (PM_BFS | PM_SSSP)) != 0u) {
            const bool sssp = (PM & PM_BFS) == 0u || ((PM & PM_SSSP) != 0u && c.rp.program == TREES_PROG_SSSP);
            constexpr uint32_t P = EXPAND_PARTS(BS);
            const uint32_t h = threadIdx.x / (uint32_t)(BS / P);  // the parts take interleaved tiles
            const uint32_t lt = threadIdx.x - h * (uint32_t)(BS / P);
            if (sssp) {
                // a part's claim buffer: claim_cap entries of the caller's buffer, or none (per-tile forks)
                uint32_t *cb = claims && claim_cap >= expand_tile_len(BS) + 32u ? claims + h * claim_cap : nullptr;
                uint32_t t = P * blockIdx.x + h;
                if (t < nt2) {
                    if (cb && lt == 0u) sm.pcnt[h] = 0u;  // the tile's descriptor load ends with a barrier of the part
                    for (; t < nt2; t += P * gridDim.x)
                        relax_tile<BS>(c, ctl, sm, t, nd2, ne2, nt2, cen, base, ep, e, h, cb, claim_cap);
                    if (cb)  // the candidates left in the buffer
                        sssp_claim_flush<BS>(c, ctl, sm, cb, claim_cap, h, lt, cen, base, ep, e);
                }
            } else {
                uint32_t t = P * blockIdx.x + h;
                if (t < nt2) {
                    if (lt == 0u) sm.pcnt[h] = 0u;  // load_tile_descriptors ends with a barrier of the part
                    uint32_t nloc = load_tile_descriptors<BS, false>(c, sm, t, nd2, nt2, h, lt);
                    for (; t < nt2; t += P * gridDim.x)
                        nloc = expand_tile<BS>(c, ctl, sm, t, t + P * gridDim.x, nloc, nd2, ne2, nt2, cen, base, ep,
                                               e, h);
                    bfs_claim_flush<BS>(c, ctl, sm, claim_buf<BS>(sm, h), h, lt, cen, base, ep, e);  // the candidates left
                }
            }
        }
    }
}

// True when some merge of the tiled list spans several tiles, so the
// partition sub-phase has splits to compute.
__device__ __forceinline__ bool needs_partition(unsigned long long mt) {
    return (uint32_t)(mt & CTR_LOW_MASK) > (uint32_t)(mt >> 40);
}

}  // namespace trees
