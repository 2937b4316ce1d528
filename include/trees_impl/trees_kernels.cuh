// The persistent epoch-loop kernel, compiled once per program (see the
// trees_k_*.cu translation units) so each kernel carries only its program's
// task types and maps.
#pragma once

#include "trees_dev.cuh"
#include "trees_programs.cuh"

namespace trees {

template <int BS>
__device__ __forceinline__ void block_add_stats(unsigned long long *blk, const Acc &acc, Smem<BS> &sm) {
    // block-reduce the per-thread counters, then one add per counter per block
    const uint32_t v = __reduce_add_sync(0xffffffffu, acc.valid);
    const uint32_t j = __reduce_add_sync(0xffffffffu, acc.joins);
    const uint32_t m = __reduce_add_sync(0xffffffffu, acc.maps);
    __syncthreads();
    if (threadIdx.x == 0) {
        sm.bc64[0] = 0;
        sm.bc64[1] = 0;
        sm.bc64[2] = 0;
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&sm.bc64[0], (unsigned long long)v);
        atomicAdd(&sm.bc64[1], (unsigned long long)j);
        atomicAdd(&sm.bc64[2], (unsigned long long)m);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long *b = blk + 4ull * (blockIdx.x % NBLK_STATS);
        atomicAdd(b + 0, sm.bc64[0]);
        atomicAdd(b + 1, sm.bc64[1]);
        atomicAdd(b + 2, sm.bc64[2]);
    }
}

template <int BS>
__device__ __forceinline__ void trace_valid_add(const Conf &c, uint32_t e, uint32_t v, Smem<BS> &sm) {
    if (!c.trace_on || e >= c.trace_cap) return;
    const uint32_t w = __reduce_add_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0 && w) atomicAdd(&c.trace_valid[e], w);
}

// The persistent scheduler: the whole epoch loop in one cooperative launch.
// Blocks per SM the kernel is compiled to fit (its register budget): the
// mergesort, BFS and SSSP kernels keep 1024 threads per SM resident (their
// map tiles would otherwise take registers for 2 blocks per SM: measured
// SSSP R-MAT 22 6.1 -> 3.8 ms, BFS 1.63 -> 1.23 ms); the fib kernel trades
// threads for registers as its slots per thread grow (1024, 768, 512 threads
// per SM for 1, 2, 4 slots: measured, each spill-free beats more resident
// warps that spill); the FFT kernel keeps 512 (128 registers: its leaf
// transforms and combine butterflies spill at 64), and so does a user
// program's (its device functions are unknown here); the others take what
// they need.
__host__ __device__ constexpr int persistent_min_blocks(int bs, uint32_t pm, int tpt) {
    const int tps = (pm == PM_MS || pm == PM_BFS || pm == PM_SSSP) ? 1024 : (pm == PM_FFT || pm == PM_USER) ? 512
                  : pm == PM_FIB ? (tpt >= 4 ? 512 : tpt == 2 ? 768 : 1024) : 0;
    return tps / bs > 0 ? tps / bs : 1;
}

// Dynamic shared memory of a persistent kernel.  The fib kernels run their
// join ranges through a ring of asynchronous copies there (fib_join_tiles):
// NA stages of (code, link) and NB of result pairs, 8 and 16 bytes per slot,
// (NA, NB) = (5, 3) when that fits beside the kernel's static shared memory
// at the residency its register budget targets (228 KB per SM, 1 KB of it
// reserved per block), else (4, 3), else (3, 2), else no ring (the register
// path).  NA - NB tiles of lookahead hide the (code, link) copies, NB - 1 the
// operand copies: (5, 3) measured 0.4403 ms per fib(34) at 512 x 2 against
// 0.4464 ms for (4, 3) in one A/B call; (6, 3) and (7, 4) gave the same as (5, 3).
constexpr int SMEM_PER_SM = 228 * 1024, SMEM_RESERVED_PER_BLOCK = 1024;

// Ranges of at most SOLO_TILES tiles, for programs without map operations,
// are worked by block 0 alone, epoch after epoch, each closed by a block
// barrier instead of a grid barrier: the same epochs, ranges and fork counts
// without the grid-wide round trip, which costs more than a tile or two of
// work.
constexpr uint32_t SOLO_TILES = 2;  // measured: 1 or 2 tiles best; 4 already slower

template <int BS, int TPT, uint32_t PM>
__host__ __device__ constexpr int ring_budget() {
    return PM != PM_FIB ? 0
                        : SMEM_PER_SM / persistent_min_blocks(BS, PM, TPT) - SMEM_RESERVED_PER_BLOCK -
                              ((int)sizeof(Smem<BS>) + 256);  // the block's static shared memory, rounded up
}

// (NA, NB) packed as NA * 16 + NB, or 0.
template <int BS, int TPT, uint32_t PM>
__host__ __device__ constexpr int ring_depths() {
    return ring_budget<BS, TPT, PM>() >= 88 * BS * TPT ? 5 * 16 + 3
           : ring_budget<BS, TPT, PM>() >= 80 * BS * TPT ? 4 * 16 + 3
           : ring_budget<BS, TPT, PM>() >= 56 * BS * TPT ? 3 * 16 + 2
                                                         : 0;
}

template <int BS, int TPT, uint32_t PM>
__host__ __device__ constexpr size_t join_ring_bytes() {
    return (size_t)((ring_depths<BS, TPT, PM>() >> 4) * 8 + (ring_depths<BS, TPT, PM>() & 15) * 16) * BS * TPT;
}

// After the join ring, the rest of the budget holds block 0's shadow of the
// task vector's first slots for fib's solo runs (fib_solo_epoch): code, n,
// link and result, 20 bytes per slot, for up to 2 * SOLO_TILES tiles of slots
// (the most a run of solo fresh epochs allocates from slot 0: each range at
// most SOLO_TILES tiles, each the children of the one before).
constexpr uint32_t SHADOW_BYTES_PER_SLOT = 20;

template <int BS, int TPT, uint32_t PM>
__host__ __device__ constexpr uint32_t shadow_slots() {
    return PM != PM_FIB || ring_budget<BS, TPT, PM>() <= (int)join_ring_bytes<BS, TPT, PM>() ? 0u
           : ((uint32_t)(ring_budget<BS, TPT, PM>() - (int)join_ring_bytes<BS, TPT, PM>()) / SHADOW_BYTES_PER_SLOT <
                      2u * SOLO_TILES * (uint32_t)(BS * TPT)
                  ? (uint32_t)(ring_budget<BS, TPT, PM>() - (int)join_ring_bytes<BS, TPT, PM>()) / SHADOW_BYTES_PER_SLOT
                  : 2u * SOLO_TILES * (uint32_t)(BS * TPT)) & ~3u;
}

template <int BS, int TPT, uint32_t PM>
__host__ __device__ constexpr size_t ring_bytes() {
    return join_ring_bytes<BS, TPT, PM>() + (size_t)SHADOW_BYTES_PER_SLOT * shadow_slots<BS, TPT, PM>();
}

// Dynamic shared memory bytes k_persistent<bs, tpt, program mask pm> is launched with:
// fib's join ring and solo shadow (ring_bytes), the FFT leaf epoch's buffers
// (fft_leaf_dyn_bytes), SSSP's claim buffers (sssp_claim_cap), else none.
// SSSP's persistent kernels keep each block part's claim buffer (relax_tile)
// in dynamic shared memory: claim_cap_of(BS) entries a part, for blocks of
// 512 threads or more when that fits beside the static shared memory at the
// kernel's residency, else none (the per-tile reservation path).  Smaller
// blocks run four or more per SM, and their buffers would take the SM's
// shared memory to ~230 KB of its 256 KB, leaving the L1 cache the tiles'
// gathers use ~25 KB (SSSP R-MAT 22 at 256 x 2: 2.80 -> 4.5-4.65 ms).
template <int BS, int TPT>
__host__ __device__ constexpr uint32_t sssp_claim_cap() {
    return BS >= 512 && SMEM_PER_SM / persistent_min_blocks(BS, PM_SSSP, TPT) - SMEM_RESERVED_PER_BLOCK -
                                ((int)sizeof(Smem<BS>) + 256) >=
                            (int)(4u * EXPAND_PARTS(BS) * claim_cap_of(BS))
               ? claim_cap_of(BS)
               : 0u;
}

// The FFT leaf epoch's buffers (fft_leaf_epoch): the next slot's 16 input
// points and a warp's 16 staged outputs per thread, 256 bytes a thread, in
// dynamic shared memory for a kernel that runs one block per SM and has the
// room beside its static shared memory; else the input buffer alone in the
// shared union when it fits there (blocks of up to 256 threads), the output
// buffer too when that fits (128 threads).  Two blocks per SM at 256 threads
// with both buffers in dynamic shared memory left the L1 cache ~28 KB and
// were slower (2^24 points, 256 x 1: 1.11 -> 1.25 ms); one block of 512
// threads gained (1.198 -> 1.094 ms).
template <int BS, int TPT, uint32_t PM>
__host__ __device__ constexpr size_t fft_leaf_dyn_bytes() {
    return PM == PM_FFT && persistent_min_blocks(BS, PM, TPT) == 1 &&
                   (size_t)BS * 32u * sizeof(float2) > sizeof(Smem<BS>::u) &&
                   SMEM_PER_SM / persistent_min_blocks(BS, PM, TPT) - SMEM_RESERVED_PER_BLOCK -
                           ((int)sizeof(Smem<BS>) + 256) >=
                       (int)(BS * 32 * sizeof(float2))
               ? (size_t)BS * 32u * sizeof(float2)
               : 0u;
}

template <int BS, int TPT, uint32_t PM>
__host__ __device__ constexpr size_t dyn_smem_bytes() {
    return PM == PM_FIB ? ring_bytes<BS, TPT, PM>()
           : PM == PM_FFT ? fft_leaf_dyn_bytes<BS, TPT, PM>()
           : PM == PM_SSSP ? (size_t)4u * EXPAND_PARTS(BS) * sssp_claim_cap<BS, TPT>()
                           : 0u;
}

inline size_t persistent_smem_bytes(uint32_t pm, int bs, int tpt) {
    if (pm == PM_FFT) {
        switch (bs * 10 + tpt) {
        case 1281: return dyn_smem_bytes<128, 1, PM_FFT>();
        case 1282: return dyn_smem_bytes<128, 2, PM_FFT>();
        case 1284: return dyn_smem_bytes<128, 4, PM_FFT>();
        case 2561: return dyn_smem_bytes<256, 1, PM_FFT>();
        case 2562: return dyn_smem_bytes<256, 2, PM_FFT>();
        case 2564: return dyn_smem_bytes<256, 4, PM_FFT>();
        case 5121: return dyn_smem_bytes<512, 1, PM_FFT>();
        case 5122: return dyn_smem_bytes<512, 2, PM_FFT>();
        case 5124: return dyn_smem_bytes<512, 4, PM_FFT>();
        case 10241: return dyn_smem_bytes<1024, 1, PM_FFT>();
        case 10242: return dyn_smem_bytes<1024, 2, PM_FFT>();
        case 10244: return dyn_smem_bytes<1024, 4, PM_FFT>();
        default: return 0;
        }
    }
    if (pm == PM_SSSP) {
        switch (bs * 10 + tpt) {
        case 1281: return dyn_smem_bytes<128, 1, PM_SSSP>();
        case 1282: return dyn_smem_bytes<128, 2, PM_SSSP>();
        case 1284: return dyn_smem_bytes<128, 4, PM_SSSP>();
        case 2561: return dyn_smem_bytes<256, 1, PM_SSSP>();
        case 2562: return dyn_smem_bytes<256, 2, PM_SSSP>();
        case 2564: return dyn_smem_bytes<256, 4, PM_SSSP>();
        case 5121: return dyn_smem_bytes<512, 1, PM_SSSP>();
        case 5122: return dyn_smem_bytes<512, 2, PM_SSSP>();
        case 5124: return dyn_smem_bytes<512, 4, PM_SSSP>();
        case 10241: return dyn_smem_bytes<1024, 1, PM_SSSP>();
        case 10242: return dyn_smem_bytes<1024, 2, PM_SSSP>();
        case 10244: return dyn_smem_bytes<1024, 4, PM_SSSP>();
        default: return 0;
        }
    }
    if (pm != PM_FIB) return 0;
    switch (bs * 10 + tpt) {
    case 1281: return ring_bytes<128, 1, PM_FIB>();
    case 1282: return ring_bytes<128, 2, PM_FIB>();
    case 1284: return ring_bytes<128, 4, PM_FIB>();
    case 2561: return ring_bytes<256, 1, PM_FIB>();
    case 2562: return ring_bytes<256, 2, PM_FIB>();
    case 2564: return ring_bytes<256, 4, PM_FIB>();
    case 5121: return ring_bytes<512, 1, PM_FIB>();
    case 5122: return ring_bytes<512, 2, PM_FIB>();
    case 5124: return ring_bytes<512, 4, PM_FIB>();
    case 10241: return ring_bytes<1024, 1, PM_FIB>();
    case 10242: return ring_bytes<1024, 2, PM_FIB>();
    case 10244: return ring_bytes<1024, 4, PM_FIB>();
    default: return 0;
    }
}

// Scheduler state a persistent block carries between epochs.  Only thread 0
// touches it, so it lives in shared memory rather than in every thread's
// registers.
struct SchedState {
    unsigned long long forks_total;
    uint32_t peak;
    uint32_t bar;  // grid barriers passed
    // trace timestamps (block 0): previous epoch's end, end of Phase 2, of partition, of maps
    unsigned long long t_prev, t_p2, t_pt, t_mp;
    unsigned long long t_solo;  // start of the current solo run
    uint32_t sh_hi;             // fib: slots [0, sh_hi) have a current shadow entry (fib_solo_epoch)
};

// Phase 1 (thread 0): pop (CEN, NDRange) for epoch e and set
// oldNextFreeCore = nextFreeCore, or stop; block 0 clears the counters epoch
// e+1 will use.
template <int BS>
__device__ __forceinline__ void phase1(const Conf &c, Ctl *ctl, Smem<BS> &sm, uint32_t e) {
    int stop = 0;
    if (sm.sp == 0) {
        stop = 1;
    } else if (e >= c.max_epochs) {
        stop = 2;
        set_err(ctl, TREES_ERR_EPOCH_LIMIT, e);
    } else {
        const Range r = sm.stk[--sm.sp];
        sm.cen = r.cen;
        sm.lo = r.lo;
        sm.hi = r.hi;
        sm.rjoin = r.join;
        sm.base = sm.next;
    }
    sm.stop = stop;
    if (!stop && blockIdx.x == 0) clear_epoch_slot(ctl, (e + 1u) % 3u);
}

// Phase 3 (thread 0): push the join range, then the fork range; or give the
// range back.  Block 0 also keeps the run's statistics and writes the trace.
template <int BS>
__device__ __forceinline__ void phase3(const Conf &c, Ctl *ctl, Smem<BS> &sm, uint32_t e, uint32_t f, uint32_t jf,
                                       unsigned long long mt, unsigned long long me, SchedState &st) {
    const uint32_t cen = sm.cen, lo = sm.lo, hi = sm.hi, base = sm.base;
    int ok = 1;
    if (jf) {
        if (sm.sp < STK_CAP) sm.stk[sm.sp++] = Range{cen, lo, hi, 1u};
        else ok = 0;
    }
    if (f) {
        if (sm.sp < STK_CAP) sm.stk[sm.sp++] = Range{cen + 1u, base, base + f, 0u};
        else ok = 0;
        sm.next = base + f;
    } else if (!jf) {
        sm.next = lo;  // neither forks nor joins: nextFreeCore decreases (Sec. 5.3)
    }
    if (!ok) {
        if (blockIdx.x == 0) set_err(ctl, TREES_ERR_STACK, e);
        sm.sp = 0;
    }
    if (blockIdx.x == 0) {
        st.forks_total += f;
        st.peak = max(st.peak, base + f);
        if (c.trace_on && e < c.trace_cap) {
            trees_epoch_t r;
            r.cen = cen;
            r.lo = lo;
            r.hi = hi;
            r.valid = 0u;
            r.forks = f;
            r.joined = jf;
            r.maps = (uint32_t)(mt >> 40) + (uint32_t)(me >> 40);
            r.t_ns = globaltimer();
            r.ns_phase2 = (uint32_t)(st.t_p2 - st.t_prev);
            r.ns_partition = (uint32_t)(st.t_pt - st.t_p2);
            r.ns_map = (uint32_t)(st.t_mp - st.t_pt);
            st.t_prev = r.t_ns;
            c.trace[e] = r;
        }
    }
}

template <int BS, int TPT, uint32_t PM>
__device__ __forceinline__ bool solo_range(const Conf &c, uint32_t lo, uint32_t hi) {
    return (PM & PM_MAPS) == 0u && c.stall_epoch < 0 && hi - lo <= SOLO_TILES * (uint32_t)(BS * TPT);
}

// Block 0's shadow of the task vector's slots [0, cap) (fib; the dynamic
// shared memory after the join ring).  Slots below SchedState::sh_hi hold the
// current code, n, link and result there: those slots are written by block 0
// alone from the solo epoch that brought them in until a grid epoch whose
// range starts at or below them (a grid epoch writes only its own range and
// the children above it, so it lowers sh_hi to its range's start).
struct FibShadow {
    unsigned long long *res;
    uint32_t *code, *a0, *link;
    uint32_t cap;
};

template <int BS, int TPT, uint32_t PM>
__device__ __forceinline__ FibShadow fib_shadow(uint32_t *ring) {
    constexpr uint32_t S = shadow_slots<BS, TPT, PM>();
    FibShadow sh;
    sh.res = reinterpret_cast<unsigned long long *>(reinterpret_cast<char *>(ring) + join_ring_bytes<BS, TPT, PM>());
    sh.code = reinterpret_cast<uint32_t *>(sh.res + S);
    sh.a0 = sh.code + S;
    sh.link = sh.a0 + S;
    sh.cap = S;
    return sh;
}

// One solo epoch of fib (Sec. 6.2's tasks; the range is at most SOLO_TILES
// tiles): every thread loads all its slots of the range at once, from the
// shadow where it holds them, else from the task vector; a fresh range's
// internal tasks take their children after one block-wide count (block 0
// forks all of the epoch's children, so no atomic is needed: they start at
// oldNextFreeCore, row by row of the range, each warp's children of a row
// contiguous so its stores coalesce), a join range's sums read their
// operands from the shadow or the task vector.  Every write goes to the task
// vector and, for slots below cap, to the shadow.  A fresh range starting at
// sh_hi is copied into the shadow as it is read and raises sh_hi to its end;
// children placed at sh_hi raise it past them.  Thread 0 updates sh_hi
// (every thread reads it after the block barrier that closes the epoch).
template <int BS, int TPT>
__device__ __forceinline__ TileOut fib_solo_epoch(const Conf &c, Ctl *ctl, Smem<BS> &sm, const FibShadow &sh,
                                                  uint32_t &sh_hi, uint32_t lo, uint32_t hi, uint32_t cen,
                                                  uint32_t base, uint32_t e, int mode, Acc &acc) {
    constexpr int R = (int)SOLO_TILES * TPT;  // rows of BS slots: the range is slots lo + j * BS + thread, j < R
    const uint32_t hv = sh_hi, tid = threadIdx.x;
    uint32_t cd[R], x[R];  // code, and n (fresh) or link (join)
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const uint32_t s = lo + (uint32_t)j * BS + tid;
        const bool in = s < hi, shd = s < hv;
        cd[j] = !in ? 0u : shd ? sh.code[s] : c.code[s];
        x[j] = !in ? 0u : mode == LOAD_FRESH ? (shd ? sh.a0[s] : c.a0[s]) : (shd ? sh.link[s] : c.link[s]);
    }
    TileOut out = {0u, false, false};
    if (mode == LOAD_FRESH) {
        const bool fill = lo == hv;  // block-uniform
        uint32_t fm = 0u;  // which of this thread's rows fork
#pragma unroll
        for (int j = 0; j < R; ++j) {
            const uint32_t s = lo + (uint32_t)j * BS + tid;
            if (fill && s < hi && s < sh.cap) {
                sh.code[s] = cd[j];
                sh.a0[s] = x[j];
            }
            const uint32_t t = task_type(cd[j], cen);
            if (!t) continue;
            acc.valid++;
            if (t == TREES_TASK_FIB) {
                const uint32_t n = x[j];
                if (n < 2u || n <= c.rp.cutoff) {  // a leaf emits in its own slot; the entry is dead
                    const unsigned long long r = n < 2u ? (unsigned long long)n : fib_leaf(n);
                    c.result[s] = r;
                    c.code[s] = 0u;
                    if (s < sh.cap) {
                        sh.res[s] = r;
                        sh.code[s] = 0u;
                    }
                } else {
                    fm |= 1u << j;
                }
            } else {  // not produced in a fresh range: run it as the general path would
                Plan p;
                p.s = s;
                p.t = t;
                p.n = 0u;
                p.m = 0u;
                plan_task<PM_FIB, merge_tile(BS)>(c, c.rp, p, cen, e, x[j], 0u, c.link[s]);
                if (s < sh.cap) {  // this thread's own writes, read back
                    sh.code[s] = c.code[s];
                    sh.res[s] = c.result[s];
                }
            }
        }
        // forking tasks per (row, warp): one ballot per row, the warp counts in the shared union, one barrier,
        // then every warp scans a row's warp counts with shuffles; rows past the range are skipped
        constexpr int NW = BS / 32;
        const uint32_t lane = tid & 31u, wid = tid >> 5, lt = (1u << lane) - 1u;
        const uint32_t nrow = (hi - lo + (uint32_t)BS - 1u) / (uint32_t)BS;  // block-uniform, at most R
        uint32_t *wc = reinterpret_cast<uint32_t *>(&sm.u);  // [R][NW]
        uint32_t m[R];
#pragma unroll
        for (int j = 0; j < R; ++j) {
            m[j] = 0u;
            if ((uint32_t)j < nrow) {
                m[j] = __ballot_sync(0xffffffffu, (fm >> j) & 1u);
                if (lane == (uint32_t)j) wc[j * NW + wid] = (uint32_t)__popc(m[j]);
            }
        }
        __syncthreads();
        uint32_t pre[R], tot[R], total = 0u;
#pragma unroll
        for (int j = 0; j < R; ++j) {
            pre[j] = tot[j] = 0u;
            if ((uint32_t)j < nrow) {
                const uint32_t q = lane < (uint32_t)NW ? wc[j * NW + lane] : 0u, inc = warp_incl_u32(q);
                tot[j] = __shfl_sync(0xffffffffu, inc, NW - 1);
                pre[j] = __shfl_sync(0xffffffffu, inc - q, (int)wid);
                total += 2u * tot[j];
            }
        }
        const bool over = (unsigned long long)base + total > c.cap;
        if (over && tid == 0) set_err(ctl, TREES_ERR_CAPACITY, e);
        if (!over && fm) {
            const uint32_t fe = enc(cen + 1u, TREES_TASK_FIB), fj = enc(cen, TREES_TASK_FIB_SUM);
            uint32_t rbase = base;  // children of row j start after those of rows 0..j-1
#pragma unroll
            for (int j = 0; j < R; ++j) {
                const uint32_t child = rbase + 2u * (pre[j] + (uint32_t)__popc(m[j] & lt));
                rbase += 2u * tot[j];
                if (!((fm >> j) & 1u)) continue;
                const uint32_t s = lo + (uint32_t)j * BS + tid, n = x[j];
                c.code[child] = fe;
                c.a0[child] = n - 1u;
                c.code[child + 1] = fe;
                c.a0[child + 1] = n - 2u;
                c.link[s] = child;
                c.code[s] = fj;
                if (child < sh.cap) {
                    sh.code[child] = fe;
                    sh.a0[child] = n - 1u;
                }
                if (child + 1u < sh.cap) {
                    sh.code[child + 1] = fe;
                    sh.a0[child + 1] = n - 2u;
                }
                if (s < sh.cap) {
                    sh.link[s] = child;
                    sh.code[s] = fj;
                }
                acc.joins++;
            }
            out.joined = true;
        }
        if (tid == 0) {  // every thread has read sh_hi before the count's barrier
            uint32_t h = hv;
            if (fill) h = hi < sh.cap ? hi : sh.cap;
            if (!over && total && base == h) h = base + total < sh.cap ? base + total : sh.cap;
            sh_hi = h;
        }
        out.forks = total;
        out.over = over;
        return out;
    }
    // a join range: sums only (fib's continuations never fork)
    unsigned long long r0[R], r1[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
        r0[j] = r1[j] = 0ull;
        if (task_type(cd[j], cen) == TREES_TASK_FIB_SUM) {
            const uint32_t lk = x[j];
            r0[j] = lk < hv ? sh.res[lk] : c.result[lk];
            r1[j] = lk + 1u < hv ? sh.res[lk + 1] : c.result[lk + 1];
        }
    }
#pragma unroll
    for (int j = 0; j < R; ++j) {
        const uint32_t s = lo + (uint32_t)j * BS + tid, t = task_type(cd[j], cen);
        if (!t) continue;
        acc.valid++;
        if (t == TREES_TASK_FIB_SUM) {
            const unsigned long long v = r0[j] + r1[j];
            c.result[s] = v;
            c.code[s] = 0u;
            if (s < sh.cap) {
                sh.res[s] = v;
                sh.code[s] = 0u;
            }
        } else {  // not produced in a join range; run it as the general path would
            Plan p;
            p.s = s;
            p.t = t;
            p.n = 0u;
            p.m = 0u;
            plan_task<PM_FIB, merge_tile(BS)>(c, c.rp, p, cen, e, c.a0[s], 0u, x[j]);
            if (s < sh.cap) {
                sh.code[s] = c.code[s];
                sh.res[s] = c.result[s];
            }
        }
    }
    return out;
}

// Block 0's run of solo epochs, starting at epoch e with its range popped.
// Returns the epoch whose range is popped when the run ends (a range too
// large for one tile, the end of the job, an error, or a quarter of the
// barrier timeout spent, so the waiting blocks never time out); block 0's
// state (stack, nextFreeCore, popped range, stop) is then published for the
// other blocks.
template <int BS, int TPT, uint32_t PM>
__device__ uint32_t solo_epochs(const Conf &c, Ctl *ctl, Smem<BS> &sm, uint32_t e, Acc &acc, SchedState &st,
                                uint32_t *ring) {
    if (threadIdx.x == 0) st.t_solo = globaltimer();
    for (;;) {
        const uint32_t cen = sm.cen, lo = sm.lo, hi = sm.hi, base = sm.base, ep = e % 3u;
        const int mode = sm.rjoin ? LOAD_JOIN : LOAD_FRESH;
        const uint32_t v0 = acc.valid;
        TileOut o = {0u, false, false};
        if constexpr (PM == PM_FIB) {
            o = fib_solo_epoch<BS, TPT>(c, ctl, sm, fib_shadow<BS, TPT, PM>(ring), st.sh_hi, lo, hi, cen, base, e,
                                        mode, acc);
        } else {
            // the range's tiles in order, each forking after the children of the ones before it
            TileLoad<TPT> cur, nxt;
            if (lo < hi) tile_load<BS, TPT, PM>(c, lo, hi, mode, cur);
            int par = 0;
            for (uint32_t t0 = lo; t0 < hi; t0 += (uint32_t)(BS * TPT)) {
                const bool more = t0 + (uint32_t)(BS * TPT) < hi;
                if (more) tile_load<BS, TPT, PM>(c, t0 + (uint32_t)(BS * TPT), hi, mode, nxt);
                if constexpr (joins_never_fork<PM>()) {
                    if (mode == LOAD_JOIN) {  // continuations only: no scan, no allocation
                        join_tile<BS, TPT, PM>(c, sm, t0, cen, e, acc, par, cur, false, nullptr);
                        if (more) cur = nxt;
                        par ^= 1;
                        continue;
                    }
                }
                const TileOut t = epoch_tile<BS, TPT, PM>(c, ctl, sm, t0, hi, cen, base, ep, e, acc, par, mode,
                                                          cur, true, o.forks);
                o.forks += t.forks;
                o.joined |= t.joined;
                o.over |= t.over;
                if (more) cur = nxt;
                par ^= 1;
            }
        }
        trace_valid_add<BS>(c, e, acc.valid - v0, sm);
        // the whole epoch is this block's tile: its fork total and join flag close the epoch
        const uint32_t jf = (uint32_t)__syncthreads_or(o.joined);
        if (threadIdx.x == 0) {
            if (c.trace_on) st.t_p2 = st.t_pt = st.t_mp = globaltimer();
            phase3<BS>(c, ctl, sm, e, o.forks, jf, 0ull, 0ull, st);
            phase1<BS>(c, ctl, sm, e + 1u);
            if (o.over) sm.stop = 3;  // the capacity error is set; the grid barrier reports it
            sm.solo_late = globaltimer() - st.t_solo > c.timeout_ns / 4u;
        }
        ++e;  // on every thread: the epoch number picks the counter slot and the trace entry
        __syncthreads();
        if (sm.stop || sm.solo_late || !solo_range<BS, TPT, PM>(c, sm.lo, sm.hi)) break;
    }
    if (threadIdx.x == 0) {
        ctl->g_e = e;
        ctl->g_sp = (uint32_t)sm.sp;
        ctl->g_next = sm.next;
        ctl->g_cen = sm.cen;
        ctl->g_lo = sm.lo;
        ctl->g_hi = sm.hi;
        ctl->g_base = sm.base;
        ctl->g_rjoin = sm.rjoin;
        ctl->g_stop = (uint32_t)sm.stop;
        for (int i = 0; i < sm.sp; ++i) c.gstack[i] = sm.stk[i];
    }
    return e;
}

// The other blocks take over block 0's published state after the grid
// barrier that ends the solo run: thread 0 the scalars, then every thread a
// share of the stack.  Returns the epoch whose range is popped.
template <int BS>
__device__ __forceinline__ uint32_t adopt_solo_state(const Conf &c, Ctl *ctl, Smem<BS> &sm) {
    if (threadIdx.x == 0) {
        sm.sp = (int)vload(&ctl->g_sp);
        sm.next = vload(&ctl->g_next);
        sm.cen = vload(&ctl->g_cen);
        sm.lo = vload(&ctl->g_lo);
        sm.hi = vload(&ctl->g_hi);
        sm.base = vload(&ctl->g_base);
        sm.rjoin = vload(&ctl->g_rjoin);
        sm.stop = (int)vload(&ctl->g_stop);
        sm.bc32[0] = vload(&ctl->g_e);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < sm.sp; i += BS) {
        const uint4 r = __ldcg(reinterpret_cast<const uint4 *>(c.gstack + i));  // past any stale L1 line
        sm.stk[i] = Range{r.x, r.y, r.z, r.w};
    }
    return sm.bc32[0];
}

template <int BS, int TPT, uint32_t PM, typename UP = NoUserProgram>
__global__ void __launch_bounds__(BS, persistent_min_blocks(BS, PM, TPT)) k_persistent(Ctl *ctl, Conf c, unsigned long long *blk) {
    __shared__ Smem<BS> sm;
    __shared__ uint32_t sm_e;
    __shared__ SchedState st;
    extern __shared__ __align__(16) uint32_t ring[];  // dyn_smem_bytes<BS, TPT, PM>() of dynamic shared memory
    Acc acc = {0u, 0u, 0u};
    if (threadIdx.x == 0) {
        st = SchedState{0ull, 1u, 0u, 0ull, 0ull, 0ull, 0ull, 0ull, 0u};
        sm.sp = 1;
        sm.stk[0] = Range{0u, 0u, 1u, 0u};
        sm.next = 1u;
        if (c.trace_on && blockIdx.x == 0) st.t_prev = globaltimer();
    }
    const bool stamp = c.trace_on && blockIdx.x == 0 && threadIdx.x == 0;
    bool popped = false;  // epoch e's range was popped by a solo run
    uint32_t e = 0;
    for (;; ++e) {
        // Phase 1: pop (CEN, NDRange); oldNextFreeCore = nextFreeCore
        if (threadIdx.x == 0 && !popped) phase1<BS>(c, ctl, sm, e);
        popped = false;
        __syncthreads();
        if (sm.stop) break;
        if constexpr ((PM & PM_MAPS) == 0u) {
            if (solo_range<BS, TPT, PM>(c, sm.lo, sm.hi)) {
                if (blockIdx.x == 0) {
                    const uint32_t ne = solo_epochs<BS, TPT, PM>(c, ctl, sm, e, acc, st, ring);
                    if (threadIdx.x == 0) sm_e = ne;
                }
                if (!grid_sync_ep<BS>(ctl, &st.bar, c.timeout_ns, sm, e % 3u)) break;
                if (blockIdx.x != 0) {
                    const uint32_t ne = adopt_solo_state<BS>(c, ctl, sm);
                    if (threadIdx.x == 0) sm_e = ne;
                }
                __syncthreads();
                e = sm_e - 1u;  // the loop's ++e lands on the popped epoch
                popped = true;
                continue;
            }
        }
        const uint32_t cen = sm.cen, lo = sm.lo, hi = sm.hi, base = sm.base, ep = e % 3u;
        const int mode = sm.rjoin ? LOAD_JOIN : LOAD_FRESH;
        if constexpr (PM == PM_FIB) {  // this grid epoch writes slots from lo up: the shadow ends below them
            if (threadIdx.x == 0 && st.sh_hi > lo) st.sh_hi = lo;
        }
        // Phase 2: every entry of [lo, hi)
        const uint32_t v0 = acc.valid;
        // tiles grid-stride over [lo, hi); the next tile's columns load while this one runs
        int par = 0;
        const bool solo = hi - lo <= (uint32_t)(BS * TPT);  // only block 0 has a tile
        const unsigned long long step = (unsigned long long)gridDim.x * (BS * TPT);
        unsigned long long t0 = (unsigned long long)lo + (unsigned long long)blockIdx.x * (BS * TPT);
        bool jn = false;     // some task of this thread joined (joinScheduled)
        bool done = false;   // Phase 2 ran on one of the specialised paths
        if constexpr (PM == PM_FIB) {
            if (mode == LOAD_FRESH && !solo) {  // count, one reservation per chunk, write
                jn = fib_fresh_tiles<BS, TPT>(c, ctl, sm, t0, step, hi, cen, base, ep, e, acc);
                done = true;
            }
        }
        if constexpr (PM == PM_FFT) {  // every task of an FFT epoch has depth CEN: the width fixes forks and maps
            const uint32_t lgm = cen <= c.rp.lgn ? c.rp.lgn - cen : 0u;
            if (mode == LOAD_FRESH && lgm == 4u && c.rp.leaf >= 16u) {
                constexpr size_t FD = fft_leaf_dyn_bytes<BS, TPT, PM>();
                fft_leaf_epoch<BS, TPT, FD ? FD : sizeof(sm.u)>(
                    c, FD ? reinterpret_cast<float2 *>(ring) : reinterpret_cast<float2 *>(&sm.u), t0, step, hi, cen, acc);  // 16-point leaves only: no forks, no scan
                done = true;
            } else if (mode == LOAD_FRESH && cen <= c.rp.lgn && (1u << lgm) > c.rp.leaf) {
                jn = fft_fork_epoch<BS, TPT>(c, ctl, t0, step, lo, hi, cen, base, ep, e, acc);
                done = true;
            } else if (mode == LOAD_JOIN && lgm >= 1u && (1u << lgm) > c.rp.cutoff) {
                fft_combine_epoch<BS, TPT>(c, ctl, t0, step, lo, hi, cen, ep, acc);
                done = true;
            }
        }
        if constexpr (PM == PM_FIB && ring_depths<BS, TPT, PM>() != 0) {
            if (mode == LOAD_JOIN) {  // sums through the ring of asynchronous copies
                constexpr int RD = ring_depths<BS, TPT, PM>();
                fib_join_tiles<BS, TPT, (RD >> 4), (RD & 15)>(c, t0, step, hi, cen, e, acc, ring);
                done = true;
            }
        }
        if constexpr (joins_never_fork<PM>()) {
            if (!done && mode == LOAD_JOIN) {  // continuations only: no scan, no allocation, no block barrier
                TileLoad<TPT> cur, nxt;
                if (t0 < hi) tile_load<BS, TPT, PM>(c, t0, hi, mode, cur);
                bool jr_use = false;  // fib: the successor tile's join operands are prefetched
                for (; t0 < hi; t0 += step) {
                    const bool more = t0 + step < hi;
                    if (more) tile_load<BS, TPT, PM>(c, t0 + step, hi, mode, nxt);
                    join_tile<BS, TPT, PM>(c, sm, t0, cen, e, acc, par, cur, jr_use, more ? &nxt : nullptr);
                    jr_use = more;
                    if (more) cur = nxt;
                    par ^= 1;
                }
                done = true;
            }
        }
        if (!done) {
            TileLoad<TPT> cur, nxt;
            if (t0 < hi) tile_load<BS, TPT, PM>(c, t0, hi, mode, cur);
            const bool jr = mode == LOAD_JOIN;  // fib: prefetch the successor tile's join operands
            bool jr_use = false;
            for (; t0 < hi; t0 += step) {
                const bool more = t0 + step < hi;
                if (more) tile_load<BS, TPT, PM>(c, t0 + step, hi, mode, nxt);
                jn |= epoch_tile<BS, TPT, PM, UP>(c, ctl, sm, t0, hi, cen, base, ep, e, acc, par, mode, cur, solo, 0u,
                                                  jr_use, jr && more ? &nxt : nullptr).joined;
                jr_use = jr && more;
                if (more) cur = nxt;
                par ^= 1;
            }
        }
        trace_valid_add<BS>(c, e, acc.valid - v0, sm);
        if ((int32_t)e == c.stall_epoch && blockIdx.x == gridDim.x - 1) {  // test hook: never arrives
            if (blockIdx.x == 0 && threadIdx.x == 0) ctl->res0 = __ldcg(c.result);
            return;
        }
        if constexpr ((PM & PM_MAPS) == 0u) {  // the epoch word carries the counters Phase 3 needs
            if (!epoch_barrier<BS>(ctl, c.timeout_ns, sm, ep, jn)) break;
        } else {
            publish_join(ctl, ep, jn);
            if (!grid_sync_ep<BS>(ctl, &st.bar, c.timeout_ns, sm, ep)) break;
        }
        if (stamp) st.t_p2 = st.t_pt = st.t_mp = globaltimer();
        const unsigned long long mt = sm.ep_mt, me = sm.ep_me;
        if (mt | me) {  // the map operations of this epoch run before the next one (Sec. 5.2.4)
            if constexpr ((PM & PM_MS) != 0u) {
                if (needs_partition(mt)) {
                    partition_phase<BS>(c, mt, nullptr, 0u);
                    if (!grid_sync_ep<BS>(ctl, &st.bar, c.timeout_ns, sm, ep)) break;
                    if (stamp) st.t_pt = st.t_mp = globaltimer();
                }
            }
            if constexpr (PM == PM_SSSP) {  // the parts' claim buffers are in the dynamic shared memory
                map_phase<BS, PM, UP>(c, ctl, sm, ep, e, cen, base, mt, me, nullptr, 0u, ring,
                                      sssp_claim_cap<BS, TPT>());
            } else {
                map_phase<BS, PM, UP>(c, ctl, sm, ep, e, cen, base, mt, me);
            }
            if (!grid_sync_ep<BS>(ctl, &st.bar, c.timeout_ns, sm, ep)) break;
            if (stamp) st.t_mp = globaltimer();
        }
        // Phase 3: push the join range, then the fork range; or give the range back
        if (threadIdx.x == 0) phase3<BS>(c, ctl, sm, e, sm.ep_cnt, sm.ep_join, mt, me, st);
    }
    block_add_stats<BS>(blk, acc, sm);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->epochs = e;
        ctl->peak = st.peak;
        ctl->final_next = sm.next;
        ctl->forks = st.forks_total;
        ctl->t_end = globaltimer();
        ctl->res0 = __ldcg(c.result);  // final: the last epoch's writes came before its grid barrier
    }
}

// Returns k_persistent<BS, TPT, PM, UP> for a runtime (bs, tpt), or nullptr.
template <uint32_t PM, typename UP = NoUserProgram>
const void *persistent_kernel_for(int bs, int tpt) {
    switch (bs * 10 + tpt) {
    case 1281: return (const void *)k_persistent<128, 1, PM, UP>;
    case 1282: return (const void *)k_persistent<128, 2, PM, UP>;
    case 1284: return (const void *)k_persistent<128, 4, PM, UP>;
    case 2561: return (const void *)k_persistent<256, 1, PM, UP>;
    case 2562: return (const void *)k_persistent<256, 2, PM, UP>;
    case 2564: return (const void *)k_persistent<256, 4, PM, UP>;
    case 5121: return (const void *)k_persistent<512, 1, PM, UP>;
    case 5122: return (const void *)k_persistent<512, 2, PM, UP>;
    case 5124: return (const void *)k_persistent<512, 4, PM, UP>;
    case 10241: return (const void *)k_persistent<1024, 1, PM, UP>;
    case 10242: return (const void *)k_persistent<1024, 2, PM, UP>;
    case 10244: return (const void *)k_persistent<1024, 4, PM, UP>;
    default: return nullptr;
    }
}

// One definition per program, each in its own translation unit.
const void *persistent_kernel_fib(int bs, int tpt);
const void *persistent_kernel_ms(int bs, int tpt);
const void *persistent_kernel_nq(int bs, int tpt);
const void *persistent_kernel_bfs(int bs, int tpt);
const void *persistent_kernel_trav(int bs, int tpt);
const void *persistent_kernel_sssp(int bs, int tpt);
const void *persistent_kernel_fft(int bs, int tpt);

}  // namespace trees
