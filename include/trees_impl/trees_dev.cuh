// Device-side internals of libtrees: the task vector layout, the control
// block, the timed grid barrier and the block-wide scans the cooperative
// allocator is built from.
//
// Layout (Sec. 5.1.2, re-designed for coalescing on sm_103a): the task vector
// is a structure of arrays in HBM -- one u32 `code` column (epoch*NTT + type,
// footnote 2 of Sec. 5.1.2; 0 = no task), two u32 argument columns, a u32
// `link` column (first child slot of a join) and a u64 `result` column (the
// value an `emit` stores, Sec. 4.3.2).  A warp touching 32 consecutive slots
// reads or writes one 128-byte line per column.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../trees.h"

namespace trees {

constexpr uint32_t NTT = TREES_NUM_TASK_TYPES;  // NumTaskTypes of footnote 2, Sec. 5.1.2
constexpr int STK_CAP = 512;                    // epoch-range stack entries per job
constexpr int LEAF_MAX = 1024;                  // largest leaf a block sorts in shared memory
constexpr uint32_t FFT_LEAF_MAX = 16;           // largest FFT leaf a thread transforms in registers
constexpr uint32_t FFT_MAX_POINTS = 1u << 25;   // twiddle quotients 2k/M stay exact in fp32 (k < 2^24)
constexpr uint32_t FFT_CHUNK = 8;               // combine-map butterflies a thread keeps in flight
// Outputs per thread of a merge tile (Sec. 5.2.4's map operations, tiled by
// merge path) for a block of bs threads: odd counts keep the threads' probes
// and run heads on distinct shared-memory banks.  A full tile is bs *
// merge_mpt(bs) outputs, as many as two staged tiles fit in the 48 KB of
// static shared memory a block may hold; a tile of at most bs *
// merge_mpt_small(bs) outputs (the whole merge of two short runs) is merged
// with the smaller count so that fewer threads idle.
__host__ __device__ constexpr uint32_t merge_mpt(int bs) { return bs <= 256 ? 17u : bs <= 512 ? 7u : 3u; }
__host__ __device__ constexpr uint32_t merge_mpt_small(int bs) { return bs <= 256 ? 9u : bs <= 512 ? 5u : 3u; }
__host__ __device__ constexpr uint32_t merge_tile(int bs) { return (uint32_t)bs * merge_mpt(bs); }
// Words of one staged tile: A's and B's 16-byte chunks, packed.
__host__ __device__ constexpr uint32_t merge_stage(int bs) { return merge_tile(bs) + 16u; }
// Merge tiles staged per block (a ring of TMA buffers): one merging while the
// next streams in.
__host__ __device__ constexpr int merge_nst(int) { return 2; }
// Parts of a block that run BFS / SSSP expansion tiles independently, and the
// adjacency entries of one tile (a part's): 512-thread blocks run sixteen
// one-warp parts of 128-entry tiles, 1024-thread blocks eight parts of 256
// (a part of several warps syncs on a named barrier, ids 1..15), smaller
// blocks four (two at 128 threads) of 512; a part's threads take 2-8 entries
// each and the parts' records fill the same shared union.  More parts are
// more tile chains in flight per SM (R-MAT 22, one call each: at 512 x 2 BFS
// 0.918 ms with 4 parts x 512, 0.844 with 8 x 256, 0.785 with 16 x 128; SSSP
// 512 x 1 2.52, 2.38, 2.27 ms); at 256 threads 4 parts x 256 were slower than
// 4 x 512 (BFS 0.94 -> 0.98 ms).
#define EXPAND_PARTS(BS) ((BS) == 512 ? 16u : (BS) >= 1024 ? 8u : (BS) >= 256 ? 4u : 2u)
__host__ __device__ constexpr uint32_t expand_tile_len(int bs) { return bs == 512 ? 128u : bs >= 1024 ? 256u : 512u; }
constexpr uint32_t JR_SLOTS = 1024;             // tile slots whose join operands can be prefetched
constexpr uint32_t SMP_SHIFT = 6;               // mergesort splitter samples: every 64th key of a run
constexpr int MCHUNK = 64;                      // merge tiles a block resolves at once
constexpr unsigned long long CTR_LOW_MASK = (1ull << 40) - 1;  // map counters: (descs << 40) | units

// MAP_FFT: the combines of an FFT epoch; they need no descriptors (fft_combine_map).
// MAP_USER: a user program's map, one tile per unit (mt_c holds the scheduling slot).
enum MapKind : uint32_t { MAP_LEAF_SORT = 1, MAP_MERGE = 2, MAP_EXPAND = 3, MAP_FFT = 4, MAP_USER = 5 };
constexpr int TPT_MAX = 4;                      // largest number of slots a thread takes per tile
constexpr int NBLK_STATS = 8192;                // per-block statistics slots

struct Range {
    uint32_t cen, lo, hi;  // epoch number and NDRange [lo, hi) (Sec. 5.1.2)
    uint32_t join;         // 1: a join range revisited (continuations), 0: freshly forked tasks
};
static_assert(sizeof(Range) == 16, "ranges move as 16-byte vectors");

// The job a single-job run executes (copied into the control block per run).
struct RunParams {
    int32_t program;
    uint32_t n, cutoff, leaf;
    uint32_t *keys, *scratch;
    const int32_t *row_ptr, *col;
    int32_t *level;
    int32_t nv;
    const int32_t *left, *right;
    int32_t *visit_epoch;
    const uint32_t *weight;    // SSSP edge weights (aligned with col)
    unsigned long long *dist;  // SSSP distances
    uint32_t *sched;           // SSSP: the last epoch each vertex was forked for
    // SSSP: per vertex, (e + 1) << 40 | the largest distance of it that a relaxation of its
    // out-edges used in epoch e, e its last relax epoch (0 = never relaxed; context-owned)
    unsigned long long *used;
    // BFS: one bit per vertex, set once the vertex is claimed (context-owned): the expansion
    // probes it before the claim's CAS on `level`
    uint32_t *visited;
    const float2 *fx;          // FFT input, N complex points
    float2 *fX;                // FFT output
    uint32_t lgn;              // FFT: log2 N
    void *up[TREES_USER_PARAMS];               // user program parameters
    unsigned long long uv[TREES_USER_PARAMS];
};

// Read-only during a run: where everything lives.
struct Conf {
    uint32_t *code, *a0, *a1, *link;
    unsigned long long *result;
    uint32_t cap;
    // tiled map list: one descriptor per map operation, `units` tiles each
    uint32_t *mt_kind, *mt_a, *mt_b, *mt_c, *mt_job, *mt_tilebase, *mt_split;
    // element map list (BFS / SSSP expansion): one descriptor per vertex, one unit per edge;
    // me_v = the vertex's first adjacency index, me_src = the vertex
    uint32_t *me_v, *me_base, *me_job, *me_tfd, *me_src;
    uint32_t mcap;
    trees_epoch_t *trace;
    uint32_t *trace_valid;
    uint32_t trace_cap;
    int32_t trace_on;
    uint32_t max_epochs;
    int32_t stall_epoch;
    unsigned long long timeout_ns;
    Range *gstack;
    uint32_t gstack_cap;
    // single-job mergesort: smp[p >> SMP_SHIFT] = the key at position p (p a multiple of 64) of the
    // runs the last map phase wrote, for the next partition's searches; null otherwise
    uint32_t *smp;
    RunParams rp;
};

// Mutable control block.  The per-epoch counters are triple-buffered by
// epoch index: epoch e allocates from slot e%3, block 0 clears slot (e+1)%3
// during epoch e (its last readers finished before the barrier that opened
// epoch e), so one grid barrier per epoch is enough.
//
// ew[q], the epoch word of slot q: the high 32 bits are the epoch's forks
// (nextFreeCore - oldNextFreeCore, the counter the cooperative allocation
// adds to); the low 32 bits serve the epoch barrier of the programs without
// maps (epoch_barrier): arrivals in bits 0..15, the blocks that joined in
// bits 16..30, and bit 31 set once any device-side error was raised.
constexpr unsigned long long EW_ARRIVALS = 0xFFFFull, EW_ERROR = 0x80000000ull;
constexpr uint32_t EW_JOIN_SHIFT = 16;
struct Ctl {
    unsigned int bar_count;          // monotonic arrival counter of the grid barrier
    unsigned int pad0[63];
    unsigned long long ew[3];        // epoch words (above)
    unsigned int join[3];            // joinScheduled (schedulers and programs that read it apart)
    unsigned long long mt_ctr[3];    // tiled maps: (descriptors << 40) | tiles
    unsigned long long me_ctr[3];    // element maps: (descriptors << 40) | elements
    int err;                         // first device-side error (sticky)
    unsigned int err_epoch;
    unsigned long long res0;         // persistent scheduler: slot 0's result at the end of the run, beside
                                     // err so that one 16-byte copy brings both to the host (trees_sync)
    unsigned long long tasks, joins, maps, forks;
    unsigned long long t_start, t_end;
    unsigned int epochs, peak, final_next, pad1;
    // scheduler state for the graph and host-loop schedulers
    unsigned int g_cen, g_lo, g_hi, g_base, g_e, g_next, g_sp, g_stop;
    unsigned int g_rjoin, pad2;      // the persistent scheduler's solo runs publish the same state
};

struct Dev {
    Ctl ctl;
    Conf conf;
};

// ------------------------------------------------------------------ helpers

__device__ __forceinline__ uint32_t task_type(uint32_t code, uint32_t cen) {
    // active iff code in [cen*NTT + 1, (cen+1)*NTT]  (footnote 2, Sec. 5.1.2)
    const uint32_t d = code - (cen * NTT + 1u);
    return d < NTT ? d + 1u : 0u;
}

__device__ __forceinline__ uint32_t enc(uint32_t epoch, uint32_t type) { return epoch * NTT + type; }

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int *p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void red_release_add(unsigned int *p, unsigned int v) {
    asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

template <typename T>
__device__ __forceinline__ T vload(const T *p) {
    return *(const volatile T *)p;
}

// The allocation counter of epoch slot ep: the high half of its epoch word.
__host__ __device__ __forceinline__ unsigned int *fork_ctr(Ctl *ctl, uint32_t ep) {
    return reinterpret_cast<unsigned int *>(&ctl->ew[ep]) + 1;
}

__device__ __forceinline__ void set_err(Ctl *ctl, int code, uint32_t epoch) {
    if (atomicCAS(&ctl->err, 0, code) == 0) ctl->err_epoch = epoch;
    for (int q = 0; q < 3; ++q) atomicOr(&ctl->ew[q], EW_ERROR);  // seen by the next epoch barrier
}

// Clears epoch slot q for reuse, keeping its error flag.
__device__ __forceinline__ void clear_epoch_slot(Ctl *ctl, uint32_t q) {
    atomicAnd(&ctl->ew[q], EW_ERROR);
    ctl->join[q] = 0u;
    ctl->mt_ctr[q] = 0ull;
    ctl->me_ctr[q] = 0ull;
}

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// ------------------------------------------------------------------ shared memory

template <int BS>
struct Smem {
    static constexpr int NW = BS / 32;
    unsigned int w32[NW];
    unsigned int wflag[NW];
    unsigned int wv[2][TPT_MAX][NW];  // vector scan words, double-buffered by tile parity
    unsigned int wvf[2][NW];
    unsigned long long w64a[NW];
    unsigned long long w64b[NW];
    unsigned int flags;
    unsigned int bc32[32];                // broadcast words (two per block part in the expansion tiles)
    unsigned int pcnt[16];                // entries waiting in each block part's claim buffer (bfs_claim_flush, sssp_claim_flush)
    unsigned long long bc64[4];
    int bar_ok;
    unsigned long long mbar[merge_nst(BS)];  // mbarriers of the merge stage buffers
    unsigned long long mvalid;            // which entries of mtab are merge tiles
    uint32_t mtab[MCHUNK][12];            // the block's next merge tiles, resolved in parallel
    unsigned int ep_cnt, ep_join;         // the epoch's counters, read right after its barrier
    unsigned long long ep_mt, ep_me;
    // replicated epoch-range stack and scheduler state (persistent scheduler)
    Range stk[STK_CAP];
    int sp;
    uint32_t next, cen, lo, hi, base, rjoin;
    int stop;
    unsigned int solo_late;  // a solo run has used its share of the barrier timeout
    union alignas(16) {
        uint32_t mg[merge_nst(BS)][merge_stage(BS)];  // staged merge tile inputs (TMA destinations)
        struct {  // one set of records per block part (its current expansion tile)
            uint32_t base[EXPAND_PARTS(BS)][expand_tile_len(BS) + 2];
            uint32_t v[EXPAND_PARTS(BS)][expand_tile_len(BS) + 2];
            unsigned long long d[EXPAND_PARTS(BS)][expand_tile_len(BS) + 2];  // SSSP: the source's distance, read once per tile
        } ex;
        unsigned long long jr[2][JR_SLOTS][2];  // fib joins: the next tile's children's results, prefetched
    } u;
};

static_assert(sizeof(Smem<128>::u) >= TREES_USER_SMEM_BYTES && sizeof(Smem<1024>::u) >= TREES_USER_SMEM_BYTES,
              "a user map unit gets the shared union");
static_assert(sizeof(Smem<256>) <= 48 * 1024 && sizeof(Smem<512>) <= 48 * 1024 && sizeof(Smem<1024>) <= 48 * 1024,
              "a block's static shared memory is limited to 48 KB");

// ------------------------------------------------------------------ scans

__device__ __forceinline__ uint32_t warp_incl_u32(uint32_t x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

__device__ __forceinline__ unsigned long long warp_incl_u64(unsigned long long x) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Exclusive block scan of v; *total gets the block sum, *any the block-wide OR
// of pred.  Two __syncthreads; the caller must __syncthreads before the next
// scan reuses the shared words.
template <int BS>
__device__ __forceinline__ uint32_t block_scan_u32(uint32_t v, int pred, uint32_t *total, int *any, Smem<BS> &sm) {
    constexpr int NW = BS / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const uint32_t inc = warp_incl_u32(v);
    const unsigned int bal = __ballot_sync(0xffffffffu, pred);
    if (lane == 31) sm.w32[wid] = inc;
    if (lane == 0) sm.wflag[wid] = bal != 0u;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = lane < NW ? sm.w32[lane] : 0u;
        const unsigned int f = __ballot_sync(0xffffffffu, lane < NW ? sm.wflag[lane] : 0u);
        w = warp_incl_u32(w);
        if (lane < NW) sm.w32[lane] = w;
        if (lane == 0) sm.flags = f != 0u;
    }
    __syncthreads();
    *total = sm.w32[NW - 1];
    *any = (int)sm.flags;
    return (wid ? sm.w32[wid - 1] : 0u) + inc - v;
}

// Exclusive block scan of K values per thread at once (one scan per k), with
// the block-wide OR of pred.  The shared words are double-buffered by `par`,
// so consecutive tiles need no barrier between them.
template <int BS, int K>
__device__ __forceinline__ void block_scan_vec(const uint32_t (&v)[K], uint32_t (&ex)[K], uint32_t (&tot)[K], int pred,
                                               int *any, Smem<BS> &sm, int par) {
    constexpr int NW = BS / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t inc[K];
#pragma unroll
    for (int k = 0; k < K; ++k) inc[k] = warp_incl_u32(v[k]);
    const unsigned int bal = __ballot_sync(0xffffffffu, pred);
    if (lane == 31) {
#pragma unroll
        for (int k = 0; k < K; ++k) sm.wv[par][k][wid] = inc[k];
    }
    if (lane == 0) sm.wvf[par][wid] = bal != 0u;
    __syncthreads();
    // one barrier: every thread sums the warp totals itself (broadcast reads); buffer `par` is
    // written again two tiles later, after a barrier every thread reaches only past these reads
    uint32_t pre[K], all[K], f = 0u;
#pragma unroll
    for (int k = 0; k < K; ++k) pre[k] = all[k] = 0u;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
#pragma unroll
        for (int k = 0; k < K; ++k) {
            const uint32_t x = sm.wv[par][k][w];
            all[k] += x;
            pre[k] += w < wid ? x : 0u;
        }
        f |= sm.wvf[par][w];
    }
#pragma unroll
    for (int k = 0; k < K; ++k) {
        tot[k] = all[k];
        ex[k] = pre[k] + inc[k] - v[k];
    }
    *any = (int)(f != 0u);
}

// Exclusive block scan of two u64 values at once.
template <int BS>
__device__ __forceinline__ void block_scan_u64x2(unsigned long long a, unsigned long long b, unsigned long long *ea,
                                                 unsigned long long *eb, unsigned long long *ta,
                                                 unsigned long long *tb, Smem<BS> &sm) {
    constexpr int NW = BS / 32;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned long long ia = warp_incl_u64(a), ib = warp_incl_u64(b);
    if (lane == 31) {
        sm.w64a[wid] = ia;
        sm.w64b[wid] = ib;
    }
    __syncthreads();
    if (wid == 0) {
        unsigned long long x = lane < NW ? sm.w64a[lane] : 0ull;
        unsigned long long y = lane < NW ? sm.w64b[lane] : 0ull;
        x = warp_incl_u64(x);
        y = warp_incl_u64(y);
        if (lane < NW) {
            sm.w64a[lane] = x;
            sm.w64b[lane] = y;
        }
    }
    __syncthreads();
    *ta = sm.w64a[NW - 1];
    *tb = sm.w64b[NW - 1];
    *ea = (wid ? sm.w64a[wid - 1] : 0ull) + ia - a;
    *eb = (wid ? sm.w64b[wid - 1] : 0ull) + ib - b;
}

// ------------------------------------------------------------------ grid barrier

// One grid-wide barrier (Tenet 1's bulk synchronisation).  Thread 0 of each
// block adds 1 to a monotonic counter with release semantics and spins with
// acquire loads until the counter reaches (barrier index) * gridDim.x.  The
// spin is bounded by timeout_ns of globaltimer: past it the block records
// TREES_ERR_TIMEOUT and returns false instead of waiting forever.
template <int BS>
__device__ __forceinline__ bool grid_sync(Ctl *ctl, uint32_t *bar_idx, unsigned long long timeout_ns, Smem<BS> &sm) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t idx = ++(*bar_idx);
        const unsigned int target = idx * gridDim.x;
        red_release_add(&ctl->bar_count, 1u);  // release: covers the block's writes ordered by bar.sync
        int ok = 1;
        uint32_t spins = 0;
        uint64_t t0 = 0;
        while ((int)(ld_acquire(&ctl->bar_count) - target) < 0) {
            if ((++spins & 63u) == 0u) {
                const uint64_t now = globaltimer();
                if (t0 == 0) {
                    t0 = now;
                } else if (now - t0 > timeout_ns) {
                    set_err(ctl, TREES_ERR_TIMEOUT, idx);
                    ok = 0;
                    break;
                }
            }
        }
        fence_acq_rel();  // acquire for the whole SM: no stale L1 line of data written before the barrier
        // one block-uniform decision: stop on a timeout or on any error raised before the barrier
        sm.bar_ok = ok && vload(&ctl->err) == 0;
    }
    __syncthreads();
    return sm.bar_ok != 0;
}

// ------------------------------------------------------------------ TMA bulk copies

__device__ __forceinline__ uint32_t smem_addr(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(unsigned long long *bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Arrive once and announce `bytes` of asynchronous copies on this phase.
__device__ __forceinline__ void mbar_arrive_expect(unsigned long long *bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Bounded wait for the phase with the given parity; false if it timed out.
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, uint32_t parity, unsigned long long timeout_ns) {
    const uint32_t a = smem_addr(bar);
    uint64_t t0 = 0;
    for (uint32_t spin = 0;; ++spin) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity)
            : "memory");
        if (done) return true;
        if ((spin & 15u) == 15u) {
            const uint64_t now = globaltimer();
            if (t0 == 0) t0 = now;
            else if (now - t0 > timeout_ns) return false;
        }
    }
}

// One-dimensional bulk copy global -> shared (16-byte aligned, multiple of
// 16 bytes), completing on `bar`.
__device__ __forceinline__ void tma_load_1d(void *dst_smem, const void *src, uint32_t bytes, unsigned long long *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst_smem)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// 8-byte asynchronous copy global -> shared (no register holds the data);
// this thread's copies since the last commit form one group.
__device__ __forceinline__ void cp_async_8(void *dst_smem, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(dst_smem)), "l"(src) : "memory");
}
// The same with 4 bytes.
__device__ __forceinline__ void cp_async_4(void *dst_smem, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst_smem)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// This thread's committed copies have landed.
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
// All but this thread's N most recent groups have landed.
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Orders this thread's view of global memory (including writes it acquired
// from other SMs) before its later async-proxy (bulk copy) reads of it.
__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// One-dimensional bulk copy shared -> global (both 16-byte aligned, a
// multiple of 16 bytes), tracked by this thread's bulk async-groups.
__device__ __forceinline__ void tma_store_1d(void *dst, const void *src_smem, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(smem_addr(src_smem)),
                 "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}

// This thread's bulk stores have finished reading their shared-memory sources.
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }

// This thread's bulk stores are complete, their global writes ordered before
// its later generic memory operations.
__device__ __forceinline__ void bulk_wait_all() {
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

// grid_sync, then (thread 0, same round trip) the counters of epoch slot ep
// into shared memory: forks, joinScheduled and both map counters.
template <int BS>
__device__ __forceinline__ bool grid_sync_ep(Ctl *ctl, uint32_t *bar_idx, unsigned long long timeout_ns, Smem<BS> &sm,
                                             uint32_t ep) {
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t idx = ++(*bar_idx);
        const unsigned int target = idx * gridDim.x;
        red_release_add(&ctl->bar_count, 1u);  // release: covers the block's writes ordered by bar.sync
        int ok = 1;
        uint32_t spins = 0;
        uint64_t t0 = 0;
        while ((int)(ld_acquire(&ctl->bar_count) - target) < 0) {
            if ((++spins & 63u) == 0u) {
                const uint64_t now = globaltimer();
                if (t0 == 0) {
                    t0 = now;
                } else if (now - t0 > timeout_ns) {
                    set_err(ctl, TREES_ERR_TIMEOUT, idx);
                    ok = 0;
                    break;
                }
            }
        }
        fence_acq_rel();  // acquire for the whole SM: no stale L1 line of data written before the barrier
        const int err = vload(&ctl->err);
        sm.ep_cnt = vload(fork_ctr(ctl, ep));
        sm.ep_join = vload(&ctl->join[ep]);
        sm.ep_mt = vload(&ctl->mt_ctr[ep]);
        sm.ep_me = vload(&ctl->me_ctr[ep]);
        sm.bar_ok = ok && err == 0;
    }
    __syncthreads();
    return sm.bar_ok != 0;
}

// The barrier that closes Phase 2 of an epoch, for programs without maps:
// thread 0 of each block adds one arrival (and, if any of its threads
// joined, one joined block) to the low half of epoch slot ep's word with
// release semantics and polls the whole 64-bit word with acquire loads until
// every block has arrived; the same load that ends the wait delivers the
// epoch's forks (the high half), its join flag and the error flag, so no
// further round trip is needed before Phase 3.  Bounded by timeout_ns like
// grid_sync.  Every thread calls it; returns false on a timeout or error.
template <int BS>
__device__ __forceinline__ bool epoch_barrier(Ctl *ctl, unsigned long long timeout_ns, Smem<BS> &sm, uint32_t ep,
                                              bool joined) {
    const int jb = __syncthreads_or(joined);  // also orders the block's writes before thread 0's release
    if (threadIdx.x == 0) {
        red_release_add(reinterpret_cast<unsigned int *>(&ctl->ew[ep]), 1u + (jb ? 1u << EW_JOIN_SHIFT : 0u));
        int ok = 1;
        uint32_t spins = 0;
        uint64_t t0 = 0;
        unsigned long long w;
        while (((w = ld_acquire_u64(&ctl->ew[ep])) & EW_ARRIVALS) < gridDim.x) {
            if ((++spins & 63u) == 0u) {
                const uint64_t now = globaltimer();
                if (t0 == 0) {
                    t0 = now;
                } else if (now - t0 > timeout_ns) {
                    set_err(ctl, TREES_ERR_TIMEOUT, ep);
                    ok = 0;
                    break;
                }
            }
        }
        fence_acq_rel();  // acquire for the whole SM: no stale L1 line of data written before the barrier
        sm.ep_cnt = (uint32_t)(w >> 32);
        sm.ep_join = (uint32_t)((w >> EW_JOIN_SHIFT) & 0x7FFFull) != 0u;
        sm.ep_mt = 0ull;
        sm.ep_me = 0ull;
        sm.bar_ok = ok && (w & EW_ERROR) == 0ull;
    }
    __syncthreads();
    return sm.bar_ok != 0;
}

}  // namespace trees
